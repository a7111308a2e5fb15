// Host-side geometry of RSRS: the adaptive quad/octree of Sec. 3 and the
// processing schedule of Algorithm 1 (levels, colours, active sizes).
#pragma once
#include <cstdint>
#include <vector>

namespace rsrs {

constexpr int kLmax = 20;  // points are binned on a 2^20 integer grid per side

struct Box {
  int level = 0;
  int64_t coord[3] = {0, 0, 0};
  int parent = -1;
  std::vector<int> children;  // Morton order of the child index (x bit lowest)
  std::vector<int64_t> pts;   // original point indices, ascending
  int64_t first_pos = 0;      // first tree position of the box's points
  uint64_t morton = 0;
  bool leaf() const { return children.empty(); }
};

struct Tree {
  int d = 2;
  int64_t n = 0;
  int leaf_cap = 0;
  int depth = 0;
  std::vector<Box> boxes;
  std::vector<std::vector<int>> levels;  // box ids per level, Morton-sorted
  std::vector<int64_t> perm;             // tree position -> original index
  std::vector<int64_t> pos;              // original index -> tree position
  std::vector<double> pts_tree;          // points in tree order, n x d
};

// One compressed box of Algorithm 1, in processing order.
struct Step {
  int box;
  int level;
  int colour;
  int64_t b, n, kp, r;
  std::vector<int> nbrs;          // neighbour box ids, ascending first_pos
  std::vector<int64_t> nbr_len;   // active count of each neighbour when the box is processed
};

struct Schedule {
  int k = 0, p = 0;
  std::vector<Step> steps;
  // [level][colour] -> range of steps
  std::vector<std::vector<std::pair<int, int>>> groups;
  std::vector<int64_t> act0;  // per box: active count when its level starts
  std::vector<int64_t> act1;  // per box: active count after its level
  std::vector<int64_t> root;  // tree positions of B_t, ascending
  int64_t max_l = 0;
  int64_t s_req = 0;
};

bool build_tree(const double* pts, int64_t n, int d, int leaf_cap, Tree& t);
void build_schedule(const Tree& t, int k, int p, Schedule& s);
bool boxes_touch(const Box& a, const Box& b, int d);

}  // namespace rsrs
