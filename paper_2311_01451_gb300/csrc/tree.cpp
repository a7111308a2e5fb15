// Adaptive 2^d-tree, 2:1 balance, neighbour lists and the processing schedule
// of Algorithm 1 (Sec. 3, Sec. 4.4) with the sample bound of Sec. 4.5.
//
// Rules (the paper leaves them open; the CPU oracle follows the same ones):
//  * root cube [0,1]^d if all points lie in it, else the bounding cube anchored
//    at the per-dimension minimum; integer coordinates floor((x-lo)/side*2^20);
//  * a box with more than leaf_cap points is split into its non-empty children;
//  * 2:1 balance: split a leaf while an adjacent leaf is >= 2 levels deeper;
//  * at level l the active points are partitioned among the level-l boxes and
//    the coarser leaves; neighbours are those that touch the box (closed cubes);
//  * a box is compressed when it holds more than k active points and its far
//    field is not empty; same-level boxes are processed colour by colour, the
//    colours from a greedy colouring in Morton order where boxes with
//    intersecting closed neighbourhoods conflict; Morton order inside a colour;
//  * s_req = max(max over compressed boxes of b + n + k + p, |B_t| + p): the root's least-squares
//    problem is oversampled by p like the boxes', which keeps Omega_Bt well conditioned.
#include "tree.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <set>

namespace rsrs {

static uint64_t morton_key(const int64_t* c, int d) {
  uint64_t key = 0;
  for (int bit = 0; bit <= kLmax; ++bit)
    for (int dim = 0; dim < d; ++dim)
      key |= (uint64_t)((c[dim] >> bit) & 1) << (bit * d + dim);
  return key;
}

bool boxes_touch(const Box& a, const Box& b, int d) {
  int L = std::max(a.level, b.level);
  int sa = L - a.level, sb = L - b.level;
  for (int dim = 0; dim < d; ++dim) {
    int64_t loa = a.coord[dim] << sa, hia = (a.coord[dim] + 1) << sa;
    int64_t lob = b.coord[dim] << sb, hib = (b.coord[dim] + 1) << sb;
    if (loa > hib || lob > hia) return false;
  }
  return true;
}

namespace {

struct Builder {
  Tree& t;
  std::vector<int64_t> ic;  // n x d integer coordinates
  explicit Builder(Tree& tt) : t(tt) {}

  int new_box(int level, const int64_t* coord, int parent, std::vector<int64_t>&& pts) {
    Box b;
    b.level = level;
    for (int i = 0; i < t.d; ++i) b.coord[i] = coord[i];
    b.parent = parent;
    b.pts = std::move(pts);
    b.morton = morton_key(b.coord, t.d);
    t.boxes.push_back(std::move(b));
    return (int)t.boxes.size() - 1;
  }

  void split(int id) {
    const int d = t.d;
    int level = t.boxes[id].level;
    int shift = kLmax - level - 1;
    int nch = 1 << d;
    std::vector<std::vector<int64_t>> part(nch);
    for (int64_t p : t.boxes[id].pts) {
      int c = 0;
      for (int dim = 0; dim < d; ++dim) {
        int64_t cc = ic[p * d + dim] >> shift;
        c |= (int)(cc - 2 * t.boxes[id].coord[dim]) << dim;
      }
      part[c].push_back(p);  // pts are ascending, so each part stays ascending
    }
    for (int c = 0; c < nch; ++c) {
      if (part[c].empty()) continue;
      int64_t coord[3];
      for (int dim = 0; dim < d; ++dim) coord[dim] = 2 * t.boxes[id].coord[dim] + ((c >> dim) & 1);
      int cid = new_box(level + 1, coord, id, std::move(part[c]));
      t.boxes[id].children.push_back(cid);
    }
  }
};

}  // namespace

bool build_tree(const double* pts, int64_t n, int d, int leaf_cap, Tree& t) {
  if (n <= 0 || (d != 2 && d != 3) || leaf_cap <= 0) return false;
  t = Tree();
  t.d = d;
  t.n = n;
  t.leaf_cap = leaf_cap;
  double lo[3], hi[3];
  for (int dim = 0; dim < d; ++dim) {
    lo[dim] = INFINITY;
    hi[dim] = -INFINITY;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int dim = 0; dim < d; ++dim) {
      double x = pts[i * d + dim];
      if (!std::isfinite(x)) return false;
      lo[dim] = std::min(lo[dim], x);
      hi[dim] = std::max(hi[dim], x);
    }
  bool unit = true;
  for (int dim = 0; dim < d; ++dim) unit = unit && lo[dim] >= 0.0 && hi[dim] <= 1.0;
  double side = 1.0;
  if (unit) {
    for (int dim = 0; dim < d; ++dim) lo[dim] = 0.0;
  } else {
    side = 0.0;
    for (int dim = 0; dim < d; ++dim) side = std::max(side, hi[dim] - lo[dim]);
    if (side <= 0.0) side = 1.0;
  }
  Builder B(t);
  B.ic.resize((size_t)n * d);
  const double scale = (double)(int64_t(1) << kLmax);
  const int64_t cmax = (int64_t(1) << kLmax) - 1;
  for (int64_t i = 0; i < n; ++i)
    for (int dim = 0; dim < d; ++dim) {
      double u = std::floor(((pts[i * d + dim] - lo[dim]) / side) * scale);
      int64_t c = (int64_t)std::max(0.0, std::min(u, (double)cmax));
      B.ic[i * d + dim] = c;
    }
  {
    std::vector<int64_t> all(n);
    std::iota(all.begin(), all.end(), 0);
    int64_t zero[3] = {0, 0, 0};
    B.new_box(0, zero, -1, std::move(all));
  }
  std::vector<int> stack = {0};
  while (!stack.empty()) {
    int id = stack.back();
    stack.pop_back();
    if ((int64_t)t.boxes[id].pts.size() > leaf_cap && t.boxes[id].level < kLmax) {
      B.split(id);
      for (int c : t.boxes[id].children) stack.push_back(c);
    }
  }
  // 2:1 balance between adjacent leaves
  for (;;) {
    std::vector<int> leaves;
    for (int i = 0; i < (int)t.boxes.size(); ++i)
      if (t.boxes[i].leaf()) leaves.push_back(i);
    std::vector<int> to_split;
    for (int a : leaves) {
      for (int c : leaves) {
        if (t.boxes[c].level >= t.boxes[a].level + 2 && boxes_touch(t.boxes[a], t.boxes[c], d)) {
          to_split.push_back(a);
          break;
        }
      }
    }
    if (to_split.empty()) break;
    for (int a : to_split) B.split(a);
  }
  // tree order: depth first, children in Morton order, points ascending in a leaf
  t.perm.clear();
  t.perm.reserve(n);
  std::vector<int> dfs = {0};
  // iterative pre-order traversal
  while (!dfs.empty()) {
    int id = dfs.back();
    dfs.pop_back();
    Box& b = t.boxes[id];
    b.first_pos = (int64_t)t.perm.size();
    if (b.leaf()) t.perm.insert(t.perm.end(), b.pts.begin(), b.pts.end());
    for (int i = (int)b.children.size() - 1; i >= 0; --i) dfs.push_back(b.children[i]);
  }
  t.pos.assign(n, 0);
  for (int64_t q = 0; q < n; ++q) t.pos[t.perm[q]] = q;
  t.depth = 0;
  for (auto& b : t.boxes) t.depth = std::max(t.depth, b.level);
  t.levels.assign(t.depth + 1, {});
  for (int i = 0; i < (int)t.boxes.size(); ++i) t.levels[t.boxes[i].level].push_back(i);
  for (auto& lv : t.levels)
    std::sort(lv.begin(), lv.end(), [&](int a, int b) { return t.boxes[a].morton < t.boxes[b].morton; });
  t.pts_tree.resize((size_t)n * d);
  for (int64_t q = 0; q < n; ++q)
    for (int dim = 0; dim < d; ++dim) t.pts_tree[q * d + dim] = pts[t.perm[q] * d + dim];
  return true;
}

void build_schedule(const Tree& t, int k, int p, Schedule& s) {
  s = Schedule();
  s.k = k;
  s.p = p < 0 ? k : p;
  const int nb = (int)t.boxes.size();
  s.act0.assign(nb, 0);
  s.act1.assign(nb, 0);
  for (int i = 0; i < nb; ++i)
    if (t.boxes[i].leaf()) s.act0[i] = s.act1[i] = (int64_t)t.boxes[i].pts.size();
  std::vector<int64_t> cur(nb, 0);  // running active count
  for (int i = 0; i < nb; ++i) cur[i] = s.act0[i];
  s.groups.assign(t.depth + 1, {});
  std::vector<int> coarse_leaves;  // leaves at levels < current level
  for (int level = t.depth; level >= 1; --level) {
    const auto& boxes = t.levels[level];
    for (int b : boxes)
      if (!t.boxes[b].leaf()) {
        int64_t a = 0;
        for (int c : t.boxes[b].children) a += s.act1[c];
        s.act0[b] = a;
        cur[b] = a;
      }
    coarse_leaves.clear();
    for (int i = 0; i < nb; ++i)
      if (t.boxes[i].leaf() && t.boxes[i].level < level) coarse_leaves.push_back(i);
    std::vector<int> cands(boxes.begin(), boxes.end());
    cands.insert(cands.end(), coarse_leaves.begin(), coarse_leaves.end());
    // neighbours of each level-l box
    std::vector<std::vector<int>> nbr(boxes.size());
    for (size_t i = 0; i < boxes.size(); ++i) {
      const Box& bx = t.boxes[boxes[i]];
      for (int c : cands)
        if (c != boxes[i] && boxes_touch(bx, t.boxes[c], t.d)) nbr[i].push_back(c);
      std::sort(nbr[i].begin(), nbr[i].end(),
                [&](int a, int b) { return t.boxes[a].first_pos < t.boxes[b].first_pos; });
    }
    // compressed boxes (Morton order, as `boxes`)
    std::vector<int> comp;  // index into boxes
    for (size_t i = 0; i < boxes.size(); ++i)
      if (cur[boxes[i]] > k && cands.size() > 1 + nbr[i].size()) comp.push_back((int)i);
    // greedy colouring: conflict when closed neighbourhoods intersect
    std::vector<std::vector<int>> members(nb);  // candidate box -> compressed boxes containing it
    for (int i : comp) {
      members[boxes[i]].push_back(i);
      for (int c : nbr[i]) members[c].push_back(i);
    }
    std::vector<int> colour(boxes.size(), -1);
    int ncol = 0;
    for (int i : comp) {
      std::set<int> used;
      auto mark = [&](int c) {
        for (int o : members[c])
          if (colour[o] >= 0) used.insert(colour[o]);
      };
      mark(boxes[i]);
      for (int c : nbr[i]) mark(c);
      int col = 0;
      while (used.count(col)) ++col;
      colour[i] = col;
      ncol = std::max(ncol, col + 1);
    }
    s.groups[level].assign(ncol, {0, 0});
    for (int col = 0; col < ncol; ++col) {
      int first = (int)s.steps.size();
      for (int i : comp) {
        if (colour[i] != col) continue;
        int b = boxes[i];
        Step st;
        st.box = b;
        st.level = level;
        st.colour = col;
        st.b = cur[b];
        st.nbrs = nbr[i];
        st.n = 0;
        for (int c : nbr[i]) {
          st.nbr_len.push_back(cur[c]);
          st.n += cur[c];
        }
        st.kp = std::min<int64_t>(k, st.b);
        st.r = st.b - st.kp;
        s.max_l = std::max(s.max_l, st.b + st.n);
        cur[b] = st.kp;
        s.steps.push_back(std::move(st));
      }
      s.groups[level][col] = {first, (int)s.steps.size()};
    }
    for (int b : boxes) s.act1[b] = cur[b];
  }
  // B_t: what stays active after level 1 (or everything if the root is a leaf)
  s.root.clear();
  if (t.depth == 0) {
    for (int64_t q = 0; q < t.n; ++q) s.root.push_back(q);
  }
  int64_t root_size = 0;
  if (t.depth >= 1)
    for (int b : t.levels[1]) root_size += s.act1[b];
  else
    root_size = t.n;
  s.s_req = std::max<int64_t>(s.steps.empty() ? 0 : s.max_l + s.k + s.p, root_size + s.p);
  s.root.resize(root_size);  // filled with tree positions by the device build
}

}  // namespace rsrs
