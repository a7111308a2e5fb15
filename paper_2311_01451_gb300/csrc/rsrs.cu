// librsrs: C ABI, build driver (Algorithm 1), solve/apply sweeps (eqs. Afact,
// Ainvfact) and FP64 iterative refinement.
//
// All sizes of Algorithm 1 (|B_act|, |N_act|, k', r per box) follow from the
// tree alone, so the whole launch sequence is planned on the host before any
// device work: per (level, colour) group a descriptor table, the segment lists
// that assemble active and near-field index lists on the device, and the
// workspace offsets.  Only the identities of skeleton/redundant points are
// data-dependent, and they stay on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

using namespace rsrs;

struct rsrs_tree {
  Tree t;
};

// One problem's boxes inside a (level, colour) launch group, in processing order.
struct GroupView {
  int level, colour;
  int64_t desc_off;        // first descriptor of this problem in the shared descriptor array
  std::vector<BoxDesc> h;  // host copies
  int max_r;
};

// Device memory shared by the factors of one build (one or several problems).
struct Shared {
  std::vector<void*> ptrs;
  // builds with opts.use_graph: the captured launch sequence (replayed by rsrs_refactor), the
  // device word its Philox draws take their key from, and its status word
  cudaGraphExec_t exec = nullptr;
  uint64_t* seed_dev = nullptr;
  int* err_dev = nullptr;
  ~Shared() {
    if (exec) cudaGraphExecDestroy(exec);
    for (void* p : ptrs) cudaFree(p);
  }
};

struct rsrs_factor {
  std::shared_ptr<Shared> sh;
  int64_t n = 0, s = 0, k = 0, p = 0;
  int64_t base = 0;  // first row of this problem in the build's tree-order index space
  int d = 2, precision = 0, kind = 0, passes = 2;
  double shift = 0.0, scale = 0.0;
  rsrs_matvec_fn fn = nullptr;
  void* ctx = nullptr;
  std::vector<int64_t> perm;  // tree position -> original index (both local to the problem)
  int32_t* perm_dev = nullptr;
  double* pts_dev = nullptr;  // local tree order
  std::vector<GroupView> groups;
  BoxDesc* desc_dev = nullptr;
  double* fd = nullptr;
  int32_t* fi = nullptr;
  int64_t root_size = 0;
  int32_t* root_idx = nullptr;  // shared index space
  double* root_A = nullptr;
  double* root_LU = nullptr;
  double* root_inv = nullptr;  // A~_BtBt^-1, for the block-diagonal solve
  // mixed precision: FP32 copies of the blocks (same offsets as fd) and of the root inverse, for
  // the solve sweeps in FP32 arithmetic
  float* fd32 = nullptr;
  float* root_inv32 = nullptr;
  int32_t* root_piv = nullptr;
  int max_r = 0;
  double *Y = nullptr, *Z = nullptr, *Om = nullptr, *Ps = nullptr;  // kept sketches (shared, rows from base)
  int sample_kernel = 0;  // mixed sampling: 1 FP32 SIMT, 2 tcgen05 3xTF32
  int residual_fp64 = 0;  // residual arithmetic, RSRS_RESIDUAL_*
  rsrs_tune_t tune{};     // launch shapes of the build and of the refinement residual
  rsrs_stats stats{};
  // the Ozaki-scheme residual's store of K's digits, made at the first residual that uses it
  // (oz_state 1), or found not to fit in device memory (-1); 0: not made yet
  mutable void* oz_store = nullptr;
  mutable int oz_state = 0;
  bool oz_in_build = false;  // the store's digits are made by the build (and its graph) itself
  // phase tables of the fused solve sweeps (device): for the solve (a = 0) and its adjoint (a = 1),
  // the upward sweep followed by the diagonal step at ph_up[a], the downward sweep at ph_down[a]
  SweepPhase* phases_dev = nullptr;
  int64_t ph_up[2] = {0, 0}, ph_down[2] = {0, 0};
  int nph_up[2] = {0, 0}, nph_down[2] = {0, 0};
  ~rsrs_factor() {
    if (oz_store) cudaFree(oz_store);
    if (phases_dev) cudaFree(phases_dev);
  }
};

namespace {

thread_local std::string g_last_error;

rsrs_status fail(rsrs_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

bool tune_valid(const rsrs_tune_t& t) {
  const int c = t.cpqr_cluster, th = t.cpqr_threads;
  bool ok = t.sample_tile >= 0 && t.sample_tile <= RSRS_SAMPLE_TILE_2x192x4_K16;
  ok = ok && (c == 0 || c == 2 || c == 4 || c == 8 || c == 16);
  ok = ok && (th == 0 || th == 256 || th == 512 || th == 1024);
  ok = ok && t.residual_split >= 0 && t.residual_split <= 16;
  for (int r : t.reserved) ok = ok && r == 0;
  return ok;
}

#define CU(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? RSRS_E_NOMEM : RSRS_E_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

// Owning device buffer list, freed when the pool goes out of scope (a graph build moves the list
// into its factors, whose replays write to the same addresses).
struct DevPool {
  std::vector<void*> ptrs;
  ~DevPool() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  cudaError_t alloc(T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, (size_t)count * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(*p);
    else (void)cudaGetLastError();  // the status is returned; leave no stale error for later checks
    return e;
  }
};

// Device memory for the Ozaki residual's store of K's digits, when it fits with a margin (2 GiB +
// 5 % of the device) for the rest of the work; the digits are made separately.
bool oz_alloc_store(const rsrs_factor* f) {
  const size_t bytes = (size_t)oz_store_bytes(f->n, f->d);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (fr < bytes + ((size_t)2 << 30) + tot / 20) return false;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  f->oz_store = p;
  return true;
}

// The fused solve's phase tables (see SweepPhase): per group of the factor, in the order of the
// separate launches of sweep_solve, a barrier after every phase (each reads rows the previous one
// writes); the diagonal step over all boxes closes the upward table (one phase when the factor's
// descriptors are contiguous, else one per group without barriers between them).
cudaError_t build_sweep_phases(rsrs_factor* f) {
  std::vector<SweepPhase> all;
  std::vector<int2> maps;             // item -> (box, tile) of every product phase, concatenated
  std::vector<int64_t> map_off;       // per phase: its first map entry, or -1
  auto phase = [&](const GroupView& g, int kind, int cset, int mat, int bset, int sync) {
    SweepPhase q{};
    q.desc = f->desc_dev + g.desc_off;
    q.nbox = (int)g.h.size();
    q.kind = kind;
    q.cset = cset;
    q.mat = mat;
    q.bset = bset;
    q.solve = 1;
    q.sync = sync;
    q.alpha = -1.0;
    q.items = kind == 2 ? 0 : sweep_phase_items(g.h, kind, cset, 0);
    q.map = nullptr;
    map_off.push_back(kind == 2 ? -1 : (int64_t)maps.size());
    if (kind != 2)
      for (size_t b = 0; b < g.h.size(); ++b) {
        const int64_t nt = sweep_phase_tiles(g.h[b], kind, cset);
        for (int64_t t = 0; t < nt; ++t) maps.push_back(make_int2((int)b, (int)t));
      }
    all.push_back(q);
  };
  bool contiguous = !f->groups.empty();
  int64_t total = 0;
  for (const GroupView& g : f->groups) {
    if (g.desc_off != f->groups[0].desc_off + total) contiguous = false;
    total += (int64_t)g.h.size();
  }
  for (int adj = 0; adj < 2; ++adj) {
    f->ph_up[adj] = (int64_t)all.size();
    for (const GroupView& g : f->groups) {
      phase(g, 0, /*C=R*/ 0, /*T*/ 0, /*B=S*/ 1, 1);
      phase(g, 0, /*C=SN*/ 2, adj ? /*Uc*/ 2 : /*LcT*/ 1, /*B=R*/ 0, 1);
    }
    if (contiguous && total <= INT32_MAX) {
      GroupView all_boxes;
      all_boxes.desc_off = f->groups[0].desc_off;
      all_boxes.h.resize((size_t)total);
      phase(all_boxes, 2, 0, 0, 0, 0);
    } else {
      for (const GroupView& g : f->groups) phase(g, 2, 0, 0, 0, 0);
    }
    f->nph_up[adj] = (int)((int64_t)all.size() - f->ph_up[adj]);
    f->ph_down[adj] = (int64_t)all.size();
    for (auto it = f->groups.rbegin(); it != f->groups.rend(); ++it) {
      phase(*it, 1, /*C=R*/ 0, adj ? /*LcT*/ 1 : /*Uc*/ 2, /*B=SN*/ 2, 1);
      phase(*it, 1, /*C=S*/ 1, /*T*/ 0, /*B=R*/ 0, 1);
    }
    f->nph_down[adj] = (int)((int64_t)all.size() - f->ph_down[adj]);
  }
  if (all.empty()) return cudaSuccess;
  // one allocation: the phase table, then the item maps (16-byte aligned)
  const size_t tbytes = (all.size() * sizeof(SweepPhase) + 15) & ~(size_t)15;
  const size_t bytes = tbytes + maps.size() * sizeof(int2);
  cudaError_t e = cudaMalloc((void**)&f->phases_dev, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    f->phases_dev = nullptr;  // the solves then take the separate launches
    return cudaSuccess;
  }
  const int2* map_dev = reinterpret_cast<const int2*>(reinterpret_cast<const char*>(f->phases_dev) + tbytes);
  for (size_t i = 0; i < all.size(); ++i)
    if (map_off[i] >= 0) all[i].map = map_dev + map_off[i];
  e = cudaMemcpy(f->phases_dev, all.data(), all.size() * sizeof(SweepPhase), cudaMemcpyHostToDevice);
  if (e != cudaSuccess || maps.empty()) return e;
  return cudaMemcpy(const_cast<int2*>(map_dev), maps.data(), maps.size() * sizeof(int2), cudaMemcpyHostToDevice);
}

// Scratch of one call from the stream-ordered allocator: allocated and freed in the order of
// `st`, so a call neither waits for the device nor serialises other streams.
struct StreamPool {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit StreamPool(cudaStream_t s) : st(s) {}
  ~StreamPool() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
  template <class T>
  cudaError_t alloc(T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMallocAsync((void**)p, (size_t)count * sizeof(T), st);
    if (e == cudaSuccess) ptrs.push_back(*p);
    else (void)cudaGetLastError();
    return e;
  }
};

// ---- layout conversions at the boundary ---------------------------------------
// rows (tree order, row-major n x c) <-> column-major original order with ld.
__global__ void k_cm_to_rows(const double* F, int64_t ld, const int32_t* perm, int64_t n, int c, double* W) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * c) return;
  int64_t t = e / c;
  int j = (int)(e % c);
  W[e] = F[(int64_t)perm[t] + (int64_t)j * ld];
}
__global__ void k_rows_to_cm(const double* W, const int32_t* perm, int64_t n, int c, double* F, int64_t ld) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * c) return;
  int64_t t = e / c;
  int j = (int)(e % c);
  F[(int64_t)perm[t] + (int64_t)j * ld] = W[e];
}
__global__ void k_gather_orig(const double* in, const int32_t* perm, int64_t n, int64_t s, double* out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * s) return;
  int64_t t = e / s, c = e % s;
  out[e] = in[(int64_t)perm[t] * s + c];
}
__global__ void k_set_u64(uint64_t* p, uint64_t v) { *p = v; }
__global__ void k_f32_to_f64(const float* in, int64_t n, double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = (double)in[e];
}
__global__ void k_axpy(double* y, const double* x, double a, int64_t n) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] += a * x[e];
}
__global__ void k_sub(double* r, const double* b, const double* ax, int64_t n) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) r[e] = b[e] - ax[e];
}
// column sums of squares of a row-major n x c block (c <= 64), accumulated with atomics
__global__ void k_colnorm2(const double* W, int64_t n, int c, double* out) {
  __shared__ double part[64];
  if (threadIdx.x < 64) part[threadIdx.x] = 0.0;
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * c; e += (int64_t)gridDim.x * blockDim.x) {
    double v = W[e];
    atomicAdd(&part[e % c], v * v);
  }
  __syncthreads();
  if (threadIdx.x < c) atomicAdd(&out[threadIdx.x], part[threadIdx.x]);
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11): 10 rounds of the
// multiply-xor round function with the published multipliers and Weyl key
// increments, counter = (pair index lo, pair index hi, stream, 0), key = seed.
__device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)p1;
    c[3] = (uint32_t)p0;
    c[0] = n0;
    c[2] = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}
// Standard normal pair number q of a stream: two 53-bit uniforms, Box-Muller.
__device__ inline void normal_pair(uint64_t seed, uint32_t stream, uint64_t q, double& z0, double& z1) {
  uint32_t c[4] = {(uint32_t)q, (uint32_t)(q >> 32), stream, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  uint64_t a = ((uint64_t)c[0] << 32 | c[1]) >> 11, b = ((uint64_t)c[2] << 32 | c[3]) >> 11;
  double u1 = ((double)a + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
  double u2 = (double)b * (1.0 / 9007199254740992.0);          // [0, 1)
  double rr = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  z0 = rr * cs;
  z1 = rr * sn;
}
// Omega (stream 0) or Psi (stream 1) in tree order: entry (t, c) is draw 2*(perm[t]*s + c) ...
__global__ void k_gauss_tree(const uint64_t* seed_dev, uint64_t add, uint32_t stream, const int32_t* perm, int64_t n,
                             int64_t s, double* out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * s) return;
  const uint64_t seed = *seed_dev + add;
  int64_t t = e / s, c = e % s;
  int64_t g = (int64_t)perm[t] * s + c;
  double z0, z1;
  normal_pair(seed, stream, (uint64_t)(g >> 1), z0, z1);
  out[e] = (g & 1) ? z1 : z0;
}
// The same for even s, one thread per pair: draws g and g + 1 (g even) are columns c and c + 1 of
// one original row, so each Box-Muller pair (FP64 log, square root, sine and cosine, at the FP64
// rate on this part) is evaluated once and both members stored.
__global__ void k_gauss_tree_pairs(const uint64_t* seed_dev, uint64_t add, uint32_t stream, const int32_t* perm,
                                   int64_t n, int64_t s, double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // pair index in tree order
  const int64_t hs = s >> 1;
  if (e >= n * hs) return;
  const uint64_t seed = *seed_dev + add;
  const int64_t t = e / hs, c = 2 * (e % hs);
  const int64_t g = (int64_t)perm[t] * s + c;
  double z0, z1;
  normal_pair(seed, stream, (uint64_t)(g >> 1), z0, z1);
  out[t * s + c] = z0;
  out[t * s + c + 1] = z1;
}

const char* kClassNames[RSRS_NCLASS] = {"sample", "lists", "gram", "chol", "gather", "proj_nt", "proj_solve",
                                        "proj_acc", "cpqr", "id_finish", "ef_update", "extract", "lu", "lu_rhs",
                                        "schur", "root"};

// Algorithmic FLOPs of one box per kernel class (what the step must compute, not padded tiles).
// xinv: X_RR^-1 formed explicitly (Gauss-Jordan, r^3 multiply-adds) instead of an LU.
void box_flops(const BoxDesc& d, int64_t s, int passes, double* fl, bool xinv) {
  const double b = d.b, l = d.l, kp = d.kp, r = d.r, w = d.kp + d.n, S = (double)s;
  fl[RSRS_K_GRAM] += 2.0 * l * (l + 1) * S;              // two SYRKs l x s
  fl[RSRS_K_CHOL] += 2.0 * l * l * l / 3.0;              // two Cholesky factorizations
  fl[RSRS_K_PROJ_NT] += passes * 2.0 * 2.0 * b * l * S;  // [Y_B; Z_B] W^T per pass
  fl[RSRS_K_PROJ_SOLVE] += passes * 2.0 * 2.0 * b * l * l;
  fl[RSRS_K_PROJ_ACC] += passes * 2.0 * 2.0 * b * l * S;
  fl[RSRS_K_CPQR] += 4.0 * (2.0 * S) * b * kp;
  fl[RSRS_K_ID] += r * kp * kp;
  fl[RSRS_K_EF] += 8.0 * r * kp * S;
  fl[RSRS_K_EXTRACT] += 4.0 * r * kp * (l + r);
  fl[RSRS_K_LU] += xinv ? 2.0 * r * r * r : 2.0 * r * r * r / 3.0;
  fl[RSRS_K_LU_RHS] += 2.0 * 2.0 * r * r * w;
  fl[RSRS_K_SCHUR] += 8.0 * r * w * S;
}

// Apply the operator to a tree-order row-major block: out = A in (adjoint for callbacks).
// fp32 products need conv: an FP32 copy of `in` (SIMT) or its hi/lo transposed planes (tensor cores),
// each n*ncols floats, hi first.
rsrs_status op_apply(const rsrs_factor* f, Launch L, const double* in, double* out, int64_t ncols, int adjoint,
                     int fp32, double* scratch_cm_in, double* scratch_cm_out, int* err = nullptr,
                     float* conv = nullptr) {
  if (f->kind == RSRS_OP_CALLBACK) {
    int64_t tot = f->n * ncols;
    k_rows_to_cm<<<nblk(tot), 256, 0, L.st>>>(in, f->perm_dev, f->n, (int)ncols, scratch_cm_in, f->n);
    if (L.counter) ++*L.counter;
    int rc = f->fn(f->ctx, adjoint, f->n, (int32_t)ncols, scratch_cm_in, f->n, scratch_cm_out, f->n, (void*)L.st);
    if (rc != 0) return fail(RSRS_E_CALLBACK, "matvec callback returned " + std::to_string(rc));
    k_cm_to_rows<<<nblk(tot), 256, 0, L.st>>>(scratch_cm_out, f->n, f->perm_dev, f->n, (int)ncols, out);
    if (L.counter) ++*L.counter;
    CU(cudaGetLastError());
    return RSRS_OK;
  }
  if (fp32 && !conv) return fail(RSRS_E_INVAL, "internal: FP32 product without conversion buffer");
  if (fp32 && f->sample_kernel == 2) {  // conv: hi and lo planes, then the FP32 points
    const int64_t ldp = tc_plane_ld(f->n);
    float *hi = conv, *lo = conv + ncols * ldp, *p32 = conv + 2 * ncols * ldp;
    launch_points_f32(L, f->pts_dev, f->n, f->d, p32);
    launch_split_transpose(L, in, f->n, ncols, hi, lo, ldp);
    if (!launch_kernel_matvec_tc(L, f->kind, p32, f->n, f->shift, f->scale, in, in, out, out, ncols, ncols, ncols,
                                 hi, lo, ldp, err, f->tune.sample_tile))
      return fail(RSRS_E_CUDA, "could not encode the TMA tensor maps of the sampling product");
    CU(cudaGetLastError());
    return RSRS_OK;
  }
  if (fp32) launch_to_f32(L, in, f->n * ncols, conv);
  launch_kernel_matvec_prec(L, f->kind, f->pts_dev, f->d, f->n, f->shift, f->scale, in, ncols, out, ncols, ncols,
                            fp32, conv);
  CU(cudaGetLastError());
  return RSRS_OK;
}

}  // namespace

// ============================================================================
extern "C" {

const char* rsrs_status_string(rsrs_status st) {
  switch (st) {
    case RSRS_OK: return "ok";
    case RSRS_E_INVAL: return "invalid argument";
    case RSRS_E_UNDERSAMPLED: return "sample count below the bound s_req";
    case RSRS_E_SINGULAR: return "singular pivot";
    case RSRS_E_NONFINITE: return "non-finite value";
    case RSRS_E_NOMEM: return "device out of memory";
    case RSRS_E_CUDA: return "CUDA error";
    case RSRS_E_CALLBACK: return "matvec callback failed";
    case RSRS_E_TIMEOUT: return "device wait timed out";
    case RSRS_E_NOT_CONVERGED: return "refinement did not converge";
  }
  return "unknown status";
}

const char* rsrs_last_error(void) { return g_last_error.c_str(); }

const char* rsrs_kernel_class_name(int cls) {
  if (cls < 0 || cls >= RSRS_NCLASS) return "";
  return kClassNames[cls];
}

rsrs_status rsrs_tree_build(const double* pts_host, int64_t n, int d, int leaf_cap, rsrs_tree** out) {
  if (!out) return fail(RSRS_E_INVAL, "out is null");
  *out = nullptr;
  if (!pts_host || n <= 0 || (d != 2 && d != 3) || leaf_cap <= 0 || n > INT32_MAX)
    return fail(RSRS_E_INVAL, "tree: need pts, n in [1, 2^31), d in {2,3}, leaf_cap > 0");
  auto t = std::make_unique<rsrs_tree>();
  if (!build_tree(pts_host, n, d, leaf_cap, t->t)) return fail(RSRS_E_INVAL, "tree: non-finite point");
  *out = t.release();
  return RSRS_OK;
}

void rsrs_tree_free(rsrs_tree* t) { delete t; }

rsrs_status rsrs_tree_perm(const rsrs_tree* tree, int64_t* perm_host) {
  if (!tree || !perm_host) return fail(RSRS_E_INVAL, "null argument");
  std::memcpy(perm_host, tree->t.perm.data(), tree->t.perm.size() * sizeof(int64_t));
  return RSRS_OK;
}

// Smallest s >= s_min for which an l-row Gaussian-like test block W (l x s) keeps its Gram
// W W^T positive definite under FP32 rounding: with cond(W) ~ (sqrt s + sqrt l) / (sqrt s - sqrt l)
// (the extreme singular values of a Gaussian matrix) the Gram's rounding, about sqrt(s) 2^-24 of
// its norm, must stay below a tenth of its smallest eigenvalue.
int64_t mixed_sample_bound(int64_t s_min, int64_t max_l) {
  auto ok = [&](int64_t s) {
    const double rs = std::sqrt((double)s), rl = std::sqrt((double)max_l);
    if (rs <= rl) return false;
    const double c = (rs + rl) / (rs - rl);
    return c * c * rs * std::ldexp(1.0, -24) <= 0.1;
  };
  int64_t s = std::max<int64_t>(s_min, 1);
  if (ok(s)) return s;
  int64_t lo = s, hi = s;
  while (!ok(hi)) hi *= 2;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    (ok(mid) ? hi : lo) = mid;
  }
  return hi;
}

rsrs_status rsrs_tree_info(const rsrs_tree* tree, int k, int p, rsrs_tree_info_t* out) {
  if (!tree || !out || k <= 0) return fail(RSRS_E_INVAL, "tree_info: null argument or k <= 0");
  Schedule sc;
  build_schedule(tree->t, k, p, sc);
  out->d = tree->t.d;
  out->depth = tree->t.depth;
  out->n = tree->t.n;
  out->n_boxes = (int64_t)tree->t.boxes.size();
  out->n_leaves = 0;
  for (auto& b : tree->t.boxes) out->n_leaves += b.leaf();
  out->n_compress = (int64_t)sc.steps.size();
  out->n_groups = 0;
  for (auto& lv : sc.groups) out->n_groups += (int64_t)lv.size();
  out->max_l = sc.max_l;
  out->root_size = (int64_t)sc.root.size();
  out->s_req = sc.s_req;
  out->s_req_mixed = sc.steps.empty() ? sc.s_req : mixed_sample_bound(sc.s_req, sc.max_l);
  return RSRS_OK;
}

rsrs_status rsrs_tree_schedule(const rsrs_tree* tree, int k, int p, int64_t* rows) {
  if (!tree || !rows || k <= 0) return fail(RSRS_E_INVAL, "tree_schedule: null argument");
  Schedule sc;
  build_schedule(tree->t, k, p, sc);
  for (size_t i = 0; i < sc.steps.size(); ++i) {
    const Step& st = sc.steps[i];
    const Box& b = tree->t.boxes[st.box];
    int64_t* r = rows + 6 * i;
    r[0] = st.level;
    r[1] = st.colour;
    r[2] = (int64_t)b.morton;
    r[3] = st.b;
    r[4] = st.n;
    r[5] = b.first_pos;
  }
  return RSRS_OK;
}

}  // extern "C"

namespace {

// Algorithm 1 for a list of independent problems in one set of launches.  Boxes of all problems at
// the same height above their deepest level and of the same colour share each launch (problems
// never share rows, so any such merge is conflict-free); the roots form one more group.
rsrs_status build_impl(int nprob, const rsrs_tree* const* trees, const rsrs_operator* ops, int k, int s,
                       const rsrs_options* opts, void* stream, rsrs_factor** out) {
  if (!out) return fail(RSRS_E_INVAL, "out is null");
  for (int p = 0; p < nprob; ++p) out[p] = nullptr;
  if (nprob <= 0 || !trees || !ops || k <= 0 || s <= 0)
    return fail(RSRS_E_INVAL, "build: need problems, k > 0, s > 0");
  rsrs_options o{};
  o.p = -1;
  if (opts) o = *opts;
  if (o.precision != RSRS_PREC_FP64 && o.precision != RSRS_PREC_MIXED)
    return fail(RSRS_E_INVAL, "build: unknown precision");
  if (o.sample_kernel < 0 || o.sample_kernel > 3) return fail(RSRS_E_INVAL, "build: unknown sample_kernel");
  if (o.sample_kernel == 3 && o.precision == RSRS_PREC_MIXED)
    return fail(RSRS_E_INVAL, "build: sample_kernel 3 (Ozaki FP64 sampling) is for FP64 builds");
  if (o.mixed_cpqr < 0 || o.mixed_cpqr > 1) return fail(RSRS_E_INVAL, "build: unknown mixed_cpqr");
  if (o.mixed_gemm < 0 || o.mixed_gemm > 1) return fail(RSRS_E_INVAL, "build: unknown mixed_gemm");
  if (!tune_valid(o.tune)) return fail(RSRS_E_INVAL, "build: tune values out of range");
  if (o.residual_fp64 < 0 || o.residual_fp64 > 3)
    return fail(RSRS_E_INVAL, "build: residual_fp64 is one of RSRS_RESIDUAL_* (0..3)");
  if (nprob > 1 && (o.omega_host || o.psi_host || o.omega_dev || o.psi_dev))
    return fail(RSRS_E_INVAL, "build: caller test matrices are for single-problem builds");
  const bool graph = o.use_graph != 0;
  if (graph && (o.omega_host || o.psi_host || o.omega_dev || o.psi_dev))
    return fail(RSRS_E_INVAL, "build: a graph build draws its test matrices on the device");
  if (graph) o.profile = 0;  // per-class event timing is not part of a captured graph
  // two least-squares passes: the second solves for the residual of the first; a third FP32 pass
  // leaves the refined mixed factor unchanged on the 65,536-point workload (same refinement
  // history to two digits), so both precisions default to two
  const int passes = o.proj_passes <= 0 ? 2 : std::min(o.proj_passes, 4);
  // tensor-core Gram factorisation and projection solve (mixed path with tcgen05 products)
  const bool tc_path = o.precision == RSRS_PREC_MIXED && o.mixed_gemm == 0;
  std::vector<Schedule> sc(nprob);
  std::vector<int64_t> base(nprob + 1, 0);
  int maxdepth = 0;
  for (int p = 0; p < nprob; ++p) {
    const rsrs_operator* op = &ops[p];
    if (!trees[p]) return fail(RSRS_E_INVAL, "build: null tree");
    if (op->kind != RSRS_OP_LOG2D && op->kind != RSRS_OP_INVR3D && op->kind != RSRS_OP_CALLBACK)
      return fail(RSRS_E_INVAL, "build: unknown operator kind");
    if (op->kind == RSRS_OP_CALLBACK && !op->fn) return fail(RSRS_E_INVAL, "build: callback operator without fn");
    const Tree& T = trees[p]->t;
    if (op->kind == RSRS_OP_LOG2D && T.d != 2) return fail(RSRS_E_INVAL, "build: log kernel needs 2D points");
    if (op->kind == RSRS_OP_INVR3D && T.d != 3) return fail(RSRS_E_INVAL, "build: 1/r kernel needs 3D points");
    build_schedule(T, k, o.p, sc[p]);
    if (s < sc[p].s_req)
      return fail(RSRS_E_UNDERSAMPLED, "problem " + std::to_string(p) + ": s=" + std::to_string(s) +
                                           " < s_req=" + std::to_string(sc[p].s_req));
    if (o.precision == RSRS_PREC_MIXED && !sc[p].steps.empty()) {
      const int64_t sm = mixed_sample_bound(sc[p].s_req, sc[p].max_l);
      if (s < sm)
        return fail(RSRS_E_UNDERSAMPLED,
                    "problem " + std::to_string(p) + ": mixed precision needs s >= " + std::to_string(sm) +
                        " (near-field Grams of up to " + std::to_string(sc[p].max_l) +
                        " rows must stay positive definite in FP32); s=" + std::to_string(s));
    }
    base[p + 1] = base[p] + T.n;
    maxdepth = std::max(maxdepth, T.depth);
  }
  const int64_t Ntot = base[nprob];
  if (Ntot > INT32_MAX) return fail(RSRS_E_INVAL, "build: more than 2^31 points in one build");
  cudaStream_t st = (cudaStream_t)stream;
  // a graph build records its launches on a private stream (the legacy default stream cannot be
  // captured); everything it enqueues is synchronised before the build returns
  struct OwnStream {
    cudaStream_t s = nullptr;
    ~OwnStream() {
      if (s) cudaStreamDestroy(s);
    }
  } own;
  if (o.use_graph) {
    CU(cudaStreamSynchronize(st));
    CU(cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking));
    st = own.s;
  }
  auto sh = std::make_shared<Shared>();
  auto dalloc = [&](auto** ptr, int64_t count) -> cudaError_t {
    using T = std::remove_reference_t<decltype(**ptr)>;
    *ptr = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc((void**)ptr, (size_t)count * sizeof(T));
    if (e == cudaSuccess) sh->ptrs.push_back((void*)*ptr);
    return e;
  };
  std::vector<std::unique_ptr<rsrs_factor>> F(nprob);
  for (int p = 0; p < nprob; ++p) {
    const Tree& T = trees[p]->t;
    auto f = std::make_unique<rsrs_factor>();
    f->sh = sh;
    f->n = T.n;
    f->base = base[p];
    f->s = s;
    f->k = k;
    f->p = sc[p].p;
    f->d = T.d;
    f->precision = o.precision;
    f->kind = ops[p].kind;
    f->passes = passes;
    f->shift = ops[p].diag_shift;
    f->scale = ops[p].scale;
    f->fn = ops[p].fn;
    f->ctx = ops[p].ctx;
    f->perm = T.perm;
    f->sample_kernel = o.sample_kernel == 0 ? 2 : o.sample_kernel;
    f->residual_fp64 = o.residual_fp64;
    f->tune = o.tune;
    F[p] = std::move(f);
  }

  // ---- plan: active-list pool, groups, descriptors, offsets --------------------
  std::vector<std::vector<int64_t>> act_off(nprob);
  int64_t act_total = 0;
  for (int p = 0; p < nprob; ++p) {
    const Tree& T = trees[p]->t;
    act_off[p].assign(T.boxes.size(), 0);
    for (size_t i = 0; i < T.boxes.size(); ++i) {
      act_off[p][i] = act_total;
      act_total += sc[p].act0[i];
    }
  }
  std::vector<int32_t> act_init(std::max<int64_t>(act_total, 1), 0);
  for (int p = 0; p < nprob; ++p) {
    const Tree& T = trees[p]->t;
    for (size_t i = 0; i < T.boxes.size(); ++i)
      if (T.boxes[i].leaf())
        for (int64_t q = 0; q < sc[p].act0[i]; ++q)
          act_init[act_off[p][i] + q] = (int32_t)(base[p] + T.boxes[i].first_pos + q);
    if (T.depth == 0)  // the root is a leaf: its slot holds every point
      for (int64_t q = 0; q < T.n; ++q) act_init[act_off[p][0] + q] = (int32_t)(base[p] + q);
  }
  struct LaunchGroup {
    int height, colour;
    int64_t desc_off, seg_off, nseg;
    std::vector<BoxDesc> h;
    std::vector<std::pair<int, int64_t>> prob_first;  // (problem, first descriptor index in h)
    int max_panels, max_b, max_r;
  };
  std::vector<LaunchGroup> groups;
  std::vector<Seg> segs;
  std::vector<std::pair<int64_t, int64_t>> height_seg(std::max(maxdepth, 1), {0, 0});
  std::vector<BoxDesc> all_desc;
  int64_t fd_total = 0, fi_total = 0, work_max = 0, workc_max = 0, iwork_max = 0;
  for (int h = 0; h < maxdepth; ++h) {
    int64_t s0 = (int64_t)segs.size();
    int ncol = 0;
    for (int p = 0; p < nprob; ++p) {
      const Tree& T = trees[p]->t;
      const int level = T.depth - h;
      if (level < 1) continue;
      for (int b : T.levels[level])
        if (!T.boxes[b].leaf()) {
          int64_t dst = act_off[p][b];
          for (int c : T.boxes[b].children) {
            if (sc[p].act1[c] > 0) segs.push_back({act_off[p][c], dst, sc[p].act1[c]});
            dst += sc[p].act1[c];
          }
        }
      ncol = std::max(ncol, (int)sc[p].groups[level].size());
    }
    height_seg[h] = {s0, (int64_t)segs.size() - s0};
    for (int col = 0; col < ncol; ++col) {
      LaunchGroup g;
      g.height = h;
      g.colour = col;
      g.desc_off = (int64_t)all_desc.size();
      g.seg_off = (int64_t)segs.size();
      g.max_panels = g.max_b = g.max_r = 0;
      int64_t w = 0, wc = 0, iw = 0;
      for (int p = 0; p < nprob; ++p) {
        const Tree& T = trees[p]->t;
        const int level = T.depth - h;
        if (level < 1 || col >= (int)sc[p].groups[level].size()) continue;
        auto [first, last] = sc[p].groups[level][col];
        if (first == last) continue;
        g.prob_first.push_back({p, (int64_t)g.h.size()});
        for (int si = first; si < last; ++si) {
          const Step& stp = sc[p].steps[si];
          BoxDesc d{};
          d.b = (int32_t)stp.b;
          d.n = (int32_t)stp.n;
          d.l = (int32_t)(stp.b + stp.n);
          d.kp = (int32_t)stp.kp;
          d.r = (int32_t)stp.r;
          d.bn_off = iw;
          iw += d.l;
          d.pv_off = iw;
          iw += d.b + 1;  // CPQR permutation and the first dependent step
          // compute-type workspace
          d.g_off = wc;
          wc += 2 * (int64_t)d.l * gram_ld(d.l);
          d.t_off = wc;
          if (tc_path) wc += 2 * (int64_t)d.b * gram_ld(d.l);
          d.x_off = wc;
          wc += 2 * (int64_t)d.b * d.l;
          d.x2_off = wc;
          if (passes > 1) wc += 2 * (int64_t)d.b * d.l;
          d.mc_off = wc;
          wc += (int64_t)d.b * 2 * s;
          d.w_off = wc;
          wc += 2 * (int64_t)d.l * s;
          d.e_off = wc;
          wc += 2 * (int64_t)d.r * d.l;
          d.li_off = wc;
          wc += li_elems(d.l);
          // FP64 workspace
          d.m_off = w;
          w += (int64_t)d.b * 2 * s;
          d.cp_off = w;
          w += (int64_t)d.kp * d.b;
          d.sn_off = w;
          w += d.b;
          d.fi_off = fi_total;
          fi_total += fi_size(d.kp, d.r, d.n);
          d.fd_off = fd_total;
          fd_total += fd_size(d.kp, d.r, d.n);
          d.act_off = act_off[p][stp.box];
          // near-field list: own active points, then each neighbour's current active points
          segs.push_back({act_off[p][stp.box], d.bn_off, stp.b});
          int64_t pos = d.bn_off + stp.b;
          for (size_t q = 0; q < stp.nbrs.size(); ++q) {
            if (stp.nbr_len[q] > 0) segs.push_back({act_off[p][stp.nbrs[q]], pos, stp.nbr_len[q]});
            pos += stp.nbr_len[q];
          }
          g.max_panels = std::max<int>(g.max_panels, (int)cdiv(d.l, kT));
          g.max_b = std::max<int>(g.max_b, d.b);
          g.max_r = std::max<int>(g.max_r, d.r);
          g.h.push_back(d);
          all_desc.push_back(d);
        }
      }
      if (g.h.empty()) continue;
      g.nseg = (int64_t)segs.size() - g.seg_off;
      work_max = std::max(work_max, w);
      workc_max = std::max(workc_max, wc);
      iwork_max = std::max(iwork_max, iw);
      groups.push_back(std::move(g));
    }
  }
  // root group: one pseudo-box per problem, B_t = what its level-1 boxes keep (or all its points)
  std::vector<BoxDesc> rh;
  int64_t root_seg_off = (int64_t)segs.size(), root_workc = 0, root_iw = 0, root_work = 0;
  std::vector<int64_t> root_iw_off(nprob, 0);
  for (int p = 0; p < nprob; ++p) {
    const Tree& T = trees[p]->t;
    const int64_t nroot = (int64_t)sc[p].root.size();
    F[p]->root_size = nroot;
    BoxDesc rd{};
    rd.b = rd.l = (int32_t)nroot;
    rd.n = rd.kp = rd.r = 0;
    rd.bn_off = root_iw;
    root_iw_off[p] = root_iw;
    root_iw += nroot;
    rd.pv_off = root_iw;
    root_iw += 1;
    rd.sn_off = root_work;  // FP64 work: the gather's row norms (unused by the root)
    root_work += nroot;
    // the root runs in FP64: its compute-type offsets count doubles
    rd.g_off = root_workc;
    root_workc += 2 * nroot * gram_ld(nroot);
    rd.t_off = root_workc;
    if (tc_path) root_workc += 2 * nroot * gram_ld(nroot);
    rd.x_off = root_workc;
    root_workc += 2 * nroot * nroot;
    rd.x2_off = root_workc;
    root_workc += 2 * nroot * nroot;
    rd.mc_off = root_workc;
    root_workc += nroot * 2 * s;
    rd.w_off = root_workc;
    root_workc += 2 * nroot * s;
    rd.e_off = root_workc;
    rd.li_off = root_workc;
    root_workc += li_elems(nroot);
    rh.push_back(rd);
    if (T.depth == 0) {
      segs.push_back({act_off[p][0], rd.bn_off, nroot});
    } else {
      int64_t dst = rd.bn_off;
      for (int b : T.levels[1]) {
        if (sc[p].act1[b] > 0) segs.push_back({act_off[p][b], dst, sc[p].act1[b]});
        dst += sc[p].act1[b];
      }
    }
  }
  const int64_t root_nseg = (int64_t)segs.size() - root_seg_off;
  iwork_max = std::max(iwork_max, root_iw);
  int max_root_panels = 0;
  for (const BoxDesc& d : rh) max_root_panels = std::max<int>(max_root_panels, (int)cdiv(d.l, kT));

  // ---- device allocations --------------------------------------------------------
  DevPool pool;  // build-only scratch
  const int64_t NS = Ntot * (int64_t)s;
  double *Y, *Z, *Om, *Ps, *work;
  int32_t *iwork, *act, *perm_all;
  Seg* segs_dev;
  BoxDesc *desc_dev, *root_desc_dev;
  int* err;
  const size_t ct_bytes = (o.precision == RSRS_PREC_MIXED) ? sizeof(float) : sizeof(double);
  unsigned char* workc;
  if (o.keep_sketches) {
    CU(dalloc(&Y, NS));
    CU(dalloc(&Z, NS));
    CU(dalloc(&Om, NS));
    CU(dalloc(&Ps, NS));
  } else {
    CU(pool.alloc(&Y, NS));
    CU(pool.alloc(&Z, NS));
    CU(pool.alloc(&Om, NS));
    CU(pool.alloc(&Ps, NS));
  }
  CU(pool.alloc(&work, std::max(work_max, root_work)));
  CU(pool.alloc(&workc, (int64_t)std::max<size_t>(workc_max * ct_bytes, root_workc * sizeof(double))));
  CU(pool.alloc(&iwork, iwork_max));
  CU(pool.alloc(&act, (int64_t)act_init.size()));
  CU(pool.alloc(&segs_dev, (int64_t)segs.size()));
  CU(pool.alloc(&root_desc_dev, nprob));
  CU(pool.alloc(&err, 1));
  CU(dalloc(&desc_dev, (int64_t)all_desc.size()));
  double* fd;
  int32_t* fi;
  CU(dalloc(&fd, fd_total));
  CU(dalloc(&fi, fi_total));
  float* fd32 = nullptr;
  if (o.precision == RSRS_PREC_MIXED) CU(dalloc(&fd32, fd_total));
  CU(dalloc(&perm_all, Ntot));
  double* pts_all;
  {
    int64_t npts = 0;
    for (int p = 0; p < nprob; ++p) npts += trees[p]->t.n * trees[p]->t.d;
    CU(dalloc(&pts_all, npts));
    int64_t po = 0;
    for (int p = 0; p < nprob; ++p) {
      const Tree& T = trees[p]->t;
      F[p]->pts_dev = pts_all + po;
      F[p]->perm_dev = perm_all + base[p];
      CU(cudaMemcpyAsync(F[p]->pts_dev, T.pts_tree.data(), T.n * T.d * sizeof(double), cudaMemcpyHostToDevice, st));
      po += T.n * T.d;
      std::vector<int32_t> p32(T.n);
      for (int64_t q = 0; q < T.n; ++q) p32[q] = (int32_t)T.perm[q];
      CU(cudaMemcpyAsync(F[p]->perm_dev, p32.data(), T.n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      CU(cudaStreamSynchronize(st));  // p32 goes out of scope
      const int64_t nroot = F[p]->root_size;
      CU(dalloc(&F[p]->root_idx, nroot));
      CU(dalloc(&F[p]->root_A, nroot * nroot));
      CU(dalloc(&F[p]->root_LU, nroot * nroot));
      CU(dalloc(&F[p]->root_piv, nroot));
      CU(dalloc(&F[p]->root_inv, nroot * nroot));
      if (fd32) CU(dalloc(&F[p]->root_inv32, nroot * nroot));
      F[p]->desc_dev = desc_dev;
      F[p]->fd = fd;
      F[p]->fd32 = fd32;
      F[p]->fi = fi;
      if (o.keep_sketches) {
        F[p]->Y = Y;
        F[p]->Z = Z;
        F[p]->Om = Om;
        F[p]->Ps = Ps;
      }
    }
  }
  int32_t* act_init_dev;
  CU(pool.alloc(&act_init_dev, (int64_t)act_init.size()));
  CU(cudaMemcpyAsync(act_init_dev, act_init.data(), act_init.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  uint64_t* seed_dev;
  CU(pool.alloc(&seed_dev, 1));
  k_set_u64<<<1, 1, 0, st>>>(seed_dev, o.seed);
  if (!segs.empty())
    CU(cudaMemcpyAsync(segs_dev, segs.data(), segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, st));
  if (!all_desc.empty())
    CU(cudaMemcpyAsync(desc_dev, all_desc.data(), all_desc.size() * sizeof(BoxDesc), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(root_desc_dev, rh.data(), rh.size() * sizeof(BoxDesc), cudaMemcpyHostToDevice, st));
  // scratch of the launch sequence, allocated before it so that it can be captured as a graph
  int64_t nmax = 0;
  for (int p = 0; p < nprob; ++p) nmax = std::max(nmax, F[p]->n);
  const int64_t nsmax = nmax * s;
  double *cm_in = nullptr, *cm_out = nullptr;
  float* conv = nullptr;
  bool any_cb = false, any_builtin = false;
  for (int p = 0; p < nprob; ++p) (F[p]->kind == RSRS_OP_CALLBACK ? any_cb : any_builtin) = true;
  if (any_cb) {
    CU(pool.alloc(&cm_in, nsmax));
    CU(pool.alloc(&cm_out, nsmax));
  }
  const bool mixed = o.precision == RSRS_PREC_MIXED;
  const bool tc = mixed && F[0]->sample_kernel == 2;
  bool root32 = mixed && o.mixed_gemm == 0;
  for (int p = 0; p < nprob; ++p)
    if (F[p]->root_size > 0 && mixed_sample_bound(0, F[p]->root_size) > s) root32 = false;
  // FP64 sampling through the Ozaki product (sample_kernel 3, one built-in-kernel problem): the
  // digit store (which the refinement residuals then reuse) and the product's scratch, before
  // any capture; without room for the store the FP64 SIMT product runs instead
  uint8_t* oz_scr = nullptr;
  const bool oz_sample = !mixed && o.sample_kernel == 3 && nprob == 1 && F[0]->kind != RSRS_OP_CALLBACK &&
                         (F[0]->oz_store || oz_alloc_store(F[0].get())) &&
                         pool.alloc(&oz_scr, oz_scratch_bytes(F[0]->n)) == cudaSuccess;
  if (oz_sample) F[0]->oz_in_build = true;
  // tensor-core path: hi/lo planes of [Omega Psi] (2s x N each) and the FP32 points; SIMT path:
  // an FP32 copy of one side
  if (mixed && any_builtin)
    CU(pool.alloc(&conv, tc ? 4 * s * tc_plane_ld(nmax) + tc_points_len(nmax, 3) : nsmax));
  std::vector<RootLU> rl;
  int64_t max_root = 0;
  for (int p = 0; p < nprob; ++p)
    if (F[p]->root_size > 0) {
      rl.push_back(RootLU{F[p]->root_LU, F[p]->root_size, F[p]->root_piv, F[p]->root_inv});
      max_root = std::max(max_root, F[p]->root_size);
    }
  RootLU* rl_dev = nullptr;
  if (!rl.empty()) {
    CU(pool.alloc(&rl_dev, (int64_t)rl.size()));
    CU(cudaMemcpyAsync(rl_dev, rl.data(), rl.size() * sizeof(RootLU), cudaMemcpyHostToDevice, st));
  }
  // caller test matrices from host memory are staged before the launch sequence
  for (int p = 0; p < nprob; ++p) {
    const Tree& T = trees[p]->t;
    const int64_t n = T.n, ns = n * s;
    for (int side = 0; side < 2; ++side) {
      double* dst = (side == 0 ? Om : Ps) + base[p] * s;
      const double* hsrc = side == 0 ? o.omega_host : o.psi_host;
      if (hsrc) {
        std::vector<double> tree_order(ns);
        for (int64_t q = 0; q < n; ++q) std::memcpy(&tree_order[q * s], &hsrc[T.perm[q] * s], s * sizeof(double));
        CU(cudaMemcpyAsync(dst, tree_order.data(), ns * sizeof(double), cudaMemcpyHostToDevice, st));
        CU(cudaStreamSynchronize(st));  // the staging buffer goes out of scope
      }
    }
  }
  CU(cudaStreamSynchronize(st));  // uploads done; rl and the host tables may go
  cudaGraph_t cgraph = nullptr;
  // ends an unfinished capture on every early return, so the caller's stream stays usable
  struct CaptureGuard {
    cudaStream_t st;
    bool active = false;
    ~CaptureGuard() {
      if (!active) return;
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
  } capture{st};
  if (graph) {
    CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    capture.active = true;
  }
  // ---- the launch sequence (captured as a graph when opts.use_graph) ------------------------
  CU(cudaMemcpyAsync(act, act_init_dev, act_init.size() * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  CU(cudaMemsetAsync(err, 0, sizeof(int), st));
  // test matrices: caller's host or device arrays (original order, single problem), or Philox draws
  // (problem p uses key seed + p); stored in tree order
  for (int p = 0; p < nprob; ++p) {
    const Tree& T = trees[p]->t;
    const int64_t n = T.n, ns = n * s;
    for (int side = 0; side < 2; ++side) {
      double* dst = (side == 0 ? Om : Ps) + base[p] * s;
      const double* hsrc = side == 0 ? o.omega_host : o.psi_host;
      const double* dsrc = side == 0 ? o.omega_dev : o.psi_dev;
      if (hsrc) {
        // staged above
      } else if (dsrc) {
        k_gather_orig<<<nblk(ns), 256, 0, st>>>(dsrc, F[p]->perm_dev, n, s, dst);
      } else {
        if ((s & 1) == 0)
          k_gauss_tree_pairs<<<nblk(ns / 2), 256, 0, st>>>(seed_dev, (uint64_t)p, (uint32_t)side, F[p]->perm_dev, n,
                                                           s, dst);
        else
          k_gauss_tree<<<nblk(ns), 256, 0, st>>>(seed_dev, (uint64_t)p, (uint32_t)side, F[p]->perm_dev, n, s, dst);
      }
      CU(cudaGetLastError());
    }
  }

  int64_t launches = 0;
  Launch L{st, &launches};
  rsrs_stats bst{};
  // per-class CUDA-event timing (opts.profile): one event pair around each class launch sequence
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> evpool;
  auto new_ev = [&]() {
    cudaEvent_t e;
    cudaEventCreate(&e);
    evpool.push_back(e);
    return e;
  };
  auto timed = [&](int cls, auto&& fn) {
    int64_t l0 = launches;
    cudaEvent_t a = nullptr;
    if (o.profile) {
      a = new_ev();
      cudaEventRecord(a, st);
    }
    fn();
    if (o.profile) {
      cudaEvent_t b = new_ev();
      cudaEventRecord(b, st);
      recs.push_back({cls, a, b});
    }
    bst.class_launches[cls] += launches - l0;
  };
  struct EvGuard {
    std::vector<cudaEvent_t>& v;
    ~EvGuard() {
      for (auto e : v) cudaEventDestroy(e);
    }
  } evguard{evpool};
  cudaEvent_t ev[4];
  for (auto& e : ev) e = new_ev();
  if (!graph) CU(cudaEventRecord(ev[0], st));
  // ---- a1: sampling Y = A Omega, Z = A* Psi, problem by problem --------------------------
  {
    rsrs_status r1 = RSRS_OK;
    timed(RSRS_K_SAMPLE, [&] {
      for (int p = 0; p < nprob && r1 == RSRS_OK; ++p) {
        const rsrs_factor* fp = F[p].get();
        const int fp32 = (mixed && fp->kind != RSRS_OP_CALLBACK) ? 1 : 0;
        const int64_t off = base[p] * s;
        if (fp32 && tc) {
          // the built-in kernels are symmetric, so Y = A Omega and Z = A* Psi are one product with
          // the 2s columns [Omega Psi]
          const int64_t ldp = tc_plane_ld(fp->n);
          float *hi = conv, *lo = conv + 2 * s * ldp, *p32 = conv + 4 * s * ldp;
          launch_points_f32(L, fp->pts_dev, fp->n, fp->d, p32);
          launch_split_transpose(L, Om + off, fp->n, s, hi, lo, ldp);
          launch_split_transpose(L, Ps + off, fp->n, s, hi + s * ldp, lo + s * ldp, ldp);
          if (!launch_kernel_matvec_tc(L, fp->kind, p32, fp->n, fp->shift, fp->scale, Om + off, Ps + off, Y + off,
                                       Z + off, s, s, 2 * s, hi, lo, ldp, err, o.tune.sample_tile))
            r1 = fail(RSRS_E_CUDA, "could not encode the TMA tensor maps of the sampling product");
          continue;
        }
        if (oz_sample) {
          // FP64-accurate Y = A Omega and Z = A Psi (the built-in kernels are symmetric) from exact
          // bf16 digit products, 16 columns per pass over the store
          launch_oz_prepare(L, fp->kind, fp->pts_dev, fp->d, fp->n, fp->oz_store);
          launch_oz_matvec(L, fp->n, fp->d, fp->oz_store, fp->shift, fp->scale, Om + off, s, Y + off, s, s, oz_scr);
          launch_oz_matvec(L, fp->n, fp->d, fp->oz_store, fp->shift, fp->scale, Ps + off, s, Z + off, s, s, oz_scr);
          fp->oz_state = 1;
          continue;
        }
        r1 = op_apply(fp, L, Om + off, Y + off, s, 0, fp32, cm_in, cm_out, err, conv);
        if (r1 == RSRS_OK) r1 = op_apply(fp, L, Ps + off, Z + off, s, 1, fp32, cm_in, cm_out, err, conv);
      }
    });
    if (r1 != RSRS_OK) return r1;
    for (int p = 0; p < nprob; ++p)
      if (F[p]->kind != RSRS_OP_CALLBACK) bst.class_gflop[RSRS_K_SAMPLE] += 4.0 * (double)F[p]->n * F[p]->n * s * 1e-9;
  }
  if (!graph) CU(cudaEventRecord(ev[1], st));
  // ---- a2..a8: heights 0.. (levels L..1 of each problem), colour by colour ------------------
  GroupArgs ga{};
  ga.s = s;
  ga.Y = Y;
  ga.Z = Z;
  ga.Om = Om;
  ga.Ps = Ps;
  ga.work = work;
  ga.workc = workc;
  ga.iwork = iwork;
  ga.fd = fd;
  ga.fi = fi;
  ga.act = act;
  ga.err = err;
  ga.fp32 = (o.precision == RSRS_PREC_MIXED) ? 1 : 0;
  double fl[RSRS_NCLASS] = {};
  size_t gi = 0;
  for (int h = 0; h < maxdepth; ++h) {
    if (height_seg[h].second > 0)
      timed(RSRS_K_LISTS, [&] {
        launch_copy_segments(L, segs_dev + height_seg[h].first, (int)height_seg[h].second, act, act);
      });
    for (; gi < groups.size() && groups[gi].height == h; ++gi) {
      const LaunchGroup& g = groups[gi];
      ga.desc = desc_dev + g.desc_off;
      ga.nbox = (int)g.h.size();
      int max_r = 0;
      for (const BoxDesc& d : g.h) max_r = std::max(max_r, d.r);
      const bool tcg_xinv = ga.fp32 && o.mixed_gemm == 0 && max_r <= kGaussJordanMaxR;
      for (const BoxDesc& d : g.h) box_flops(d, s, passes, fl, tcg_xinv);
      timed(RSRS_K_LISTS, [&] { launch_copy_segments(L, segs_dev + g.seg_off, (int)g.nseg, act, iwork); });
      timed(RSRS_K_GATHER, [&] { launch_gather_box(L, ga, items_gather(g.h)); });
      const bool tcg = ga.fp32 && o.mixed_gemm == 0;
      timed(RSRS_K_GRAM, [&] {
        if (tcg) launch_gram_tc(L, ga, g.h);
        else launch_gram(L, ga, items_gram(g.h));
      });
      timed(RSRS_K_CHOL, [&] {
        if (tcg) {
          launch_chol_tc(L, ga, g.h);
          return;
        }
        for (int pn = 0; pn < g.max_panels; ++pn) {
          launch_chol_panel(L, ga, pn);
          launch_chol_trsm(L, ga, pn, items_chol_trsm(g.h, pn));
          launch_chol_update(L, ga, pn, items_chol_update(g.h, pn));
        }
      });
      for (int pass = 0; pass < passes; ++pass) {
        timed(RSRS_K_PROJ_NT, [&] {
          if (tcg) launch_proj_nt_tc(L, ga, pass, g.h);
          else launch_proj_nt(L, ga, pass, items_proj_nt(g.h));
        });
        timed(RSRS_K_PROJ_SOLVE, [&] {
          if (tcg) launch_solve_tc(L, ga, pass, g.h);
          else launch_proj_solve(L, ga, pass, items_proj_solve(g.h));
        });
        timed(RSRS_K_PROJ_ACC, [&] {
          if (tcg) launch_proj_acc_tc(L, ga, pass, g.h);
          else launch_proj_acc(L, ga, pass, items_proj_acc(g.h, s));
        });
      }
      bool cpqr_done = false;
      if (ga.fp32 && o.mixed_cpqr == 0) timed(RSRS_K_CPQR, [&] { cpqr_done = launch_cpqr32(L, ga, g.max_b, o.tune.cpqr_cluster, o.tune.cpqr_threads); });
      if (!cpqr_done) {
        timed(RSRS_K_GATHER, [&] { launch_m_finalize(L, ga, items_finalize(g.h)); });
        timed(RSRS_K_CPQR, [&] { launch_cpqr(L, ga, g.max_b); });
      }
      timed(RSRS_K_ID, [&] { launch_id_finish(L, ga, g.max_b); });
      timed(RSRS_K_EF, [&] { launch_ef_update(L, ga, items_ef(g.h, s)); });
      timed(RSRS_K_EXTRACT, [&] { launch_extract(L, ga, items_extract(g.h)); });
      // mixed path: X_RR^-1 by FP32 Gauss-Jordan where the boxes fit shared memory (no LU), else
      // from the FP64 LU by substitution; Uc and Lc^T as tensor-core products with it
      bool gj = false;
      if (tcg) timed(RSRS_K_LU, [&] { gj = launch_gj_inv32(L, ga, max_r); });
      if (!gj) timed(RSRS_K_LU, [&] { launch_lu(L, ga); });
      if (tcg) {
        timed(RSRS_K_LU_RHS, [&] {
          if (!gj) launch_lu_inv(L, ga, items_lu_inv(g.h));
          launch_lcuc_prep(L, ga, items_lcuc_prep(g.h, gj ? 0 : 1), gj ? 0 : 1);
          launch_lcuc_tc(L, ga, g.h);
          launch_lcuc_store(L, ga, items_lcuc_store(g.h));
        });
        timed(RSRS_K_SCHUR, [&] {
          launch_schur(L, ga, items_schur(g.h, s), items_schur_prep(g.h, s, 1), 1, &g.h);
        });
      } else {
        timed(RSRS_K_LU_RHS, [&] { launch_lu_rhs(L, ga, items_lu_rhs(g.h)); });
        timed(RSRS_K_SCHUR, [&] { launch_schur(L, ga, items_schur(g.h, s), items_schur_prep(g.h, s)); });
      }
    }
    CU(cudaGetLastError());
  }
  for (int c = 0; c < RSRS_NCLASS; ++c)
    if (c != RSRS_K_SAMPLE) bst.class_gflop[c] = fl[c] * 1e-9;
  if (!graph) CU(cudaEventRecord(ev[2], st));
  // ---- a9: root extraction A~_{Bt Bt} = Y_Bt pinv(Om_Bt) for every problem, then LU ----------
  {
    ga.desc = root_desc_dev;
    ga.nbox = nprob;
    // the mixed path extracts the root blocks like its boxes (FP32 workspace, 3xTF32 products) when
    // Omega_Bt is well conditioned for that (s comfortably above |B_t|); otherwise in FP64.  The
    // root LU and its inverse are FP64 either way.
    ga.fp32 = root32 ? 1 : 0;
    bool any = false;
    for (const BoxDesc& d : rh) any = any || d.l > 0;
    if (any) {
      timed(RSRS_K_ROOT, [&] {
        launch_copy_segments(L, segs_dev + root_seg_off, (int)root_nseg, act, iwork);
        launch_gather_box(L, ga, items_gather(rh));
        if (root32) {
          launch_gram_tc(L, ga, rh);
          launch_chol_tc(L, ga, rh);
        } else {
          launch_gram(L, ga, items_gram(rh));
          for (int pn = 0; pn < max_root_panels; ++pn) {
            launch_chol_panel(L, ga, pn);
            launch_chol_trsm(L, ga, pn, items_chol_trsm(rh, pn));
            launch_chol_update(L, ga, pn, items_chol_update(rh, pn));
          }
        }
        // two least-squares passes: the second solves for the residual of the first, so that the
        // normal equations' squared conditioning (Om_Bt can be square when s = |B_t|) is corrected
        for (int pass = 0; pass < 2; ++pass) {
          if (pass) {
            if (root32) launch_proj_acc_tc(L, ga, 0, rh);
            else launch_proj_acc(L, ga, 0, items_proj_acc(rh, s));
          }
          if (root32) {
            launch_proj_nt_tc(L, ga, pass, rh);
            launch_solve_tc(L, ga, pass, rh);
          } else {
            launch_proj_nt(L, ga, pass, items_proj_nt(rh));
            launch_proj_solve(L, ga, pass, items_proj_solve(rh));
          }
        }
      });
    }
    for (int p = 0; p < nprob; ++p) {
      const int64_t nroot = F[p]->root_size;
      if (nroot == 0) continue;
      CU(cudaMemcpyAsync(F[p]->root_idx, iwork + root_iw_off[p], nroot * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                         st));
      if (root32) {
        const float* xroot = reinterpret_cast<const float*>(workc) + rh[p].x_off;
        k_f32_to_f64<<<nblk(nroot * nroot), 256, 0, st>>>(xroot, nroot * nroot, F[p]->root_A);
        ++launches;
      } else {
        const double* xroot = reinterpret_cast<const double*>(workc) + rh[p].x_off;
        CU(cudaMemcpyAsync(F[p]->root_A, xroot, nroot * nroot * sizeof(double), cudaMemcpyDeviceToDevice, st));
      }
      CU(cudaMemcpyAsync(F[p]->root_LU, F[p]->root_A, nroot * nroot * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    if (rl_dev) timed(RSRS_K_ROOT, [&] { launch_root_lu_inverse(L, rl_dev, (int)rl.size(), max_root, err); });
    if (fd32)  // FP32 copies for the mixed factor's solves
      timed(RSRS_K_ROOT, [&] {
        launch_to_f32(L, fd, fd_total, fd32);
        for (int p = 0; p < nprob; ++p)
          if (F[p]->root_size > 0)
            launch_to_f32(L, F[p]->root_inv, F[p]->root_size * F[p]->root_size, F[p]->root_inv32);
      });
    for (int p = 0; p < nprob; ++p) {
      const int64_t nroot = F[p]->root_size;
      if (nroot == 0) continue;
      const double nr = (double)nroot;
      bst.class_gflop[RSRS_K_ROOT] += (2.0 * nr * (nr + 1) * s + nr * nr * nr / 3.0 + 2.0 * nr * nr * s +
                                       2.0 * nr * nr * nr + 2.0 * nr * nr * nr / 3.0 + 2.0 * nr * nr * nr) *
                                      1e-9;
    }
  }
  if (!graph) CU(cudaEventRecord(ev[3], st));
  CU(cudaGetLastError());
  if (graph) {
    capture.active = false;
    CU(cudaStreamEndCapture(st, &cgraph));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, cgraph, 0);
    cudaGraphDestroy(cgraph);
    CU(ie);
    sh->exec = exec;
    sh->seed_dev = seed_dev;
    sh->err_dev = err;
    // the workspace stays with the factors: replays write to the same addresses
    for (void* q : pool.ptrs) sh->ptrs.push_back(q);
    pool.ptrs.clear();
    CU(cudaGraphLaunch(exec, st));
  }
  CU(cudaStreamSynchronize(st));
  int herr = 0;
  CU(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr == kDevSingular) return fail(RSRS_E_SINGULAR, "zero pivot in an LU factorization");
  if (herr == kDevNonfinite) return fail(RSRS_E_NONFINITE, "non-finite or non-positive pivot");
  if (herr == kDevTimeout) return fail(RSRS_E_TIMEOUT, "a bounded device wait expired");
  if (oz_sample) {
    int hoz = 0;
    CU(cudaMemcpy(&hoz, oz_status_word(F[0]->oz_store, F[0]->n, F[0]->d), sizeof(int), cudaMemcpyDeviceToHost));
    if (hoz == kDevNonfinite) return fail(RSRS_E_NONFINITE, "sampling: two points coincide (the kernel is unbounded)");
    if (hoz == kDevTimeout) return fail(RSRS_E_TIMEOUT, "sampling: a bounded device wait expired");
  }
  float t01 = 0.f, t12 = 0.f, t23 = 0.f;
  if (!graph) {
    CU(cudaEventElapsedTime(&t01, ev[0], ev[1]));
    CU(cudaEventElapsedTime(&t12, ev[1], ev[2]));
    CU(cudaEventElapsedTime(&t23, ev[2], ev[3]));
  }
  for (const Rec& rc : recs) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, rc.a, rc.b));
    bst.class_ms[rc.cls] += ms;
  }
  bst.s = s;
  bst.k = k;
  bst.t_sample_ms = t01;
  bst.t_compress_ms = t12;
  bst.t_root_ms = t23;
  bst.kernel_launches = launches;
  bst.work_bytes = work_max * 8 + workc_max * (int64_t)ct_bytes + iwork_max * 4 + 4 * NS * 8;
  // per-problem views of the launch groups
  for (const LaunchGroup& g : groups)
    for (size_t q = 0; q < g.prob_first.size(); ++q) {
      const int p = g.prob_first[q].first;
      const int64_t a0 = g.prob_first[q].second;
      const int64_t a1 = (q + 1 < g.prob_first.size()) ? g.prob_first[q + 1].second : (int64_t)g.h.size();
      GroupView v;
      v.level = trees[p]->t.depth - g.height;
      v.colour = g.colour;
      v.desc_off = g.desc_off + a0;
      v.h.assign(g.h.begin() + a0, g.h.begin() + a1);
      v.max_r = 0;
      for (const BoxDesc& d : v.h) v.max_r = std::max<int>(v.max_r, d.r);
      F[p]->max_r = std::max(F[p]->max_r, v.max_r);
      F[p]->groups.push_back(std::move(v));
    }
  for (int p = 0; p < nprob; ++p) {
    rsrs_factor* f = F[p].get();
    f->stats = bst;
    f->stats.n = f->n;
    f->stats.root_size = f->root_size;
    int64_t nb = 0, fdb = 0, fib = 0, sweep = 0;
    for (const GroupView& v : f->groups)
      for (const BoxDesc& d : v.h) {
        ++nb;
        fdb += fd_size(d.kp, d.r, d.n);
        fib += fi_size(d.kp, d.r, d.n);
        const int64_t r = d.r, w = (int64_t)d.kp + d.n;
        sweep += 2 * (int64_t)d.kp * r + 2 * r * w + r * r;
      }
    f->stats.n_boxes = nb;
    f->stats.factor_bytes = fdb * 8 + fib * 4 + f->root_size * f->root_size * 24 + f->root_size * 8;
    if (f->fd32) f->stats.factor_bytes += fdb * 4 + f->root_size * f->root_size * 4;
    f->stats.solve_bytes = (sweep + f->root_size * f->root_size) * (f->fd32 ? 4 : 8);
    CU(build_sweep_phases(f));
    out[p] = F[p].release();
  }
  return RSRS_OK;
}

// ---- the refinement residual's product with A ---------------------------------------------------
// Which arithmetic computes A x for a refinement, GMRES or rsrs_residual call, and its scratch.
struct ResidualOp {
  int kind = RSRS_RESIDUAL_FP64;  // RSRS_RESIDUAL_FP64 (op_apply), _FLOAT_FLOAT or _OZAKI
  float* ffs = nullptr;
  void* ozs = nullptr;
};

// The factor's store of K's digits for the Ozaki-scheme product, made on first use when it fits
// next to a margin of 2 GiB + 5 % of the device's memory; RSRS_E_NOMEM when it does not.
rsrs_status oz_ensure(const rsrs_factor* f, Launch L) {
  if (f->oz_state == 1) return RSRS_OK;
  if (f->oz_state < 0) return fail(RSRS_E_NOMEM, "Ozaki residual: the digit store does not fit");
  const size_t bytes = (size_t)oz_store_bytes(f->n, f->d);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    (void)cudaGetLastError();
    fr = 0;
  }
  const size_t margin = ((size_t)2 << 30) + tot / 20;
  if (fr < bytes + margin) {
    f->oz_state = -1;
    return fail(RSRS_E_NOMEM, "Ozaki residual: " + std::to_string(bytes >> 20) + " MiB of digits do not fit");
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    f->oz_state = -1;
    return fail(RSRS_E_NOMEM, "Ozaki residual: allocation of the digit store failed");
  }
  f->oz_store = p;
  launch_oz_prepare(L, f->kind, f->pts_dev, f->d, f->n, p);
  CU(cudaGetLastError());
  f->oz_state = 1;
  return RSRS_OK;
}

rsrs_status residual_setup(const rsrs_factor* f, Launch L, DevPool& pool, int64_t ncols, ResidualOp& ro) {
  ro = ResidualOp{};
  if (f->kind == RSRS_OP_CALLBACK || f->residual_fp64 == RSRS_RESIDUAL_FP64) return RSRS_OK;
  if (f->residual_fp64 != RSRS_RESIDUAL_FLOAT_FLOAT) {
    rsrs_status r = oz_ensure(f, L);
    if (r == RSRS_OK) {
      uint8_t* scr = nullptr;
      if (pool.alloc(&scr, oz_scratch_bytes(f->n)) == cudaSuccess) {
        ro.kind = RSRS_RESIDUAL_OZAKI;
        ro.ozs = scr;
        return RSRS_OK;
      }
      r = fail(RSRS_E_NOMEM, "Ozaki residual: scratch allocation failed");
    }
    if (f->residual_fp64 == RSRS_RESIDUAL_OZAKI) return r;
  }
  ro.kind = RSRS_RESIDUAL_FLOAT_FLOAT;
  CU(pool.alloc(&ro.ffs, ff_scratch_floats(f->n, f->d, (int)ncols, f->tune.residual_split)));
  return RSRS_OK;
}

// out = A in (rows in tree order, ld = ncols) in the arithmetic of ro.
rsrs_status residual_apply(const rsrs_factor* f, Launch L, const ResidualOp& ro, const double* in, double* out,
                           int64_t ncols, double* c1, double* c2) {
  if (ro.kind == RSRS_RESIDUAL_OZAKI) {
    launch_oz_matvec(L, f->n, f->d, f->oz_store, f->shift, f->scale, in, ncols, out, ncols, ncols, ro.ozs);
  } else if (ro.kind == RSRS_RESIDUAL_FLOAT_FLOAT) {
    launch_kernel_matvec_ff(L, f->kind, f->pts_dev, f->d, f->n, f->shift, f->scale, in, ncols, out, ncols, ncols,
                            ro.ffs, f->tune.residual_split);
  } else {
    return op_apply(f, L, in, out, ncols, 0, 0, c1, c2);
  }
  CU(cudaGetLastError());
  return RSRS_OK;
}

// Device-detected conditions of the Ozaki product (read after the stream has synchronised).
rsrs_status residual_check(const rsrs_factor* f, const ResidualOp& ro) {
  if (ro.kind != RSRS_RESIDUAL_OZAKI) return RSRS_OK;
  int h = 0;
  CU(cudaMemcpy(&h, oz_status_word(f->oz_store, f->n, f->d), sizeof(int), cudaMemcpyDeviceToHost));
  if (h == kDevNonfinite) return fail(RSRS_E_NONFINITE, "residual: two points coincide (the kernel is unbounded)");
  if (h == kDevTimeout) return fail(RSRS_E_TIMEOUT, "residual: a bounded device wait expired");
  return RSRS_OK;
}

}  // namespace

extern "C" {

rsrs_status rsrs_build(const rsrs_tree* tree, const rsrs_operator* op, int k, int s, const rsrs_options* opts,
                       void* stream, rsrs_factor** out) {
  if (!out) return fail(RSRS_E_INVAL, "out is null");
  *out = nullptr;
  if (!tree || !op) return fail(RSRS_E_INVAL, "build: null tree or operator");
  return build_impl(1, &tree, op, k, s, opts, stream, out);
}

rsrs_status rsrs_build_batched(int nprob, const rsrs_tree* const* trees, const rsrs_operator* ops, int k, int s,
                               const rsrs_options* opts, void* stream, rsrs_factor** out) {
  return build_impl(nprob, trees, ops, k, s, opts, stream, out);
}

rsrs_status rsrs_refactor(rsrs_factor* f, uint64_t seed, void* stream) {
  if (!f) return fail(RSRS_E_INVAL, "refactor: null factor");
  Shared* sh = f->sh.get();
  if (!sh || !sh->exec) return fail(RSRS_E_INVAL, "refactor: the factor was built without use_graph");
  cudaStream_t st = (cudaStream_t)stream;
  if (f->oz_in_build) {
    // the build's own sampling makes the digits: the replay below makes them again
  } else {
    if (f->oz_store) {  // made again at the next residual, so that a rebuild costs what a build does
      cudaFree(f->oz_store);
      f->oz_store = nullptr;
    }
    f->oz_state = 0;
  }
  k_set_u64<<<1, 1, 0, st>>>(sh->seed_dev, seed);
  CU(cudaGetLastError());
  CU(cudaGraphLaunch(sh->exec, st));
  CU(cudaStreamSynchronize(st));
  int herr = 0;
  CU(cudaMemcpy(&herr, sh->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr == kDevSingular) return fail(RSRS_E_SINGULAR, "zero pivot in an LU factorization");
  if (herr == kDevNonfinite) return fail(RSRS_E_NONFINITE, "non-finite or non-positive pivot");
  if (herr == kDevTimeout) return fail(RSRS_E_TIMEOUT, "a bounded device wait expired");
  return RSRS_OK;
}

void rsrs_factor_free(rsrs_factor* f) {
  if (!f) return;
  delete f;  // shared device storage goes with the last factor of its build
}

}  // extern "C"

// ---- autotuner ----------------------------------------------------------------------------
namespace {

// Cache key: device name (blanks as '_'), operator kind, problems, total N, d, k, s, precision.
std::string tune_key(int nprob, const rsrs_tree* const* trees, const rsrs_operator* ops, int k, int s, int prec) {
  int dev = 0;
  cudaDeviceProp prop{};
  std::string name = "unknown";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  cudaGetLastError();
  for (char& c : name)
    if (c == ' ' || c == '\t') c = '_';
  int64_t ntot = 0;
  for (int p = 0; p < nprob; ++p) ntot += trees[p]->t.n;
  char buf[256];
  std::snprintf(buf, sizeof buf, " %d %d %lld %d %d %d %d", ops[0].kind, nprob, (long long)ntot, trees[0]->t.d, k, s,
                prec);
  return name + buf;
}

bool tune_cache_find(const char* path, const std::string& key, rsrs_tune_t* out) {
  FILE* fh = std::fopen(path, "r");
  if (!fh) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof line, fh)) {
    const size_t kl = key.size();
    if (std::strncmp(line, key.c_str(), kl) != 0 || line[kl] != ' ') continue;
    rsrs_tune_t t{};
    if (std::sscanf(line + kl, " %d %d %d %d", &t.sample_tile, &t.cpqr_cluster, &t.cpqr_threads,
                    &t.residual_split) == 4 &&
        tune_valid(t)) {
      *out = t;  // the last matching line wins
      found = true;
    }
  }
  std::fclose(fh);
  return found;
}

void tune_cache_add(const char* path, const std::string& key, const rsrs_tune_t& t) {
  FILE* fh = std::fopen(path, "a");
  if (!fh) return;
  std::fprintf(fh, "%s %d %d %d %d\n", key.c_str(), t.sample_tile, t.cpqr_cluster, t.cpqr_threads, t.residual_split);
  std::fclose(fh);
}

}  // namespace

extern "C" rsrs_status rsrs_autotune(int nprob, const rsrs_tree* const* trees, const rsrs_operator* ops, int k,
                                     int s, const rsrs_options* opts, int reps, const char* cache_path, void* stream,
                                     rsrs_tune_t* out, rsrs_tune_report* report) {
  if (!out || nprob < 1 || !trees || !ops) return fail(RSRS_E_INVAL, "autotune: null argument");
  for (int p = 0; p < nprob; ++p)
    if (!trees[p]) return fail(RSRS_E_INVAL, "autotune: null tree");
  rsrs_options o{};
  if (opts) o = *opts;
  if (!tune_valid(o.tune)) return fail(RSRS_E_INVAL, "autotune: tune values out of range");
  reps = std::max(1, std::min(reps, 10));
  rsrs_tune_report rep{};
  const std::string key = tune_key(nprob, trees, ops, k, s, o.precision);
  if (cache_path && tune_cache_find(cache_path, key, out)) {
    rep.from_cache = 1;
    if (report) *report = rep;
    return RSRS_OK;
  }
  o.profile = 1;
  o.use_graph = 0;
  o.keep_sketches = 0;
  const bool mixed = o.precision == RSRS_PREC_MIXED;
  bool builtin = true;
  for (int p = 0; p < nprob; ++p) builtin = builtin && ops[p].kind != RSRS_OP_CALLBACK;
  const bool tune_sample = mixed && builtin && (o.sample_kernel == 0 || o.sample_kernel == 2);
  const bool tune_cpqr = mixed && o.mixed_cpqr == 0;
  const bool tune_resid = builtin && o.residual_fp64 == RSRS_RESIDUAL_FLOAT_FLOAT;

  // best-of-reps device time per kernel class of one build configuration
  auto time_build = [&](const rsrs_tune_t& t, double* cls) -> rsrs_status {
    for (int c = 0; c < RSRS_NCLASS; ++c) cls[c] = 1e300;
    o.tune = t;
    for (int r = 0; r < reps; ++r) {
      std::vector<rsrs_factor*> F(nprob, nullptr);
      const rsrs_status st = build_impl(nprob, trees, ops, k, s, &o, stream, F.data());
      if (st != RSRS_OK) return st;
      for (int c = 0; c < RSRS_NCLASS; ++c) cls[c] = std::min(cls[c], F[0]->stats.class_ms[c]);
      for (rsrs_factor* f : F) rsrs_factor_free(f);
    }
    ++rep.candidates;
    return RSRS_OK;
  };
  // keep a candidate only when it is at least 1% faster (ties keep the earlier, default-first value)
  auto better = [](double t, double best) { return t < 0.99 * best; };

  rsrs_tune_t best = o.tune;
  double cls[RSRS_NCLASS], def[RSRS_NCLASS];
  rsrs_status st = time_build(rsrs_tune_t{}, def);
  if (st != RSRS_OK) return st;
  double cur[RSRS_NCLASS];
  bool start_zero = true;
  {
    const rsrs_tune_t z{};
    start_zero = std::memcmp(&best, &z, sizeof z) == 0;
  }
  if (start_zero) {
    std::copy(def, def + RSRS_NCLASS, cur);
  } else {
    st = time_build(best, cur);
    if (st != RSRS_OK) return st;
  }
  if (tune_sample) {
    double bt = cur[RSRS_K_SAMPLE];
    const int cand[] = {RSRS_SAMPLE_TILE_2x256x3_K16, RSRS_SAMPLE_TILE_2x192x4_K16, RSRS_SAMPLE_TILE_256x4_K16,
                        RSRS_SAMPLE_TILE_256x2, RSRS_SAMPLE_TILE_128x3, RSRS_SAMPLE_TILE_192x2,
                        RSRS_SAMPLE_TILE_192x5_K16};
    for (int v : cand) {
      if (v == best.sample_tile || (v == RSRS_SAMPLE_TILE_2x256x3_K16 && best.sample_tile == 0)) continue;
      rsrs_tune_t t = best;
      t.sample_tile = v;
      st = time_build(t, cls);
      if (st != RSRS_OK) return st;
      if (better(cls[RSRS_K_SAMPLE], bt)) {
        bt = cls[RSRS_K_SAMPLE];
        best = t;
        std::copy(cls, cls + RSRS_NCLASS, cur);
      }
    }
  }
  if (tune_cpqr) {
    double bt = cur[RSRS_K_CPQR];
    for (int c : {2, 4, 8, 16}) {
      if (c == best.cpqr_cluster) continue;
      rsrs_tune_t t = best;
      t.cpqr_cluster = c;
      st = time_build(t, cls);
      if (st != RSRS_OK) return st;
      if (better(cls[RSRS_K_CPQR], bt)) {
        bt = cls[RSRS_K_CPQR];
        best = t;
        std::copy(cls, cls + RSRS_NCLASS, cur);
      }
    }
    for (int th : {512, 256}) {
      if (th == best.cpqr_threads) continue;
      rsrs_tune_t t = best;
      t.cpqr_threads = th;
      st = time_build(t, cls);
      if (st != RSRS_OK) return st;
      if (better(cls[RSRS_K_CPQR], bt)) {
        bt = cls[RSRS_K_CPQR];
        best = t;
        std::copy(cls, cls + RSRS_NCLASS, cur);
      }
    }
  }
  rep.default_ms = (tune_sample ? def[RSRS_K_SAMPLE] : 0.0) + (tune_cpqr ? def[RSRS_K_CPQR] : 0.0);
  rep.tuned_ms = (tune_sample ? cur[RSRS_K_SAMPLE] : 0.0) + (tune_cpqr ? cur[RSRS_K_CPQR] : 0.0);
  if (tune_resid) {
    // one float-float residual product of 16 columns on the first problem, per split value
    o.tune = best;
    o.profile = 0;
    std::vector<rsrs_factor*> F(nprob, nullptr);
    st = build_impl(nprob, trees, ops, k, s, &o, stream, F.data());
    if (st != RSRS_OK) return st;
    const rsrs_factor* f = F[0];
    cudaStream_t cs = (cudaStream_t)stream;
    Launch L{cs, nullptr};
    DevPool pool;
    const int nc = 16;
    double *Wx = nullptr, *Wax = nullptr;
    float* scr = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int64_t need = 0;
    for (int sp : {0, 1, 2, 4, 8, 16}) need = std::max(need, ff_scratch_floats(f->n, f->d, nc, sp));
    cudaError_t ce = pool.alloc(&Wx, f->n * nc);
    if (ce == cudaSuccess) ce = pool.alloc(&Wax, f->n * nc);
    if (ce == cudaSuccess) ce = pool.alloc(&scr, need);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(Wx, 0, (size_t)f->n * nc * sizeof(double), cs);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    double def_ms = 0.0, best_ms = 1e300;
    for (int sp : {0, 1, 2, 4, 8, 16}) {
      if (ce != cudaSuccess) break;
      double tmin = 1e300;
      for (int r = 0; r < reps + 1 && ce == cudaSuccess; ++r) {  // the first run warms up
        cudaEventRecord(e0, cs);
        launch_kernel_matvec_ff(L, f->kind, f->pts_dev, f->d, f->n, f->shift, f->scale, Wx, nc, Wax, nc, nc, scr, sp);
        cudaEventRecord(e1, cs);
        ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) tmin = std::min(tmin, (double)ms);
      }
      ++rep.candidates;
      if (sp == 0) def_ms = tmin;
      if (sp == 0 || better(tmin, best_ms)) {
        best_ms = tmin;
        best.residual_split = sp;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (rsrs_factor* ff : F) rsrs_factor_free(ff);
    if (ce != cudaSuccess) return fail(RSRS_E_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
    rep.default_ms += def_ms;
    rep.tuned_ms += best_ms;
  }
  *out = best;
  if (cache_path) tune_cache_add(cache_path, key, best);
  if (report) *report = rep;
  return RSRS_OK;
}

// ---- sweeps on a tree-order row-major block ------------------------------------------
namespace {

// W <- A_approx^-1 W (eq. Ainvfact).  A mixed-precision factor solves in FP32 arithmetic when the
// caller passes w32 (N x nrhs floats): W is converted once, swept with the FP32 copies of the
// blocks, and converted back (its corrections feed FP64 refinement, whose residual sets the final
// accuracy); an FP64 factor, or w32 null, sweeps in FP64.
// f_R <- X_RR^-1 f_R (solve) or X_RR f_R (apply) for every box: the boxes touch disjoint rows, so
// one launch covers all levels when the factor's descriptors are contiguous (a single-problem
// build), else one per group.
void diag_sweep(const rsrs_factor* f, Launch L, SweepArgs a, int nrhs, int solve) {
  bool contiguous = !f->groups.empty();
  int64_t total = 0, items = 0;
  for (size_t i = 0; i < f->groups.size(); ++i) {
    const GroupView& g = f->groups[i];
    if (g.desc_off != f->groups[0].desc_off + total) contiguous = false;
    total += (int64_t)g.h.size();
    items += items_diag(g.h, nrhs);
  }
  if (contiguous && total <= INT32_MAX) {
    a.desc = f->desc_dev + f->groups[0].desc_off;
    a.nbox = (int)total;
    launch_sweep_diag(L, a, solve, items, f->max_r);
    return;
  }
  for (const GroupView& g : f->groups) {
    a.desc = f->desc_dev + g.desc_off;
    a.nbox = (int)g.h.size();
    launch_sweep_diag(L, a, solve, items_diag(g.h, nrhs), g.max_r);
  }
}

// bar (optional): three zeroed words of device scratch for the fused sweeps' grid barrier; with it
// each sweep direction is one cooperative launch over the factor's phase table, else (or when the
// cooperative launch is refused) one launch per group and product.
rsrs_status sweep_solve(const rsrs_factor* f, Launch L, double* W, int nrhs, int adjoint, float* w32 = nullptr,
                        unsigned* bar = nullptr) {
  SweepArgs a{};
  a.fd = f->fd;
  a.fi = f->fi;
  a.F = W;
  a.nrhs = nrhs;
  a.adjoint = adjoint;
  a.row_base = f->base;
  const bool fp32 = w32 && f->fd32;
  if (fp32) {
    a.fd32 = f->fd32;
    a.F32 = w32;
    launch_to_f32(L, W, f->n * nrhs, w32);
  }
  const int ad = adjoint ? 1 : 0;
  if (bar && f->phases_dev &&
      launch_sweep_fused(L, a, f->phases_dev + f->ph_up[ad], f->nph_up[ad], f->max_r, bar)) {
    if (f->root_size > 0) {
      if (fp32) launch_dense_apply(L, f->root_inv32, f->root_size, f->root_idx, f->base, w32, nrhs, adjoint);
      else launch_dense_apply(L, f->root_inv, f->root_size, f->root_idx, f->base, W, nrhs, adjoint);
    }
    if (!launch_sweep_fused(L, a, f->phases_dev + f->ph_down[ad], f->nph_down[ad], f->max_r, bar))
      return fail(RSRS_E_CUDA, "solve: the cooperative launch of the downward sweep failed");
    if (fp32) launch_to_f64(L, w32, f->n * nrhs, W);
    CU(cudaGetLastError());
    return RSRS_OK;
  }
  // upward: V_1^-1 first (V^-1 = L E), or W^-* = U^* F^* for the adjoint
  for (const GroupView& g : f->groups) {
    a.desc = f->desc_dev + g.desc_off;
    a.nbox = (int)g.h.size();
    launch_sweep_op(L, a, /*C=R*/ 0, /*T*/ 0, /*trans*/ 1, /*B=S*/ 1, -1.0, g.h);
    if (!adjoint)
      launch_sweep_op(L, a, 2, /*LcT*/ 1, 1, 0, -1.0, g.h);
    else
      launch_sweep_op(L, a, 2, /*Uc*/ 2, 1, 0, -1.0, g.h);
  }
  diag_sweep(f, L, a, nrhs, 1);
  if (f->root_size > 0) {
    if (fp32) launch_dense_apply(L, f->root_inv32, f->root_size, f->root_idx, f->base, w32, nrhs, adjoint);
    else launch_dense_apply(L, f->root_inv, f->root_size, f->root_idx, f->base, W, nrhs, adjoint);
  }
  for (auto it = f->groups.rbegin(); it != f->groups.rend(); ++it) {
    const GroupView& g = *it;
    a.desc = f->desc_dev + g.desc_off;
    a.nbox = (int)g.h.size();
    if (!adjoint)
      launch_sweep_op(L, a, 0, /*Uc*/ 2, 0, 2, -1.0, g.h);
    else
      launch_sweep_op(L, a, 0, /*LcT*/ 1, 0, 2, -1.0, g.h);
    launch_sweep_op(L, a, /*C=S*/ 1, /*T*/ 0, 0, /*B=R*/ 0, -1.0, g.h);
  }
  if (fp32) launch_to_f64(L, w32, f->n * nrhs, W);
  CU(cudaGetLastError());
  return RSRS_OK;
}

// Status of the fused sweeps run with barrier words bar (after the stream has reached them).
rsrs_status sweep_status(const unsigned* bar) {
  unsigned h[4] = {0, 0, 0, 0};
  CU(cudaMemcpy(h, bar, sizeof(h), cudaMemcpyDeviceToHost));
  if ((int)h[2] == kDevTimeout) return fail(RSRS_E_TIMEOUT, "solve: a grid barrier of the fused sweeps gave up");
  return RSRS_OK;
}

rsrs_status sweep_apply(const rsrs_factor* f, Launch L, double* W, int nrhs, int adjoint) {
  SweepArgs a{};
  a.fd = f->fd;
  a.fi = f->fi;
  a.F = W;
  a.nrhs = nrhs;
  a.adjoint = adjoint;
  a.row_base = f->base;
  for (const GroupView& g : f->groups) {  // W_1 first: F^-1 then U^-1 (or V^*: E^-* then L^-*)
    a.desc = f->desc_dev + g.desc_off;
    a.nbox = (int)g.h.size();
    launch_sweep_op(L, a, 1, 0, 0, 0, 1.0, g.h);
    if (!adjoint)
      launch_sweep_op(L, a, 0, 2, 0, 2, 1.0, g.h);
    else
      launch_sweep_op(L, a, 0, 1, 0, 2, 1.0, g.h);
  }
  diag_sweep(f, L, a, nrhs, 0);
  if (f->root_size > 0) launch_dense_apply(L, f->root_A, f->root_size, f->root_idx, f->base, W, nrhs, adjoint);
  for (auto it = f->groups.rbegin(); it != f->groups.rend(); ++it) {  // V_M first: L^-1 then E^-1
    const GroupView& g = *it;
    a.desc = f->desc_dev + g.desc_off;
    a.nbox = (int)g.h.size();
    if (!adjoint)
      launch_sweep_op(L, a, 2, 1, 1, 0, 1.0, g.h);
    else
      launch_sweep_op(L, a, 2, 2, 1, 0, 1.0, g.h);
    launch_sweep_op(L, a, 0, 0, 1, 1, 1.0, g.h);
  }
  CU(cudaGetLastError());
  return RSRS_OK;
}

rsrs_status check_block(const rsrs_factor* f, const void* F, int64_t ld, int32_t nrhs) {
  if (!f || !F) return fail(RSRS_E_INVAL, "null factor or block");
  if (nrhs <= 0 || nrhs > 4096 || ld < f->n) return fail(RSRS_E_INVAL, "need 0 < nrhs <= 4096 and ld >= N");
  return RSRS_OK;
}

}  // namespace

extern "C" {

rsrs_status rsrs_solve(const rsrs_factor* f, double* F, int64_t ldf, int32_t nrhs, int adjoint, void* stream) {
  rsrs_status r = check_block(f, F, ldf, nrhs);
  if (r != RSRS_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  Launch L{st, nullptr};
  StreamPool pool(st);
  double* W;
  float* w32 = nullptr;
  unsigned* bar = nullptr;
  CU(pool.alloc(&W, f->n * nrhs));
  if (f->fd32) CU(pool.alloc(&w32, f->n * nrhs));
  CU(pool.alloc(&bar, 4));
  CU(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st));
  k_cm_to_rows<<<nblk(f->n * nrhs), 256, 0, st>>>(F, ldf, f->perm_dev, f->n, nrhs, W);
  r = sweep_solve(f, L, W, nrhs, adjoint, w32, bar);
  if (r != RSRS_OK) return r;
  k_rows_to_cm<<<nblk(f->n * nrhs), 256, 0, st>>>(W, f->perm_dev, f->n, nrhs, F, ldf);
  CU(cudaGetLastError());
  return RSRS_OK;
}

rsrs_status rsrs_apply(const rsrs_factor* f, double* F, int64_t ldf, int32_t nrhs, int adjoint, void* stream) {
  rsrs_status r = check_block(f, F, ldf, nrhs);
  if (r != RSRS_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  Launch L{st, nullptr};
  StreamPool pool(st);
  double* W;
  CU(pool.alloc(&W, f->n * nrhs));
  k_cm_to_rows<<<nblk(f->n * nrhs), 256, 0, st>>>(F, ldf, f->perm_dev, f->n, nrhs, W);
  r = sweep_apply(f, L, W, nrhs, adjoint);
  if (r != RSRS_OK) return r;
  k_rows_to_cm<<<nblk(f->n * nrhs), 256, 0, st>>>(W, f->perm_dev, f->n, nrhs, F, ldf);
  CU(cudaGetLastError());
  return RSRS_OK;
}

rsrs_status rsrs_matvec(const rsrs_factor* f, const double* X, double* Yout, int64_t ld, int32_t nrhs,
                        void* stream) {
  rsrs_status r = check_block(f, X, ld, nrhs);
  if (r != RSRS_OK) return r;
  if (!Yout) return fail(RSRS_E_INVAL, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  Launch L{st, nullptr};
  DevPool pool;
  double *Wx, *Wy, *c1 = nullptr, *c2 = nullptr;
  CU(pool.alloc(&Wx, f->n * nrhs));
  CU(pool.alloc(&Wy, f->n * nrhs));
  if (f->kind == RSRS_OP_CALLBACK) {
    CU(pool.alloc(&c1, f->n * nrhs));
    CU(pool.alloc(&c2, f->n * nrhs));
  }
  k_cm_to_rows<<<nblk(f->n * nrhs), 256, 0, st>>>(X, ld, f->perm_dev, f->n, nrhs, Wx);
  r = op_apply(f, L, Wx, Wy, nrhs, 0, 0, c1, c2);
  if (r != RSRS_OK) return r;
  k_rows_to_cm<<<nblk(f->n * nrhs), 256, 0, st>>>(Wy, f->perm_dev, f->n, nrhs, Yout, ld);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  return RSRS_OK;
}

rsrs_status rsrs_refine(const rsrs_factor* f, const double* B, double* X, int64_t ld, int32_t nrhs, double rtol,
                        int maxit, void* stream, rsrs_refine_report* rep) {
  rsrs_status r = check_block(f, B, ld, nrhs);
  if (r != RSRS_OK) return r;
  if (!X || nrhs > 64 || maxit < 0 || !(rtol >= 0.0)) return fail(RSRS_E_INVAL, "refine: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t nl = 0;  // kernels launched, for the report
  Launch L{st, &nl};
  DevPool pool;
  const int64_t tot = f->n * nrhs;
  double *Wb, *Wx, *Wr, *Wax, *nrm, *c1 = nullptr, *c2 = nullptr;
  CU(pool.alloc(&Wb, tot));
  CU(pool.alloc(&Wx, tot));
  CU(pool.alloc(&Wr, tot));
  CU(pool.alloc(&Wax, tot));
  CU(pool.alloc(&nrm, 2 * 64));
  float* w32 = nullptr;
  if (f->fd32) CU(pool.alloc(&w32, tot));
  if (f->kind == RSRS_OP_CALLBACK) {
    CU(pool.alloc(&c1, tot));
    CU(pool.alloc(&c2, tot));
  }
  unsigned* bar = nullptr;  // the fused sweeps' barrier words, shared by this call's solves
  CU(pool.alloc(&bar, 4));
  CU(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st));
  ResidualOp ro;
  r = residual_setup(f, L, pool, nrhs, ro);
  if (r != RSRS_OK) return r;
  k_cm_to_rows<<<nblk(tot), 256, 0, st>>>(B, ld, f->perm_dev, f->n, nrhs, Wb);
  ++nl;
  CU(cudaMemcpyAsync(Wx, Wb, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
  r = sweep_solve(f, L, Wx, nrhs, 0, w32, bar);
  if (r != RSRS_OK) return r;
  double hn[128];
  CU(cudaMemsetAsync(nrm, 0, 64 * sizeof(double), st));
  k_colnorm2<<<std::min<int64_t>(1024, nblk(tot)), 256, 0, st>>>(Wb, f->n, nrhs, nrm);
  ++nl;
  CU(cudaMemcpyAsync(hn, nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  std::vector<double> bn(hn, hn + nrhs);
  rsrs_refine_report rr{};
  double rel = 0.0;
  int it = 0;
  for (;; ++it) {
    r = residual_apply(f, L, ro, Wx, Wax, nrhs, c1, c2);
    if (r != RSRS_OK) return r;
    k_sub<<<nblk(tot), 256, 0, st>>>(Wr, Wb, Wax, tot);
    CU(cudaMemsetAsync(nrm, 0, 64 * sizeof(double), st));
    k_colnorm2<<<std::min<int64_t>(1024, nblk(tot)), 256, 0, st>>>(Wr, f->n, nrhs, nrm);
    nl += 2;  // k_sub, k_colnorm2
    CU(cudaMemcpyAsync(hn, nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (it == 0) {
      r = residual_check(f, ro);
      if (r != RSRS_OK) return r;
    }
    rel = 0.0;
    for (int j = 0; j < nrhs; ++j) rel = std::max(rel, std::sqrt(hn[j]) / std::max(std::sqrt(bn[j]), 1e-300));
    if (it < 64) rr.history[it] = rel;
    if (!std::isfinite(rel)) return fail(RSRS_E_NONFINITE, "refine: non-finite residual");
    if (rel <= rtol || it >= maxit) break;
    r = sweep_solve(f, L, Wr, nrhs, 0, w32, bar);
    if (r != RSRS_OK) return r;
    k_axpy<<<nblk(tot), 256, 0, st>>>(Wx, Wr, 1.0, tot);
    ++nl;
  }
  k_rows_to_cm<<<nblk(tot), 256, 0, st>>>(Wx, f->perm_dev, f->n, nrhs, X, ld);
  ++nl;
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  r = residual_check(f, ro);
  if (r != RSRS_OK) return r;
  r = sweep_status(bar);
  if (r != RSRS_OK) return r;
  rr.iterations = it;
  rr.rel_residual = rel;
  rr.kernel_launches = nl;
  rr.residual_kind = ro.kind;
  if (rep) *rep = rr;
  if (rel > rtol) return fail(RSRS_E_NOT_CONVERGED, "refine: residual " + std::to_string(rel) + " > rtol");
  return RSRS_OK;
}

rsrs_status rsrs_residual(const rsrs_factor* f, const double* B, const double* X, double* Rout, int64_t ld,
                          int32_t nrhs, void* stream) {
  rsrs_status r = check_block(f, B, ld, nrhs);
  if (r != RSRS_OK) return r;
  if (!X || !Rout) return fail(RSRS_E_INVAL, "residual: null block");
  cudaStream_t st = (cudaStream_t)stream;
  Launch L{st, nullptr};
  DevPool pool;
  const int64_t tot = f->n * nrhs;
  double *Wb, *Wx, *Wax, *c1 = nullptr, *c2 = nullptr;
  CU(pool.alloc(&Wb, tot));
  CU(pool.alloc(&Wx, tot));
  CU(pool.alloc(&Wax, tot));
  ResidualOp ro;
  r = residual_setup(f, L, pool, nrhs, ro);
  if (r != RSRS_OK) return r;
  if (f->kind == RSRS_OP_CALLBACK) {
    CU(pool.alloc(&c1, tot));
    CU(pool.alloc(&c2, tot));
  }
  k_cm_to_rows<<<nblk(tot), 256, 0, st>>>(B, ld, f->perm_dev, f->n, nrhs, Wb);
  k_cm_to_rows<<<nblk(tot), 256, 0, st>>>(X, ld, f->perm_dev, f->n, nrhs, Wx);
  r = residual_apply(f, L, ro, Wx, Wax, nrhs, c1, c2);
  if (r != RSRS_OK) return r;
  k_sub<<<nblk(tot), 256, 0, st>>>(Wx, Wb, Wax, tot);
  k_rows_to_cm<<<nblk(tot), 256, 0, st>>>(Wx, f->perm_dev, f->n, nrhs, Rout, ld);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  return residual_check(f, ro);
}

}  // extern "C"

// ---- GMRES with the factor as right preconditioner ----------------------------------------
namespace {

// Krylov blocks are n x c row-major (c = nrhs <= 64), block i of a basis at base + i * n * c.
// Partial column dot products of w with blocks 0..kk-1 of V: grid (row chunks, kk); thread
// (col, lane) sums its column over the chunk's rows, the lanes are added in a fixed order.
constexpr int kDotRows = 2048;
__global__ void k_vdot_part(const double* __restrict__ V, const double* __restrict__ w, int64_t n, int c,
                            double* __restrict__ part) {
  __shared__ double red[256];
  const int col = threadIdx.x % c, lane = threadIdx.x / c, nl = blockDim.x / c;
  const int i = blockIdx.y;
  const double* v = V + (int64_t)i * n * c;
  const int64_t r0 = (int64_t)blockIdx.x * kDotRows, r1 = imin64(r0 + kDotRows, n);
  double acc = 0.0;
  if (lane < nl)
    for (int64_t r = r0 + lane; r < r1; r += nl) acc = fma(v[r * c + col], w[r * c + col], acc);
  red[threadIdx.x] = (lane < nl) ? acc : 0.0;
  __syncthreads();
  if (threadIdx.x < c) {
    double t = 0.0;
    for (int q = 0; q < nl; ++q) t += red[q * c + threadIdx.x];
    part[((int64_t)i * gridDim.x + blockIdx.x) * c + threadIdx.x] = t;
  }
}
// h[i][col] = sum over chunks (in order) of the partials.
__global__ void k_vdot_final(const double* __restrict__ part, int nchunk, int kk, int c, double* __restrict__ h) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kk * c) return;
  const int i = e / c, col = e % c;
  double t = 0.0;
  for (int q = 0; q < nchunk; ++q) t += part[((int64_t)i * nchunk + q) * c + col];
  h[e] = t;
}
// w[r][col] += sign * sum_i V_i[r][col] h[i][col]
__global__ void k_vcomb(double* __restrict__ w, const double* __restrict__ V, const double* __restrict__ h, int kk,
                        int64_t n, int c, double sign) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * c) return;
  const int col = (int)(e % c);
  double t = 0.0;
  for (int i = 0; i < kk; ++i) t = fma(V[(int64_t)i * n * c + e], h[i * c + col], t);
  w[e] += sign * t;
}
// out[r][col] = in[r][col] * s[col]
__global__ void k_colscale(const double* __restrict__ in, const double* __restrict__ sc, int64_t n, int c,
                           double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * c) out[e] = in[e] * sc[e % c];
}

struct Gmres {
  cudaStream_t st;
  int64_t n;
  int c;
  double *part, *h_dev;
  int nchunk;
  int64_t* launches;  // kernels launched, for the report
  // h[0..kk)[col] = V_i^T w, copied to the host
  rsrs_status dots(const double* V, int kk, const double* w, double* h_host) {
    const int threads = (256 / c) * c;
    k_vdot_part<<<dim3((unsigned)nchunk, (unsigned)kk), threads, 0, st>>>(V, w, n, c, part);
    k_vdot_final<<<nblk((int64_t)kk * c), 256, 0, st>>>(part, nchunk, kk, c, h_dev);
    *launches += 2;
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(h_host, h_dev, (size_t)kk * c * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return RSRS_OK;
  }
  rsrs_status comb(double* w, const double* V, const double* h_host, int kk, double sign) {
    CU(cudaMemcpyAsync(h_dev, h_host, (size_t)kk * c * sizeof(double), cudaMemcpyHostToDevice, st));
    k_vcomb<<<nblk(n * c), 256, 0, st>>>(w, V, h_dev, kk, n, c, sign);
    ++*launches;
    CU(cudaGetLastError());
    return RSRS_OK;
  }
  rsrs_status scale(const double* in, const double* s_host, double* out) {
    CU(cudaMemcpyAsync(h_dev, s_host, (size_t)c * sizeof(double), cudaMemcpyHostToDevice, st));
    k_colscale<<<nblk(n * c), 256, 0, st>>>(in, h_dev, n, c, out);
    ++*launches;
    CU(cudaGetLastError());
    return RSRS_OK;
  }
};

}  // namespace

extern "C" {

rsrs_status rsrs_gmres(const rsrs_factor* f, const double* B, double* X, int64_t ld, int32_t nrhs, double rtol,
                       int restart, int maxit, void* stream, rsrs_refine_report* rep) {
  rsrs_status r = check_block(f, B, ld, nrhs);
  if (r != RSRS_OK) return r;
  if (!X || nrhs > 64 || restart < 1 || restart > 64 || maxit < 1 || !(rtol >= 0.0))
    return fail(RSRS_E_INVAL, "gmres: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t nl = 0;  // kernels launched, for the report
  Launch L{st, &nl};
  DevPool pool;
  const int c = nrhs, m = restart;
  const int64_t n = f->n, tot = n * c;
  double *Wb, *Wx, *Ww, *V, *Z, *c1 = nullptr, *c2 = nullptr;
  Gmres gm{st, n, c, nullptr, nullptr, (int)cdiv(n, kDotRows), &nl};
  CU(pool.alloc(&Wb, tot));
  CU(pool.alloc(&Wx, tot));
  CU(pool.alloc(&Ww, tot));
  CU(pool.alloc(&V, (int64_t)(m + 1) * tot));
  CU(pool.alloc(&Z, (int64_t)m * tot));
  float* w32 = nullptr;  // the mixed factor's FP32 solve (the stored z_k keep GMRES exact in it)
  if (f->fd32) CU(pool.alloc(&w32, tot));
  CU(pool.alloc(&gm.part, (int64_t)(m + 1) * gm.nchunk * c));
  CU(pool.alloc(&gm.h_dev, (int64_t)(m + 1) * c));
  if (f->kind == RSRS_OP_CALLBACK) {
    CU(pool.alloc(&c1, tot));
    CU(pool.alloc(&c2, tot));
  }
  unsigned* bar = nullptr;  // the fused sweeps' barrier words, shared by this call's solves
  CU(pool.alloc(&bar, 4));
  CU(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st));
  ResidualOp ro;
  r = residual_setup(f, L, pool, c, ro);
  if (r != RSRS_OK) return r;
  // A y in the refinement's residual arithmetic
  auto apply_A = [&](const double* in, double* out) -> rsrs_status {
    return residual_apply(f, L, ro, in, out, c, c1, c2);
  };
  k_cm_to_rows<<<nblk(tot), 256, 0, st>>>(B, ld, f->perm_dev, n, c, Wb);
  ++nl;
  CU(cudaMemsetAsync(Wx, 0, tot * sizeof(double), st));
  std::vector<double> bn(c), beta(c), hcol((size_t)(m + 1) * c), h2((size_t)(m + 1) * c), sc(c);
  r = gm.dots(Wb, 1, Wb, bn.data());
  if (r != RSRS_OK) return r;
  for (double& v : bn) v = std::sqrt(v);
  // per column: Hessenberg columns (m+1) x m, Givens rotations, least-squares right-hand side
  std::vector<double> H((size_t)c * (m + 1) * m), cs((size_t)c * m), sn((size_t)c * m), g((size_t)c * (m + 1));
  rsrs_refine_report rr{};
  int total = 0, hist = 0;
  double rel = 0.0;
  bool first = true;
  for (;;) {
    // residual of the current iterate (the first one is b itself: x = 0)
    if (first) {
      CU(cudaMemcpyAsync(Ww, Wb, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      r = apply_A(Wx, Ww);
      if (r != RSRS_OK) return r;
      k_sub<<<nblk(tot), 256, 0, st>>>(Ww, Wb, Ww, tot);
      ++nl;
      CU(cudaGetLastError());
    }
    first = false;
    r = gm.dots(Ww, 1, Ww, beta.data());
    if (r != RSRS_OK) return r;
    rel = 0.0;
    for (int j = 0; j < c; ++j) {
      beta[j] = std::sqrt(beta[j]);
      rel = std::max(rel, beta[j] / std::max(bn[j], 1e-300));
    }
    if (!std::isfinite(rel)) return fail(RSRS_E_NONFINITE, "gmres: non-finite residual");
    if (hist < 64) rr.history[hist++] = rel;
    if (rel <= rtol || total >= maxit) break;
    for (int j = 0; j < c; ++j) sc[j] = beta[j] > 0.0 ? 1.0 / beta[j] : 0.0;
    r = gm.scale(Ww, sc.data(), V);
    if (r != RSRS_OK) return r;
    std::fill(g.begin(), g.end(), 0.0);
    for (int j = 0; j < c; ++j) g[(size_t)j * (m + 1)] = beta[j];
    int k = 0;
    for (; k < m && total < maxit; ++k) {
      double* Vk = V + (int64_t)k * tot;
      double* Zk = Z + (int64_t)k * tot;
      CU(cudaMemcpyAsync(Zk, Vk, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
      r = sweep_solve(f, L, Zk, c, 0, w32, bar);  // z_k = M^-1 v_k
      if (r != RSRS_OK) return r;
      r = apply_A(Zk, Ww);              // w = A z_k
      if (r != RSRS_OK) return r;
      // classical Gram-Schmidt, twice
      r = gm.dots(V, k + 1, Ww, hcol.data());
      if (r == RSRS_OK) r = gm.comb(Ww, V, hcol.data(), k + 1, -1.0);
      if (r == RSRS_OK) r = gm.dots(V, k + 1, Ww, h2.data());
      if (r == RSRS_OK) r = gm.comb(Ww, V, h2.data(), k + 1, -1.0);
      if (r != RSRS_OK) return r;
      for (size_t e = 0; e < (size_t)(k + 1) * c; ++e) hcol[e] += h2[e];
      std::vector<double> hn(c);
      r = gm.dots(Ww, 1, Ww, hn.data());
      if (r != RSRS_OK) return r;
      double est = 0.0;
      for (int j = 0; j < c; ++j) {
        hn[j] = std::sqrt(hn[j]);
        double* Hj = H.data() + (size_t)j * (m + 1) * m + (size_t)k * (m + 1);  // column k of H_j
        for (int i = 0; i <= k; ++i) Hj[i] = hcol[(size_t)i * c + j];
        Hj[k + 1] = hn[j];
        // previous rotations, then a new one that zeroes H[k+1][k]
        for (int i = 0; i < k; ++i) {
          const double a = Hj[i], b2 = Hj[i + 1];
          Hj[i] = cs[(size_t)j * m + i] * a + sn[(size_t)j * m + i] * b2;
          Hj[i + 1] = -sn[(size_t)j * m + i] * a + cs[(size_t)j * m + i] * b2;
        }
        const double a = Hj[k], b2 = Hj[k + 1];
        const double rho = std::hypot(a, b2);
        const double cc = rho > 0.0 ? a / rho : 1.0, ss = rho > 0.0 ? b2 / rho : 0.0;
        cs[(size_t)j * m + k] = cc;
        sn[(size_t)j * m + k] = ss;
        Hj[k] = rho;
        Hj[k + 1] = 0.0;
        double* gj = g.data() + (size_t)j * (m + 1);
        gj[k + 1] = -ss * gj[k];
        gj[k] = cc * gj[k];
        est = std::max(est, std::fabs(gj[k + 1]) / std::max(bn[j], 1e-300));
        sc[j] = hn[j] > 0.0 ? 1.0 / hn[j] : 0.0;
      }
      ++total;
      if (hist < 64) rr.history[hist++] = est;
      r = gm.scale(Ww, sc.data(), V + (int64_t)(k + 1) * tot);
      if (r != RSRS_OK) return r;
      if (est <= rtol) {
        ++k;
        break;
      }
    }
    // x += Z y with H y = g (upper triangular k x k per column)
    std::vector<double> y((size_t)k * c, 0.0);
    for (int j = 0; j < c; ++j) {
      const double* Hj = H.data() + (size_t)j * (m + 1) * m;
      const double* gj = g.data() + (size_t)j * (m + 1);
      for (int i = k - 1; i >= 0; --i) {
        double t = gj[i];
        for (int q = i + 1; q < k; ++q) t -= Hj[(size_t)q * (m + 1) + i] * y[(size_t)q * c + j];
        const double d = Hj[(size_t)i * (m + 1) + i];
        y[(size_t)i * c + j] = d != 0.0 ? t / d : 0.0;
      }
    }
    if (k > 0) {
      r = gm.comb(Wx, Z, y.data(), k, 1.0);
      if (r != RSRS_OK) return r;
    }
  }
  k_rows_to_cm<<<nblk(tot), 256, 0, st>>>(Wx, f->perm_dev, n, c, X, ld);
  ++nl;
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  r = residual_check(f, ro);
  if (r != RSRS_OK) return r;
  r = sweep_status(bar);
  if (r != RSRS_OK) return r;
  rr.iterations = total;
  rr.rel_residual = rel;
  rr.kernel_launches = nl;
  rr.residual_kind = ro.kind;
  if (rep) *rep = rr;
  if (rel > rtol) return fail(RSRS_E_NOT_CONVERGED, "gmres: residual " + std::to_string(rel) + " > rtol");
  return RSRS_OK;
}

rsrs_status rsrs_factor_stats(const rsrs_factor* f, rsrs_stats* out) {
  if (!f || !out) return fail(RSRS_E_INVAL, "null argument");
  *out = f->stats;
  return RSRS_OK;
}

rsrs_status rsrs_factor_box(const rsrs_factor* f, int64_t i, rsrs_box_view* v) {
  if (!f || !v || i < 0) return fail(RSRS_E_INVAL, "null argument");
  int64_t acc = 0;
  for (const GroupView& g : f->groups) {
    if (i < acc + (int64_t)g.h.size()) {
      const BoxDesc& d = g.h[i - acc];
      v->level = g.level;
      v->colour = g.colour;
      v->b = d.b;
      v->n = d.n;
      v->kp = d.kp;
      v->r = d.r;
      const int64_t w = (int64_t)d.kp + d.n;
      std::vector<int32_t> idx(fi_size(d.kp, d.r, d.n));
      CU(cudaMemcpy(idx.data(), f->fi + d.fi_off, idx.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
      auto orig = [&](int32_t t) { return f->perm[t - f->base]; };
      if (v->R)
        for (int q = 0; q < d.r; ++q) v->R[q] = orig(idx[q]);
      if (v->S)
        for (int q = 0; q < d.kp; ++q) v->S[q] = orig(idx[d.r + q]);
      if (v->N)
        for (int q = 0; q < d.n; ++q) v->N[q] = orig(idx[d.r + d.kp + q]);
      std::vector<double> fd(fd_size(d.kp, d.r, d.n));
      CU(cudaMemcpy(fd.data(), f->fd + d.fd_off, fd.size() * sizeof(double), cudaMemcpyDeviceToHost));
      const double* T = fd.data();
      const double* XRR = T + (int64_t)d.kp * d.r;
      const double* LcT = XRR + 2 * (int64_t)d.r * d.r;
      const double* Uc = LcT + (int64_t)d.r * w;
      if (v->T) std::memcpy(v->T, T, sizeof(double) * d.kp * d.r);
      if (v->XRR) std::memcpy(v->XRR, XRR, sizeof(double) * d.r * d.r);
      for (int64_t a = 0; a < d.r; ++a)
        for (int64_t q = 0; q < w; ++q) {
          double lc = LcT[a * w + q], uc = Uc[a * w + q];
          if (q < d.kp) {
            if (v->LcS) v->LcS[q * d.r + a] = lc;
            if (v->UcS) v->UcS[a * d.kp + q] = uc;
          } else {
            if (v->LcN) v->LcN[(q - d.kp) * d.r + a] = lc;
            if (v->UcN) v->UcN[a * d.n + (q - d.kp)] = uc;
          }
        }
      return RSRS_OK;
    }
    acc += (int64_t)g.h.size();
  }
  return fail(RSRS_E_INVAL, "box index out of range");
}

rsrs_status rsrs_factor_root(const rsrs_factor* f, int64_t* idx, double* A, int64_t* size_out) {
  if (!f) return fail(RSRS_E_INVAL, "null factor");
  if (size_out) *size_out = f->root_size;
  if (idx && f->root_size) {
    std::vector<int32_t> t(f->root_size);
    CU(cudaMemcpy(t.data(), f->root_idx, t.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int64_t q = 0; q < f->root_size; ++q) idx[q] = f->perm[t[q] - f->base];
  }
  if (A && f->root_size)
    CU(cudaMemcpy(A, f->root_A, f->root_size * f->root_size * sizeof(double), cudaMemcpyDeviceToHost));
  return RSRS_OK;
}

rsrs_status rsrs_factor_sketches(const rsrs_factor* f, double* Yh, double* Zh, double* Omh, double* Psh) {
  if (!f || !f->Y) return fail(RSRS_E_INVAL, "sketches were not kept (keep_sketches = 0)");
  const int64_t N = f->n, s = f->s;
  std::vector<double> tmp(N * s);
  const int64_t off = f->base * s;
  const double* src[4] = {f->Y + off, f->Z + off, f->Om + off, f->Ps + off};
  double* dst[4] = {Yh, Zh, Omh, Psh};
  for (int m = 0; m < 4; ++m) {
    if (!dst[m]) continue;
    CU(cudaMemcpy(tmp.data(), src[m], N * s * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t q = 0; q < N; ++q) std::memcpy(dst[m] + f->perm[q] * s, &tmp[q * s], s * sizeof(double));
  }
  return RSRS_OK;
}

}  // extern "C"

// ---- solve without device allocation ---------------------------------------------------------
// One static staging buffer per device (the module's copy of this array on that device).
static __device__ __align__(256) double g_noalloc_stage[RSRS_NOALLOC_MAX_ELEMS];
// ... and its FP32 copy, for a mixed-precision factor's FP32 solve
static __device__ __align__(256) float g_noalloc_stage32[RSRS_NOALLOC_MAX_ELEMS];
static __device__ __align__(16) unsigned g_noalloc_bar[4];  // the fused sweeps' barrier words

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {};
float* g_noalloc_addr32[kMaxDevices] = {};
unsigned* g_noalloc_bar_addr[kMaxDevices] = {};
}  // namespace

extern "C" rsrs_status rsrs_solve_noalloc(const rsrs_factor* f, double* F, int64_t ldf, int32_t nrhs, int adjoint,
                                          void* stream) {
  rsrs_status r = check_block(f, F, ldf, nrhs);
  if (r != RSRS_OK) return r;
  if (f->n * (int64_t)nrhs > RSRS_NOALLOC_MAX_ELEMS)
    return fail(RSRS_E_INVAL, "solve_noalloc: N * nrhs = " + std::to_string(f->n * (int64_t)nrhs) +
                                  " exceeds the static staging buffer of " +
                                  std::to_string(RSRS_NOALLOC_MAX_ELEMS) + " doubles");
  int dev = -1;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(RSRS_E_INVAL, "solve_noalloc: device ordinal out of range");
  double* W = nullptr;
  float* W32 = nullptr;
  unsigned* bar = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {  // set-up, once per device, with that device current
      void* p = nullptr;
      void* p32 = nullptr;
      CU(cudaGetSymbolAddress(&p, g_noalloc_stage));
      CU(cudaGetSymbolAddress(&p32, g_noalloc_stage32));
      void* pb = nullptr;
      CU(cudaGetSymbolAddress(&pb, g_noalloc_bar));
      g_noalloc_addr[dev] = static_cast<double*>(p);
      g_noalloc_addr32[dev] = static_cast<float*>(p32);
      g_noalloc_bar_addr[dev] = static_cast<unsigned*>(pb);
    }
    W = g_noalloc_addr[dev];
    W32 = g_noalloc_addr32[dev];
    bar = g_noalloc_bar_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  Launch L{st, nullptr};
  CU(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st));
  k_cm_to_rows<<<nblk(f->n * nrhs), 256, 0, st>>>(F, ldf, f->perm_dev, f->n, nrhs, W);
  r = sweep_solve(f, L, W, nrhs, adjoint, f->fd32 ? W32 : nullptr, bar);
  if (r != RSRS_OK) return r;
  k_rows_to_cm<<<nblk(f->n * nrhs), 256, 0, st>>>(W, f->perm_dev, f->n, nrhs, F, ldf);
  CU(cudaGetLastError());
  return RSRS_OK;
}

extern "C" rsrs_status rsrs_convert_selftest(const double* x, int64_t n, float* f, double* g, void* stream) {
  if (n < 0 || (n > 0 && (!x || !f || !g))) return fail(RSRS_E_INVAL, "convert_selftest: bad arguments");
  launch_convert_selftest(Launch{(cudaStream_t)stream, nullptr}, x, n, f, g);
  CU(cudaGetLastError());
  return RSRS_OK;
}

extern "C" rsrs_status rsrs_grid_wait_selftest(int64_t polls, int arrive, void* stream) {
  if (polls <= 0 || polls > ((int64_t)1 << 26) || (arrive != 0 && arrive != 1))
    return fail(RSRS_E_INVAL, "grid_wait_selftest: polls outside 1..2^26 or arrive not 0/1");
  cudaStream_t st = (cudaStream_t)stream;
  DevPool pool;
  unsigned* bar = nullptr;
  CU(pool.alloc(&bar, 4));
  CU(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st));
  if (!launch_grid_wait_selftest(Launch{st, nullptr}, bar, (long long)polls, arrive))
    return fail(RSRS_E_CUDA, "grid_wait_selftest: the cooperative launch was refused");
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  return sweep_status(bar) == RSRS_OK ? RSRS_OK : fail(RSRS_E_TIMEOUT, "grid_wait_selftest: the bounded wait expired");
}

extern "C" rsrs_status rsrs_wait_selftest(int64_t polls, int arrive, void* stream) {
  if (polls <= 0 || polls > ((int64_t)1 << 26) || (arrive != 0 && arrive != 1))
    return fail(RSRS_E_INVAL, "wait_selftest: polls outside 1..2^26 or arrive not 0/1");
  cudaStream_t st = (cudaStream_t)stream;
  DevPool pool;
  int* err = nullptr;
  CU(pool.alloc(&err, 1));
  CU(cudaMemsetAsync(err, 0, sizeof(int), st));
  launch_wait_selftest(Launch{st, nullptr}, (long long)polls, arrive, err);
  CU(cudaGetLastError());
  int herr = 0;
  CU(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (herr == kDevTimeout) return fail(RSRS_E_TIMEOUT, "wait_selftest: the bounded wait expired");
  if (herr != 0) return fail(RSRS_E_CUDA, "wait_selftest: unexpected device status " + std::to_string(herr));
  return RSRS_OK;
}
