// Batched FP64 kernels for one (level, colour) group of Algorithm 1.
//
// Every kernel runs over the boxes of one group (boxes with disjoint closed
// neighbourhoods, so their row sets never overlap).  A 1D grid of "items"
// (tiles, row chunks or whole boxes) is decoded on the device: each CTA scans
// the group's descriptors with the same per-box item count the host used to
// size the launch.
//
// GB300 note: FP64 runs at about 1 TFLOP/s on this part (1/64 of FP32), so
// these kernels are bound by the FP64 pipe as soon as a tile reuses its
// operands a few times; 64x64 output tiles with 16-deep K slices in shared
// memory are enough to keep the pipe busy.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>

#include <mutex>

#include "common.cuh"

namespace rsrs {

namespace {

constexpr int TB = 64;   // output tile edge
constexpr int TB_ = TB;
constexpr int KC = 16;   // K slice
constexpr int NT = 256;  // threads per tiled CTA (16 x 16), 4 x 4 outputs each

__host__ __device__ inline int64_t tri(int64_t t) { return t * (t + 1) / 2; }

__device__ inline void tri_decode(int64_t idx, int64_t& ti, int64_t& tj) {
  int64_t t = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
  while (tri(t) > idx) --t;
  while (tri(t + 1) <= idx) ++t;
  ti = t;
  tj = idx - tri(t);
}

__host__ __device__ inline int64_t cdv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <class F>
__device__ inline int find_item(const BoxDesc* desc, int nbox, int64_t item, F count, int64_t& local) {
  // the CTA scans the boxes' item counts in chunks of blockDim.x (one box per thread, block-wide
  // inclusive prefix sum), so the search costs a few dependent loads instead of one per box
  __shared__ int s_box;
  __shared__ int64_t s_local;
  __shared__ int64_t s_warp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (threadIdx.x == 0) s_box = -1;
  int64_t base = 0;
  for (int c0 = 0; c0 < nbox; c0 += blockDim.x) {
    const int i = c0 + (int)threadIdx.x;
    const int64_t c = i < nbox ? count(desc[i]) : 0;
    int64_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int64_t wbase = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) wbase += s_warp[w];
      total += s_warp[w];
    }
    incl += wbase;
    const int64_t excl = incl - c;
    if (i < nbox && c > 0 && item >= base + excl && item < base + incl) {
      s_box = i;
      s_local = item - base - excl;
    }
    __syncthreads();
    base += total;
    if (s_box >= 0 || item < base) break;  // uniform: read after the barrier
  }
  __syncthreads();
  local = s_local;
  return s_box;
}

template <typename T>
__device__ __forceinline__ T mad(T a, T b, T c);
template <>
__device__ __forceinline__ float mad<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double mad<double>(double a, double b, double c) { return fma(a, b, c); }

__device__ inline void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// Row source: row i of a row-major matrix of T, through an optional int32 index list.
template <typename T>
struct RowsT {
  const T* base;
  int64_t ld;
  const int32_t* idx;  // may be null: row i -> base + i*ld
  __device__ const T* row(int64_t i) const { return base + (idx ? (int64_t)idx[i] : i) * ld; }
};
template <typename T>
struct RowsWT {
  T* base;
  int64_t ld;
  const int32_t* idx;
  __device__ T* row(int64_t i) const { return base + (idx ? (int64_t)idx[i] : i) * ld; }
};
using Rows = RowsT<double>;
using RowsW = RowsWT<double>;

// C tile (64 x 64) = sum_t A[i][t] B[j][t] over t < K, rows gathered.  acc: 4 x 4 per thread,
// rows ty + 16a, cols tx + 16c (a, c < 4).  Operands are read in their storage type and used in CT.
template <typename CT, typename TA, typename TB>
__device__ void tile_nt(RowsT<TA> A, int64_t ma, RowsT<TB> B, int64_t mb, int64_t koff, int64_t K, int64_t i0,
                        int64_t j0, CT acc[4][4]) {
  __shared__ CT As[KC][TB_ + 1];
  __shared__ CT Bs[KC][TB_ + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const TA* arow = (i0 + lr < ma) ? A.row(i0 + lr) + koff : nullptr;
  const TB* brow = (j0 + lr < mb) ? B.row(j0 + lr) + koff : nullptr;
  for (int64_t k0 = 0; k0 < K; k0 += KC) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int64_t k = k0 + lk + u;
      As[lk + u][lr] = (arow && k < K) ? (CT)arow[k] : (CT)0;
      Bs[lk + u][lr] = (brow && k < K) ? (CT)brow[k] : (CT)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      CT a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty + 16 * u];
        b[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = mad<CT>(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
}

// A operand of C += alpha A B: element (i, q) of an m x K matrix, row-major or transposed storage.
template <typename T>
struct MatAT {
  const T* p;
  int64_t lda;
  bool trans;
  __device__ T at(int64_t i, int64_t q) const { return trans ? p[q * lda + i] : p[i * lda + q]; }
};
using MatA = MatAT<double>;

// A value in the compute type; FP64 -> FP32 by the integer-pipe rounding (the FP64 pipe, which
// the hardware conversion uses, is this part's scarcest unit).
template <typename CT, typename S>
__device__ inline CT to_ct(S v) {
  if constexpr (sizeof(CT) == 4 && sizeof(S) == 8)
    return f64_bits_to_f32((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v));
  else
    return (CT)v;
}
template <typename CT>
__device__ inline CT from_f64(double v) { return to_ct<CT>(v); }

// C[crow(i)][coff + t] += alpha * sum_q A(i,q) B[brow(q)][t] for the 64 x 64 tile (i0, t0);
// t ranges over ncols, q over K.
template <typename CT, typename TA, typename TB, typename TC>
__device__ void tile_acc(double alpha, MatAT<TA> A, int64_t m, int64_t K, RowsT<TB> B, int64_t boff,
                         RowsWT<TC> C, int64_t coff, int64_t ncols, int64_t i0, int64_t t0) {
  __shared__ CT As[KC][TB_ + 1];
  __shared__ CT Bs[KC][TB_ + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  CT acc[4][4] = {};
  for (int64_t q0 = 0; q0 < K; q0 += KC) {
    // A tile: 64 rows x 16 q
    if (!A.trans) {
      int lr = tid >> 2, lq = (tid & 3) * 4;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int64_t i = i0 + lr, q = q0 + lq + u;
        As[lq + u][lr] = (i < m && q < K) ? (CT)A.at(i, q) : (CT)0;
      }
    } else {
      int lr = tid & 63, lq = (tid >> 6) * 4;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int64_t i = i0 + lr, q = q0 + lq + u;
        As[lq + u][lr] = (i < m && q < K) ? (CT)A.at(i, q) : (CT)0;
      }
    }
    // B tile: 16 rows (q) x 64 cols (t)
    {
      int lq = tid >> 4, lt = (tid & 15) * 4;
      int64_t q = q0 + lq;
      const TB* brow = (q < K) ? B.row(q) + boff : nullptr;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int64_t t = t0 + lt + u;
        Bs[lq][lt + u] = (brow && t < ncols) ? (CT)brow[t] : (CT)0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      CT a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty + 16 * u];
        b[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = mad<CT>(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t i = i0 + ty + 16 * u;
    if (i >= m) continue;
    TC* crow = C.row(i) + coff;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t t = t0 + tx + 16 * v;
      if (t < ncols) {
        if constexpr (sizeof(TC) == 4)
          crow[t] = crow[t] + (TC)alpha * (TC)acc[u][v];
        else
          crow[t] = crow[t] + alpha * (double)acc[u][v];
      }
    }
  }
}

// ---- kernels -----------------------------------------------------------------

__global__ void k_copy_segments(const Seg* segs, int nseg, const int32_t* src, int32_t* dst) {
  int sidx = blockIdx.x;
  if (sidx >= nseg) return;
  Seg sg = segs[sidx];
  for (int64_t i = threadIdx.x; i < sg.len; i += blockDim.x) dst[sg.dst + i] = src[sg.src + i];
}

__global__ void k_gather_rows(const double* in, int64_t ld_in, const int32_t* rows, int64_t m, int64_t ncols,
                              double* out, int64_t ld_out) {
  int64_t i = blockIdx.x;
  if (i >= m) return;
  const double* src = in + (int64_t)rows[i] * ld_in;
  double* dst = out + i * ld_out;
  for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) dst[c] = src[c];
}

struct CntGram {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return 2 * tri(cdv(d.l, TB)); }
};
template <typename CT>
__global__ void __launch_bounds__(NT) k_gram(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntGram(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  int64_t per = tri(cdv(d.l, TB));
  int side = (int)(loc / per);
  int64_t ti, tj;
  tri_decode(loc % per, ti, tj);
  CT* wc = reinterpret_cast<CT*>(g.workc);
  RowsT<CT> W{wc + d.w_off + (int64_t)side * d.l * g.s, g.s, nullptr};
  CT acc[4][4] = {};
  tile_nt<CT>(W, d.l, W, d.l, 0, g.s, ti * TB, tj * TB, acc);
  CT* G = wc + d.g_off + (int64_t)side * d.l * d.l;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t i = ti * TB + ty + 16 * u;
    if (i >= d.l) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t j = tj * TB + tx + 16 * v;
      if (j < d.l) G[i * d.l + j] = acc[u][v];
    }
  }
}

// Blocked right-looking Cholesky, lower, in place on each l x l Gram, 64-wide panels.
struct CntPanel {
  int p;
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return (d.l > (int64_t)p * TB) ? 2 : 0; }
};
template <typename CT>
__global__ void __launch_bounds__(NT) k_chol_panel(GroupArgs g, int p) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntPanel{p}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int side = (int)loc;
  CT* G = reinterpret_cast<CT*>(g.workc) + d.g_off + (int64_t)side * d.l * d.l;
  const int64_t o = (int64_t)p * TB;
  const int nb = (int)imin64(TB, d.l - o);
  __shared__ CT S[TB][TB + 1];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int i = e / nb, j = e % nb;
    S[i][j] = G[(o + i) * d.l + o + j];
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    // column c: pivot, scale, rank-1 update of the trailing block (lower part)
    if (threadIdx.x == 0) {
      CT piv = S[c][c];
      if (!(piv > (CT)0) || !isfinite(piv)) {
        s_bad = 1;
        piv = (CT)1;
      }
      S[c][c] = sqrt(piv);
    }
    __syncthreads();
    CT dc = S[c][c];
    for (int i = c + 1 + threadIdx.x; i < nb; i += blockDim.x) S[i][c] /= dc;
    __syncthreads();
    int rem = nb - c - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int i = c + 1 + e / rem, j = c + 1 + e % rem;
      if (j <= i) S[i][j] -= S[i][c] * S[j][c];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_bad) set_err(g.err, kDevNonfinite);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int i = e / nb, j = e % nb;
    G[(o + i) * d.l + o + j] = (j <= i) ? S[i][j] : (CT)0;
  }
}

struct CntPanelRows {
  int p;
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    if (d.l <= (int64_t)p * TB) return 0;
    int64_t below = d.l - (int64_t)(p + 1) * TB;
    return 2 * ((below > 0 ? cdv(below, TB) : 0) + 1);
  }
};
// L_ip = G_ip L_pp^-T for the 64-row tiles below the diagonal block of panel p, and one more tile
// with the identity as right-hand side, whose solution L_pp^-T gives the inverse of the diagonal
// block (stored for the triangular solves of the projection).
template <typename CT>
__global__ void __launch_bounds__(NT) k_chol_trsm(GroupArgs g, int p) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntPanelRows{p}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  int64_t below = d.l - (int64_t)(p + 1) * TB;
  int64_t per = (below > 0 ? cdv(below, TB) : 0) + 1;
  int side = (int)(loc / per);
  int64_t ti = loc % per;
  const bool inv = (ti == per - 1);  // the identity tile
  CT* G = reinterpret_cast<CT*>(g.workc) + d.g_off + (int64_t)side * d.l * d.l;
  const int64_t o = (int64_t)p * TB;
  const int nb = (int)imin64(TB, d.l - o);
  const int64_t r0 = (int64_t)(p + 1) * TB + ti * TB;
  const int nr = inv ? nb : (int)imin64(TB, d.l - r0);
  extern __shared__ __align__(16) unsigned char trsm_raw[];
  CT* trsm_sm = reinterpret_cast<CT*>(trsm_raw);
  CT(*Lp)[TB + 1] = reinterpret_cast<CT(*)[TB + 1]>(trsm_sm);
  CT(*X)[TB + 1] = reinterpret_cast<CT(*)[TB + 1]>(trsm_sm + TB * (TB + 1));
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    int i = e / TB, j = e % TB;
    Lp[i][j] = (i < nb && j < nb) ? G[(o + i) * d.l + o + j] : (CT)0;
    if (inv)
      X[i][j] = (i == j && i < nb) ? (CT)1 : (CT)0;
    else
      X[i][j] = (i < nr && j < nb) ? G[(r0 + i) * d.l + o + j] : (CT)0;
  }
  __syncthreads();
  // x L^T = g, column by column; threads over the rows of the tile (4 threads per row, 16 cols each)
  for (int c = 0; c < nb; ++c) {
    if (threadIdx.x < nr) X[threadIdx.x][c] /= Lp[c][c];
    __syncthreads();
    for (int e = threadIdx.x; e < nr * (nb - c - 1); e += blockDim.x) {
      int i = e / (nb - c - 1), j = c + 1 + e % (nb - c - 1);
      X[i][j] -= X[i][c] * Lp[j][c];
    }
    __syncthreads();
  }
  if (inv) {  // X = L_pp^-T; store L_pp^-1 and L_pp^-T (zero padded to 64 x 64)
    CT* Li = reinterpret_cast<CT*>(g.workc) + d.li_off + ((int64_t)side * cdv(d.l, TB) + p) * 2 * TB * TB;
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
      int i = e / TB, j = e % TB;
      const bool in = (i < nb && j < nb);
      Li[e] = in ? X[j][i] : (CT)0;
      Li[TB * TB + e] = in ? X[i][j] : (CT)0;
    }
    return;
  }
  for (int e = threadIdx.x; e < nr * nb; e += blockDim.x) {
    int i = e / nb, j = e % nb;
    G[(r0 + i) * d.l + o + j] = X[i][j];
  }
}

struct CntUpdate {
  int p;
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    int64_t t = cdv(d.l, TB) - p - 1;
    return t > 0 ? 2 * tri(t) : 0;
  }
};
// G_ij -= L_ip L_jp^T for trailing tiles i >= j > p.
template <typename CT>
__global__ void __launch_bounds__(NT) k_chol_update(GroupArgs g, int p) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntUpdate{p}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  int64_t t = cdv(d.l, TB) - p - 1;
  int64_t per = tri(t);
  int side = (int)(loc / per);
  int64_t ti, tj;
  tri_decode(loc % per, ti, tj);
  ti += p + 1;
  tj += p + 1;
  CT* G = reinterpret_cast<CT*>(g.workc) + d.g_off + (int64_t)side * d.l * d.l;
  const int64_t o = (int64_t)p * TB;
  const int64_t nb = imin64(TB, d.l - o);
  RowsT<CT> L{G, d.l, nullptr};
  CT acc[4][4] = {};
  tile_nt<CT>(L, d.l, L, d.l, o, nb, ti * TB, tj * TB, acc);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t i = ti * TB + ty + 16 * u;
    if (i >= d.l) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t j = tj * TB + tx + 16 * v;
      if (j < d.l) G[i * d.l + j] -= acc[u][v];
    }
  }
}

// Gather the box's rows once, in the compute type: M = [Y_B | Z_B] (b x 2s) and the near-field
// test rows W = Om[B u N], V = Ps[B u N] (l x s each); 4 rows per CTA, M rows first.
struct CntGather {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return cdv(d.b, 4) + cdv(d.l, 4); }
};
template <typename CT>
__global__ void k_gather_box(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntGather(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int32_t* bn = g.iwork + d.bn_off;
  CT* wc = reinterpret_cast<CT*>(g.workc);
  const int64_t mb = cdv(d.b, 4);
  if (loc < mb) {
    __shared__ CT red[32];
    for (int rr = 0; rr < 4; ++rr) {
      int64_t i = loc * 4 + rr;
      if (i >= d.b) break;  // uniform
      const double* y = g.Y + (int64_t)bn[i] * g.s;
      const double* z = g.Z + (int64_t)bn[i] * g.s;
      CT* m = wc + d.mc_off + i * 2 * g.s;
      CT acc = 0;
      for (int64_t c = threadIdx.x; c < g.s; c += blockDim.x) {
        const CT a = from_f64<CT>(y[c]), bz = from_f64<CT>(z[c]);
        m[c] = a;
        m[g.s + c] = bz;
        acc = mad(a, a, mad(bz, bz, acc));
      }
      // squared row norm before nullification: the ID's noise floor
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        CT t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        g.work[d.sn_off + i] = (double)t;
      }
      __syncthreads();
    }
  } else {
    for (int rr = 0; rr < 4; ++rr) {
      int64_t i = (loc - mb) * 4 + rr;
      if (i >= d.l) break;
      const double* w = g.Om + (int64_t)bn[i] * g.s;
      const double* v = g.Ps + (int64_t)bn[i] * g.s;
      CT* W = wc + d.w_off + i * g.s;
      CT* V = wc + d.w_off + ((int64_t)d.l + i) * g.s;
      for (int64_t c = threadIdx.x; c < g.s; c += blockDim.x) {
        W[c] = from_f64<CT>(w[c]);
        V[c] = from_f64<CT>(v[c]);
      }
    }
  }
}

// M (FP64, for the CPQR) = the projected sketches from the compute-type workspace.
struct CntFinal {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return cdv(d.b, 4); }
};
template <typename CT>
__global__ void k_m_finalize(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntFinal(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const CT* mc = reinterpret_cast<const CT*>(g.workc) + d.mc_off;
  for (int rr = 0; rr < 4; ++rr) {
    int64_t i = loc * 4 + rr;
    if (i >= d.b) break;
    for (int64_t c = threadIdx.x; c < 2 * g.s; c += blockDim.x)
      g.work[d.m_off + i * 2 * g.s + c] = (double)mc[i * 2 * g.s + c];
  }
}

// X_side = M_side W_side^T (b x l), pass 0 -> x_off, pass 1 -> x2_off.
struct CntProjNT {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return 2 * cdv(d.b, TB) * cdv(d.l, TB); }
};
template <typename CT>
__global__ void __launch_bounds__(NT) k_proj_nt(GroupArgs g, int pass) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntProjNT(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  int64_t per = cdv(d.b, TB) * cdv(d.l, TB);
  int side = (int)(loc / per);
  int64_t rem = loc % per;
  int64_t ti = rem / cdv(d.l, TB), tj = rem % cdv(d.l, TB);
  CT* wc = reinterpret_cast<CT*>(g.workc);
  RowsT<CT> M{wc + d.mc_off + (int64_t)side * g.s, 2 * g.s, nullptr};
  RowsT<CT> W{wc + d.w_off + (int64_t)side * d.l * g.s, g.s, nullptr};
  CT acc[4][4] = {};
  tile_nt<CT>(M, d.b, W, d.l, 0, g.s, ti * TB, tj * TB, acc);
  CT* X = wc + (pass ? d.x2_off : d.x_off) + (int64_t)side * d.b * d.l;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t i = ti * TB + ty + 16 * u;
    if (i >= d.b) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t j = tj * TB + tx + 16 * v;
      if (j < d.l) X[i * d.l + j] = acc[u][v];
    }
  }
}

// X <- X G^-1 with G = L L^T, 64 rows per CTA, entirely as tile products: with the stored
// inverses of the 64 x 64 diagonal blocks of L,
//   forward  (U L^T = X):  U_j = (X_j - sum_{k<j} U_k L_jk^T) L_jj^-T
//   backward (X L = U):    X_j = (U_j - sum_{k>j} X_k L_kj) L_jj^-1
// Each block result is written back into X in place (the CTA owns its rows).
constexpr int SR = 64;
struct CntProjSolve {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return 2 * cdv(d.b, SR); }
};
template <typename CT>
__device__ void store_tile(CT* X, int64_t ld, int64_t r0, int64_t nr, int64_t c0, int64_t nc, CT acc[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t i = ty + 16 * u;
    if (i >= nr) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t c = tx + 16 * v;
      if (c < nc) X[(r0 + i) * ld + c0 + c] = acc[u][v];
    }
  }
}
template <typename CT>
__global__ void __launch_bounds__(NT) k_proj_solve(GroupArgs g, int pass) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntProjSolve(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t per = cdv(d.b, SR);
  const int side = (int)(loc / per);
  const int64_t r0 = (loc % per) * SR;
  const int64_t nr = imin64(SR, d.b - r0);
  const int64_t l = d.l, nblk = cdv(l, TB);
  CT* wc = reinterpret_cast<CT*>(g.workc);
  const CT* L = wc + d.g_off + (int64_t)side * l * l;
  const CT* Linv = wc + d.li_off + (int64_t)side * nblk * 2 * TB * TB;
  CT* X = wc + (pass ? d.x2_off : d.x_off) + (int64_t)side * d.b * l;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const RowsT<CT> Xr{X + r0 * l, l, nullptr};
  // forward
  for (int64_t jb = 0; jb < nblk; ++jb) {
    const int64_t c0 = jb * TB, nc = imin64(TB, l - c0);
    CT acc[4][4] = {};
    if (jb > 0) tile_nt<CT>(Xr, nr, RowsT<CT>{L + c0 * l, l, nullptr}, nc, 0, c0, 0, 0, acc);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int64_t i = ty + 16 * u, c = tx + 16 * v;
        acc[u][v] = (i < nr && c < nc) ? X[(r0 + i) * l + c0 + c] - acc[u][v] : (CT)0;
      }
    __syncthreads();
    store_tile<CT>(X, l, r0, nr, c0, nc, acc);
    __syncthreads();
    CT out[4][4] = {};
    tile_nt<CT>(RowsT<CT>{X + r0 * l + c0, l, nullptr}, nr, RowsT<CT>{Linv + jb * 2 * TB * TB, TB, nullptr}, nc, 0,
                nc, 0, 0, out);
    store_tile<CT>(X, l, r0, nr, c0, nc, out);
    __syncthreads();
  }
  // backward
  for (int64_t jb = nblk - 1; jb >= 0; --jb) {
    const int64_t c0 = jb * TB, nc = imin64(TB, l - c0);
    const int64_t q0 = c0 + nc;
    if (q0 < l) {  // X_j -= X_{>j} L_{>j, j}
      tile_acc<CT>(-1.0, MatAT<CT>{X + r0 * l + q0, l, false}, nr, l - q0, RowsT<CT>{L + q0 * l, l, nullptr}, c0,
                   RowsWT<CT>{X + r0 * l, l, nullptr}, c0, nc, 0, 0);
    }
    __syncthreads();
    CT out[4][4] = {};
    tile_nt<CT>(RowsT<CT>{X + r0 * l + c0, l, nullptr}, nr, RowsT<CT>{Linv + jb * 2 * TB * TB + TB * TB, TB, nullptr},
                nc, 0,
                nc, 0, 0, out);
    store_tile<CT>(X, l, r0, nr, c0, nc, out);
    __syncthreads();
  }
  if (pass) {  // accumulate the least-squares correction into the first-pass coefficients
    CT* X1 = wc + d.x_off + (int64_t)side * d.b * l + r0 * l;
    const CT* X2 = X + r0 * l;
    for (int64_t e = threadIdx.x; e < nr * l; e += blockDim.x) X1[e] += X2[e];
  }
}

// M_side -= X_side W_side  (b x s).
struct CntProjAcc {
  int64_t s;
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return 2 * cdv(d.b, TB) * cdv(s, TB); }
};
template <typename CT>
__global__ void __launch_bounds__(NT) k_proj_acc(GroupArgs g, int pass) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntProjAcc{g.s}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  int64_t nt = cdv(g.s, TB);
  int64_t per = cdv(d.b, TB) * nt;
  int side = (int)(loc / per);
  int64_t rem = loc % per;
  int64_t ti = rem / nt, tt = rem % nt;
  CT* wc = reinterpret_cast<CT*>(g.workc);
  MatAT<CT> X{wc + (pass ? d.x2_off : d.x_off) + (int64_t)side * d.b * d.l, d.l, false};
  RowsT<CT> W{wc + d.w_off + (int64_t)side * d.l * g.s, g.s, nullptr};
  RowsWT<CT> M{wc + d.mc_off, 2 * g.s, nullptr};
  tile_acc<CT>(-1.0, X, d.b, d.l, W, 0, M, (int64_t)side * g.s, g.s, ti * TB, tt * TB);
}

// Largest row norm of the box's sketch [Y_B | Z_B] before nullification.
__device__ inline double id_scale(const double* sn, int b) {
  double m = 0.0;
  for (int i = 0; i < b; ++i) m = fmax(m, sn[i]);
  return sqrt(m);
}

// Thresholds of the dependent-pivot rule of the ID (Sec. 2.3 greedy pivoted QR at the fixed rank of
// Sec. 4.5).  tau: residuals below tau |R_00| are numerically dependent, 64 eps max(b, 2s) bounding
// the rounding of the Householder steps on the b x 2s sketch.  floor_abs: the rounding level of
// block nullification (Sec. 4.1) when the box's far field is exactly zero -- each entry of the
// nullified sketch is a sum of s products of a sketch row with a unit vector, rounded to about eps
// times the row's norm, so a 2s-column row keeps about eps sqrt(2s) of the largest
// pre-nullification row; a box with no far field (a sparse operator's box before fill-in reaches
// it) then has only dependent pivots and T = 0.
struct IdThresholds {
  double tau, floor_abs;
};
__device__ inline IdThresholds id_thresholds(int b, int64_t s, const double* sn) {
  IdThresholds t;
  t.tau = 64.0 * DBL_EPSILON * (double)max((int64_t)b, 2 * s);
  t.floor_abs = DBL_EPSILON * sqrt(2.0 * (double)s) * id_scale(sn, b);
  return t;
}

// Column-pivoted Householder QR of M^T (pivoting over the b rows of M), kp steps.
// One CTA per box; the reflectors act on the 2s columns of M in place.
// Once the largest remaining residual is <= tau |R_00| or <= the nullification's rounding floor
// (id_thresholds) the remaining pivots are numerically dependent and are taken in ascending local
// (tree) order; the first such step is stored after the permutation for the interpolation matrix.
__global__ void __launch_bounds__(512) k_cpqr(GroupArgs g) {
  const BoxDesc d = g.desc[blockIdx.x];
  const int b = d.b, kp = d.kp;
  const int64_t c = 2 * g.s;
  double* M = g.work + d.m_off;
  double* Rp = g.work + d.cp_off;  // kp x b, Rp[j][local row id]: row j of R, columns by point
  int32_t* perm = g.iwork + d.pv_off;
  extern __shared__ double sm[];
  double* nrm = sm;                       // b
  int* rid = (int*)(sm + b);              // b
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double s_vn2, s_r00;
  __shared__ int s_j0;
  const IdThresholds th = id_thresholds(b, g.s, g.work + d.sn_off);
  const double tau = th.tau, floor_abs = th.floor_abs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < b; i += blockDim.x) rid[i] = i;
  if (threadIdx.x == 0) {
    s_r00 = -1.0;
    s_j0 = kp;
  }
  // initial squared row norms
  for (int i = warp; i < b; i += nw) {
    const double* row = M + (int64_t)i * c;
    double acc = 0.0;
    for (int64_t t = lane; t < c; t += 32) acc = fma(row[t], row[t], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) nrm[i] = acc;
  }
  __syncthreads();
  for (int j = 0; j < kp; ++j) {
    // pivot: largest residual norm, ties to the lowest local index
    double bv = -1.0;
    int bp = -1;
    for (int pos = j + threadIdx.x; pos < b; pos += blockDim.x) {
      double v = nrm[pos];
      if (v > bv || (v == bv && rid[pos] < rid[bp])) {
        bv = v;
        bp = pos;
      }
    }
    for (int o = 16; o; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (op >= 0 && (ov > bv || (ov == bv && (bp < 0 || rid[op] < rid[bp])))) {
        bv = ov;
        bp = op;
      }
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v0 = -1.0;
      int p0 = -1;
      for (int w = 0; w < nw; ++w) {
        int op = red_i[w];
        double ov = red_v[w];
        if (op >= 0 && (ov > v0 || (ov == v0 && (p0 < 0 || rid[op] < rid[p0])))) {
          v0 = ov;
          p0 = op;
        }
      }
      if (p0 < 0) {  // no finite candidate: keep the order, report
        p0 = j;
        set_err(g.err, kDevNonfinite);
      }
      if (s_j0 == kp && (sqrt(v0) <= floor_abs || (s_r00 >= 0.0 && sqrt(v0) <= tau * s_r00) || v0 == 0.0)) s_j0 = j;
      if (s_j0 <= j) {  // dependent: lowest remaining local index
        p0 = j;
        for (int pos = j + 1; pos < b; ++pos)
          if (rid[pos] < rid[p0]) p0 = pos;
      }
      if (p0 != j) {
        int ti = rid[j];
        rid[j] = rid[p0];
        rid[p0] = ti;
        double tv = nrm[j];
        nrm[j] = nrm[p0];
        nrm[p0] = tv;
      }
    }
    __syncthreads();
    // reflector from the pivot row x = M[rid[j]][j:]
    double* x = M + (int64_t)rid[j] * c;
    {
      double acc = 0.0;
      for (int64_t t = j + threadIdx.x; t < c; t += blockDim.x) acc = fma(x[t], x[t], acc);
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) red_v[warp] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double a2 = 0.0;
        for (int w = 0; w < nw; ++w) a2 += red_v[w];
        double alpha = sqrt(a2);
        double x0 = x[j];
        double sg = (x0 >= 0.0) ? 1.0 : -1.0;
        s_vn2 = 2.0 * alpha * (alpha + fabs(x0));
        if (j == 0) s_r00 = alpha;
        Rp[(int64_t)j * b + rid[j]] = -sg * alpha;
        x[j] = x0 + sg * alpha;
      }
      __syncthreads();
    }
    const double vn2 = s_vn2;
    for (int pos = j + 1 + warp; pos < b; pos += nw) {
      double* row = M + (int64_t)rid[pos] * c;
      double w = 0.0;
      if (vn2 > 0.0) {
        for (int64_t t = j + lane; t < c; t += 32) w = fma(row[t], x[t], w);
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      }
      const double f = (vn2 > 0.0) ? 2.0 * w / vn2 : 0.0;
      double nn = 0.0;
      for (int64_t t = j + lane; t < c; t += 32) {
        double v = fma(-f, x[t], row[t]);
        row[t] = v;
        if (t > j) nn = fma(v, v, nn);
      }
      for (int o = 16; o; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
      if (lane == 0) {
        nrm[pos] = nn;
        Rp[(int64_t)j * b + rid[pos]] = row[j];
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < b; i += blockDim.x) perm[i] = rid[i];
  if (threadIdx.x == 0) perm[b] = s_j0;
}

// Cluster version of the CPQR: CPQR_C CTAs per box (one thread-block cluster), CTA r owning the
// columns [r*cs, (r+1)*cs) of M.  Per pivot step the row dot products with the Householder vector
// and the updated row norms are summed over the cluster through distributed shared memory
// (partials summed in rank order, so every CTA holds identical norms and picks the same pivot);
// two hardware cluster barriers per step.  Same pivot rule as k_cpqr.
constexpr int CPQR_C = 8;
__global__ void __launch_bounds__(256) k_cpqr_cluster(GroupArgs g) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const BoxDesc d = g.desc[blockIdx.x / CPQR_C];
  const int b = d.b, kp = d.kp;
  const int64_t c = 2 * g.s;
  const int64_t cs = ((c + CPQR_C - 1) / CPQR_C + 31) / 32 * 32;
  const int64_t t_lo = imin64((int64_t)rank * cs, c), t_hi = imin64(t_lo + cs, c);
  double* M = g.work + d.m_off;
  double* Rp = g.work + d.cp_off;
  int32_t* perm = g.iwork + d.pv_off;
  extern __shared__ double csm[];
  double* nrm = csm;            // b, replicated in every CTA
  double* wpart = csm + b;      // b, this CTA's partial dot products
  double* npart = csm + 2 * b;  // b, this CTA's partial norms
  int* rid = (int*)(csm + 3 * b);
  __shared__ double s_x0, s_vn2, s_r00;
  __shared__ int s_j0;
  const IdThresholds th = id_thresholds(b, g.s, g.work + d.sn_off);
  const double tau = th.tau, floor_abs = th.floor_abs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < b; i += blockDim.x) rid[i] = i;
  if (threadIdx.x == 0) {
    s_r00 = -1.0;
    s_j0 = kp;
  }
  // initial squared row norms
  for (int i = warp; i < b; i += nw) {
    const double* row = M + (int64_t)i * c;
    double acc = 0.0;
    for (int64_t t = t_lo + lane; t < t_hi; t += 32) acc = fma(row[t], row[t], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) npart[i] = acc;
  }
  cluster.sync();
  for (int i = threadIdx.x; i < b; i += blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < CPQR_C; ++q) v += cluster.map_shared_rank(npart, q)[i];
    nrm[i] = v;
  }
  __syncthreads();
  for (int j = 0; j < kp; ++j) {
    if (threadIdx.x == 0) {  // identical in every CTA: same norms, same order
      double v0 = -1.0;
      int p0 = -1;
      for (int pos = j; pos < b; ++pos) {
        double v = nrm[pos];
        if (v > v0 || (v == v0 && p0 >= 0 && rid[pos] < rid[p0])) {
          v0 = v;
          p0 = pos;
        }
      }
      if (p0 < 0) {
        p0 = j;
        if (rank == 0) set_err(g.err, kDevNonfinite);
      }
      if (s_j0 == kp && (sqrt(v0) <= floor_abs || (s_r00 >= 0.0 && sqrt(v0) <= tau * s_r00) || v0 == 0.0)) s_j0 = j;
      if (s_j0 <= j) {
        p0 = j;
        for (int pos = j + 1; pos < b; ++pos)
          if (rid[pos] < rid[p0]) p0 = pos;
      }
      if (p0 != j) {
        int ti = rid[j];
        rid[j] = rid[p0];
        rid[p0] = ti;
        double tv = nrm[j];
        nrm[j] = nrm[p0];
        nrm[p0] = tv;
      }
      const double alpha = sqrt(fmax(nrm[j], 0.0));
      const double x0 = M[(int64_t)rid[j] * c + j];
      const double sg = (x0 >= 0.0) ? 1.0 : -1.0;
      s_x0 = x0 + sg * alpha;  // v_j
      s_vn2 = 2.0 * alpha * (alpha + fabs(x0));
      if (j == 0) s_r00 = alpha;
      if (rank == 0) Rp[(int64_t)j * b + rid[j]] = -sg * alpha;
    }
    __syncthreads();
    const double vj = s_x0, vn2 = s_vn2;
    const double* x = M + (int64_t)rid[j] * c;
    // partial dot products of the remaining rows with v over this CTA's columns
    for (int pos = j + 1 + warp; pos < b; pos += nw) {
      const double* row = M + (int64_t)rid[pos] * c;
      double w = 0.0;
      for (int64_t t = imax64(t_lo, j) + lane; t < t_hi; t += 32) w = fma(row[t], t == j ? vj : x[t], w);
      for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      if (lane == 0) wpart[pos] = w;
    }
    cluster.sync();
    for (int pos = j + 1 + warp; pos < b; pos += nw) {
      double w = 0.0;
      for (int q = 0; q < CPQR_C; ++q) w += cluster.map_shared_rank(wpart, q)[pos];
      const double f = (vn2 > 0.0) ? 2.0 * w / vn2 : 0.0;
      double* row = M + (int64_t)rid[pos] * c;
      double nn = 0.0;
      for (int64_t t = imax64(t_lo, j) + lane; t < t_hi; t += 32) {
        double v = fma(-f, t == j ? vj : x[t], row[t]);
        row[t] = v;
        if (t > j) nn = fma(v, v, nn);
        else Rp[(int64_t)j * b + rid[pos]] = v;  // t == j lives in exactly one CTA
      }
      for (int o = 16; o; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
      if (lane == 0) npart[pos] = nn;
    }
    cluster.sync();
    for (int pos = j + 1 + threadIdx.x; pos < b; pos += blockDim.x) {
      double v = 0.0;
      for (int q = 0; q < CPQR_C; ++q) v += cluster.map_shared_rank(npart, q)[pos];
      nrm[pos] = v;
    }
    __syncthreads();
  }
  if (rank == 0) {
    for (int i = threadIdx.x; i < b; i += blockDim.x) perm[i] = rid[i];
    if (threadIdx.x == 0) perm[b] = s_j0;
  }
  cluster.sync();  // keep every CTA's shared memory alive until the last remote read
}

// Mixed-precision CPQR with the box's projected sketch resident in distributed shared memory: a
// cluster of C CTAs (C = 1..16) per box, CTA r holding columns [r*cs, (r+1)*cs) of all b rows of
// the FP32 sketch M, so the k' reflector steps never go back to global memory.  The arithmetic on
// M is FP32 (M carries the FP32 rounding of the projections already), including the warp and
// cluster sums of the dot products and row norms and the Householder scalars: this part's FP64
// pipe is 1/64 of its FP32 pipe, and FP64 work on the serial path of every step would dominate it.
// The pivot decisions stay in FP64: the residual norms are held as FP64, the largest is found by
// comparing their bit patterns (monotone for non-negative doubles; ties to the lowest tree index),
// and the dependent-pivot test of k_cpqr is evaluated on them (squared, no square roots).  The two
// cluster sums of every step are pushed: each CTA stores its partial sums into a slot of every
// CTA's shared memory (remote stores, no round trips) and, after the cluster barrier, adds its C
// local slots in rank order.  Output as k_cpqr_cluster: R rows by point (FP64), permutation and
// first dependent step.
__host__ __device__ inline size_t cpqr32_head_bytes(int b, int C) {
  return (((size_t)b * 8 + (size_t)2 * C * b * 4 + (size_t)b * 4 + (size_t)b * 4) + 15) & ~(size_t)15;
}
__global__ void __launch_bounds__(1024, 1) k_cpqr32_cluster(GroupArgs g, int cs, int in_global) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const BoxDesc d = g.desc[blockIdx.x / C];
  const int b = d.b, kp = d.kp;
  const int64_t c = 2 * g.s;
  const int64_t t_lo = imin64((int64_t)rank * cs, c), t_hi = imin64(t_lo + cs, c);
  float* Mg = reinterpret_cast<float*>(g.workc) + d.mc_off;
  double* Rp = g.work + d.cp_off;
  int32_t* perm = g.iwork + d.pv_off;
  extern __shared__ double csm[];
  double* nrm = csm;                                         // b, replicated in every CTA
  float* wbuf = reinterpret_cast<float*>(csm + b);          // C x b: partial dot products, slot per CTA
  float* nbuf = wbuf + (size_t)C * b;                        // C x b: partial squared norms, slot per CTA
  float* fvec = nbuf + (size_t)C * b;                        // b, reflector coefficients
  int* rid = reinterpret_cast<int*>(fvec + b);               // b
  // this CTA's b x (t_hi - t_lo) slice of M: in shared memory (row pitch cs), or in place in the
  // workspace when the box is too large for the cluster's shared memory (row pitch 2s)
  float* S = in_global ? Mg + t_lo
                       : reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(csm) + cpqr32_head_bytes(b, C));
  const int64_t lds = in_global ? c : (int64_t)cs;
  __shared__ unsigned long long red_v[32];
  __shared__ int red_i[32], red_m[32];
  __shared__ double s_r00;
  __shared__ float s_vj, s_f2;
  __shared__ int s_j0;
  __shared__ double s_floor2, s_tau2;
  if (threadIdx.x == 0) {  // FP64 work once per CTA, not per thread (the FP64 pipe is narrow)
    const IdThresholds th = id_thresholds(b, g.s, g.work + d.sn_off);
    s_floor2 = th.floor_abs * th.floor_abs;
    s_tau2 = th.tau * th.tau;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int wid = (int)(t_hi - t_lo);
  // a warp-reduced partial sum of row pos goes to slot `rank` of every CTA's buffer (lane q -> CTA q)
  auto push = [&](float* buf, int pos, float v) {
    if (lane < C) cluster.map_shared_rank(buf, lane)[(size_t)rank * b + pos] = v;
  };
  auto sum_slots = [&](const float* buf, int pos) {
    float v = 0.f;
    for (int q = 0; q < C; ++q) v += buf[(size_t)q * b + pos];
    return v;
  };
  for (int i = threadIdx.x; i < b; i += blockDim.x) rid[i] = i;
  if (threadIdx.x == 0) {
    s_r00 = -1.0;
    s_j0 = kp;
  }
  // slice into shared memory; initial partial squared row norms
  for (int i = warp; i < b; i += nw) {
    const float* row = Mg + (int64_t)i * c + t_lo;
    float* srow = S + (int64_t)i * lds;
    float acc = 0.f;
    for (int t = lane; t < wid; t += 32) {
      const float v = row[t];
      if (!in_global) srow[t] = v;
      acc = fmaf(v, v, acc);
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    push(nbuf, i, acc);
  }
  cluster.sync();
  for (int pos = threadIdx.x; pos < b; pos += blockDim.x) nrm[pos] = (double)sum_slots(nbuf, pos);
  __syncthreads();
  // candidate order: larger norm bits first, then the lower tree index
  auto better = [&](unsigned long long v, int p, unsigned long long bv, int bp) {
    return p >= 0 && (bp < 0 || v > bv || (v == bv && rid[p] < rid[bp]));
  };
  for (int j = 0; j < kp; ++j) {
    // pivot candidates (identical in every CTA): the largest residual norm, and the lowest tree
    // index (taken once the remaining pivots are numerically dependent)
    unsigned long long bv = 0ull;
    int bp = -1, mp = -1;
    for (int pos = j + threadIdx.x; pos < b; pos += blockDim.x) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(nrm[pos]);
      if (better(v, pos, bv, bp)) {
        bv = v;
        bp = pos;
      }
      if (mp < 0 || rid[pos] < rid[mp]) mp = pos;
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int op = __shfl_xor_sync(0xffffffffu, bp, o);
      const int om = __shfl_xor_sync(0xffffffffu, mp, o);
      if (better(ov, op, bv, bp)) {
        bv = ov;
        bp = op;
      }
      if (om >= 0 && (mp < 0 || rid[om] < rid[mp])) mp = om;
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bp;
      red_m[warp] = mp;
    }
    __syncthreads();
    if (warp == 0) {
      bv = lane < nw ? red_v[lane] : 0ull;
      bp = lane < nw ? red_i[lane] : -1;
      mp = lane < nw ? red_m[lane] : -1;
      for (int o = 16; o; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int om = __shfl_xor_sync(0xffffffffu, mp, o);
        if (better(ov, op, bv, bp)) {
          bv = ov;
          bp = op;
        }
        if (om >= 0 && (mp < 0 || rid[om] < rid[mp])) mp = om;
      }
    }
    if (threadIdx.x == 0) {
      const double floor2 = s_floor2, tau2 = s_tau2;
      int p0 = bp;
      const double dv0 = p0 >= 0 ? __longlong_as_double((long long)bv) : 0.0;
      if (p0 < 0 || !isfinite(dv0)) {
        p0 = j;
        if (rank == 0) set_err(g.err, kDevNonfinite);
      }
      if (s_j0 == kp && (dv0 <= floor2 || (s_r00 >= 0.0 && dv0 <= tau2 * s_r00 * s_r00) || dv0 == 0.0)) s_j0 = j;
      if (s_j0 <= j) p0 = mp >= 0 ? mp : j;
      if (p0 != j) {
        const int ti = rid[j];
        rid[j] = rid[p0];
        rid[p0] = ti;
        const double tv = nrm[j];
        nrm[j] = nrm[p0];
        nrm[p0] = tv;
      }
      // x0 = M[pivot][j] lives in the CTA that owns column j
      const int owner = (int)(j / cs);
      const float x0 = in_global ? Mg[(int64_t)rid[j] * c + j]
                                 : cluster.map_shared_rank(S, owner)[(int64_t)rid[j] * cs + (j - (int64_t)owner * cs)];
      const float alpha = sqrtf((float)fmax(nrm[j], 0.0));
      const float sg = (x0 >= 0.f) ? 1.f : -1.f;
      const float vn2 = 2.f * alpha * (alpha + fabsf(x0));
      s_vj = x0 + sg * alpha;
      s_f2 = vn2 > 0.f ? 2.f / vn2 : 0.f;
      if (j == 0) s_r00 = (double)alpha;
      if (rank == 0) Rp[(int64_t)j * b + rid[j]] = (double)(-sg * alpha);
    }
    __syncthreads();
    const float vj = s_vj, f2 = s_f2;
    const float* xs = S + (int64_t)rid[j] * lds;
    const int t0 = (int)(imax64(t_lo, j) - t_lo);  // first local column of the reflector
    const int tj = (int)(j - t_lo);                 // local index of column j (in range for its owner)
    // partial dot products of the remaining rows with v over this CTA's columns
    // column j (in its owner CTA only, where t0 == tj) uses v_j; the other columns x itself
    const bool own_j = (tj >= 0 && tj < wid);  // this CTA holds column j (then t0 == tj)
    const int t1 = own_j ? t0 + 1 : t0;
    for (int pos = j + 1 + warp; pos < b; pos += nw) {
      const float* row = S + (int64_t)rid[pos] * lds;
      float w = (own_j && lane == 0) ? row[tj] * vj : 0.f;
      for (int t = t1 + lane; t < wid; t += 32) w = fmaf(row[t], xs[t], w);
      for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      push(wbuf, pos, w);
    }
    cluster.sync();
    for (int pos = j + 1 + threadIdx.x; pos < b; pos += blockDim.x) fvec[pos] = sum_slots(wbuf, pos) * f2;
    __syncthreads();
    for (int pos = j + 1 + warp; pos < b; pos += nw) {
      const float f = fvec[pos];
      float* row = S + (int64_t)rid[pos] * lds;
      if (own_j && lane == 0) {  // R[j][pos], written by the CTA that owns column j
        const float v = fmaf(-f, vj, row[tj]);
        row[tj] = v;
        Rp[(int64_t)j * b + rid[pos]] = (double)v;
      }
      float nn = 0.f;
      for (int t = t1 + lane; t < wid; t += 32) {
        const float v = fmaf(-f, xs[t], row[t]);
        row[t] = v;
        nn = fmaf(v, v, nn);
      }
      for (int o = 16; o; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
      push(nbuf, pos, nn);
    }
    cluster.sync();
    for (int pos = j + 1 + threadIdx.x; pos < b; pos += blockDim.x) nrm[pos] = (double)sum_slots(nbuf, pos);
    __syncthreads();
  }
  if (rank == 0) {
    for (int i = threadIdx.x; i < b; i += blockDim.x) perm[i] = rid[i];
    if (threadIdx.x == 0) perm[b] = s_j0;
  }
  cluster.sync();  // keep every CTA's shared memory alive until the last remote access
}

// T = R11^-1 R12 (truncated at the first dependent pivot), R/S/N lists, new active list.
__global__ void __launch_bounds__(256) k_id_finish(GroupArgs g) {
  const BoxDesc d = g.desc[blockIdx.x];
  const int b = d.b, kp = d.kp, r = d.r;
  const double* Rp = g.work + d.cp_off;
  int32_t* perm = g.iwork + d.pv_off;
  const int32_t* bn = g.iwork + d.bn_off;
  double* T = g.fd + fd_T(d);
  int32_t* Rl = g.fi + fi_R(d);
  int32_t* Sl = g.fi + fi_S(d);
  int32_t* Nl = g.fi + fi_N(d);
  extern __shared__ int ism[];
  int* rloc = ism;          // r: sorted redundant local indices
  int* rcol = ism + r;      // r: column of T for permuted position kp+q
  int* ssort = ism + 2 * r; // kp: skeleton local indices, ascending
  __shared__ int s_j0;
  // sorted R: rank of each redundant local index
  for (int q = threadIdx.x; q < r; q += blockDim.x) {
    int v = perm[kp + q], rank = 0;
    for (int u = 0; u < r; ++u) rank += perm[kp + u] < v;
    rloc[rank] = v;
    rcol[q] = rank;
  }
  for (int q = threadIdx.x; q < kp; q += blockDim.x) {
    int v = perm[q], rank = 0;
    for (int u = 0; u < kp; ++u) rank += perm[u] < v;
    ssort[rank] = v;
  }
  if (threadIdx.x == 0) s_j0 = perm[b];  // first dependent pivot, from the CPQR
  __syncthreads();
  const int j0 = s_j0;
  // back substitution, one thread per column of R12
  for (int q = threadIdx.x; q < r; q += blockDim.x) {
    const int col = rcol[q];
    for (int j = kp - 1; j >= 0; --j) {
      double v = 0.0;
      if (j < j0) {
        v = Rp[(int64_t)j * b + perm[kp + q]];
        for (int u = j + 1; u < j0; ++u) v -= Rp[(int64_t)j * b + perm[u]] * T[(int64_t)u * r + col];
        v /= Rp[(int64_t)j * b + perm[j]];
      }
      T[(int64_t)j * r + col] = v;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < r; q += blockDim.x) {
    Rl[q] = bn[rloc[q]];
    perm[kp + q] = rloc[q];  // the tail of perm now holds R in ascending order
  }
  for (int q = threadIdx.x; q < kp; q += blockDim.x) {
    Sl[q] = bn[perm[q]];
    g.act[d.act_off + q] = bn[ssort[q]];
  }
  for (int q = threadIdx.x; q < d.n; q += blockDim.x) Nl[q] = bn[d.b + q];
}

// E and F on the sketches: Y_R -= T^T Y_S, Z_R -= T^T Z_S, Om_S += T Om_R, Ps_S += T Ps_R.
struct CntEF {
  int64_t s;
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    return (2 * cdv(d.r, TB) + 2 * cdv(d.kp, TB)) * cdv(s, TB);
  }
};
template <typename CT>
__global__ void __launch_bounds__(NT) k_ef_update(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntEF{g.s}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t nt = cdv(g.s, TB);
  const int64_t tr = cdv(d.r, TB), tk = cdv(d.kp, TB);
  int64_t row_tile = loc / nt, tt = loc % nt;
  const int32_t* Rl = g.fi + fi_R(d);
  const int32_t* Sl = g.fi + fi_S(d);
  const double* T = g.fd + fd_T(d);
  int job;
  if (row_tile < tr) job = 0;
  else if (row_tile < 2 * tr) { job = 1; row_tile -= tr; }
  else if (row_tile < 2 * tr + tk) { job = 2; row_tile -= 2 * tr; }
  else { job = 3; row_tile -= 2 * tr + tk; }
  if (job < 2) {
    double* Mx = job == 0 ? g.Y : g.Z;
    tile_acc<CT>(-1.0, MatA{T, d.r, true}, d.r, d.kp, Rows{Mx, g.s, Sl}, 0, RowsW{Mx, g.s, Rl}, 0, g.s,
             row_tile * TB, tt * TB);
  } else {
    double* Mx = job == 2 ? g.Om : g.Ps;
    tile_acc<CT>(1.0, MatA{T, d.r, false}, d.kp, d.r, Rows{Mx, g.s, Rl}, 0, RowsW{Mx, g.s, Sl}, 0, g.s,
             row_tile * TB, tt * TB);
  }
}

// Block extraction on the hatted sketches from the least-squares coefficients:
// X_side = (C_R - T^T C_S) G_T^-1 with C the b x l coefficients of [Y_B ; Z_B] on W, V.
constexpr int ER = 8;
struct CntExtract {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return 2 * cdv(d.r, ER); }
};
template <typename CT>
__global__ void __launch_bounds__(256) k_extract(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntExtract(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  int64_t per = cdv(d.r, ER);
  int side = (int)(loc / per);
  int64_t i0 = (loc % per) * ER;
  const int nr = (int)imin64(ER, d.r - i0);
  const int kp = d.kp, r = d.r, l = d.l, b = d.b;
  const int32_t* perm = g.iwork + d.pv_off;  // [S (pivot order) | R ascending]
  CT* wc = reinterpret_cast<CT*>(g.workc);
  const CT* C = wc + d.x_off + (int64_t)side * b * l;
  const double* T = g.fd + fd_T(d);
  CT* E = wc + d.e_off + (int64_t)side * r * l;
  __shared__ CT tcol[ER][128];  // columns i of T for this CTA's rows (kp <= 128)
  for (int e = threadIdx.x; e < nr * kp; e += blockDim.x) {
    int ii = e / kp, q = e % kp;
    tcol[ii][q] = (CT)T[(int64_t)q * r + i0 + ii];
  }
  __syncthreads();
  // phase 1: Q = C_R - T^T C_S
  for (int64_t e = threadIdx.x; e < (int64_t)nr * l; e += blockDim.x) {
    int ii = (int)(e / l);
    int64_t col = e % l;
    int i = (int)i0 + ii;
    CT v = C[(int64_t)perm[kp + i] * l + col];
    for (int q = 0; q < kp; ++q) v -= tcol[ii][q] * C[(int64_t)perm[q] * l + col];
    E[(int64_t)i * l + col] = v;
  }
  __syncthreads();
  // phase 2: columns R -= columns S times T
  for (int64_t e = threadIdx.x; e < (int64_t)nr * r; e += blockDim.x) {
    int i = (int)i0 + (int)(e / r), u = (int)(e % r);
    CT v = E[(int64_t)i * l + perm[kp + u]];
    for (int q = 0; q < kp; ++q) v -= E[(int64_t)i * l + perm[q]] * (CT)T[(int64_t)q * r + u];
    E[(int64_t)i * l + perm[kp + u]] = v;
  }
  __syncthreads();
  // phase 3: scatter into the factor blocks
  const int64_t w = (int64_t)kp + d.n;
  if (side == 0) {
    double* XRR = g.fd + fd_XRR(d);
    double* Uc = g.fd + fd_Uc(d);  // [X_RS X_RN] until the LU solve
    for (int64_t e = threadIdx.x; e < (int64_t)nr * r; e += blockDim.x) {
      int i = (int)i0 + (int)(e / r), u = (int)(e % r);
      XRR[(int64_t)i * r + u] = (double)E[(int64_t)i * l + perm[kp + u]];
    }
    for (int64_t e = threadIdx.x; e < (int64_t)nr * w; e += blockDim.x) {
      int i = (int)i0 + (int)(e / w);
      int64_t q = e % w;
      int64_t col = q < kp ? perm[q] : b + (q - kp);
      Uc[(int64_t)i * w + q] = (double)E[(int64_t)i * l + col];
    }
  } else {
    double* LcT = g.fd + fd_LcT(d);  // [X_SR^T X_NR^T] until the LU solve
    for (int64_t e = threadIdx.x; e < (int64_t)nr * w; e += blockDim.x) {
      int i = (int)i0 + (int)(e / w);
      int64_t q = e % w;
      int64_t col = q < kp ? perm[q] : b + (q - kp);
      LcT[(int64_t)i * w + q] = (double)E[(int64_t)i * l + col];
    }
  }
}

// LU with partial pivoting of X_RR (copied to the LU block), one CTA per box.
__device__ void lu_inplace(double* A, int64_t n, int64_t lda, int32_t* piv, int* err) {
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t j = 0; j < n; ++j) {
    double bv = -1.0;
    int bp = -1;
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) {
      double v = fabs(A[i * lda + j]);
      if (v > bv) {  // ascending i per thread: ties keep the lower row
        bv = v;
        bp = (int)i;
      }
    }
    for (int o = 16; o; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (op >= 0 && (ov > bv || (ov == bv && (bp < 0 || op < bp)))) {
        bv = ov;
        bp = op;
      }
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v0 = -1.0;
      int p0 = (int)j;
      for (int w = 0; w < nw; ++w)
        if (red_i[w] >= 0 && (red_v[w] > v0 || (red_v[w] == v0 && red_i[w] < p0))) {
          v0 = red_v[w];
          p0 = red_i[w];
        }
      if (!(v0 > 0.0)) set_err(err, kDevSingular);
      else if (!isfinite(v0)) set_err(err, kDevNonfinite);
      s_p = p0;
      piv[j] = p0;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j)
      for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
        double t = A[j * lda + c];
        A[j * lda + c] = A[(int64_t)p * lda + c];
        A[(int64_t)p * lda + c] = t;
      }
    __syncthreads();
    double dj = A[j * lda + j];
    if (dj == 0.0) dj = 1.0;
    for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * lda + j] /= dj;
    __syncthreads();
    const int64_t rem = n - j - 1;
    for (int64_t e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int64_t i = j + 1 + e / rem, c = j + 1 + e % rem;
      A[i * lda + c] -= A[i * lda + j] * A[j * lda + c];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(512) k_lu(GroupArgs g) {
  const BoxDesc d = g.desc[blockIdx.x];
  const double* X = g.fd + fd_XRR(d);
  double* LU = g.fd + fd_LU(d);
  for (int64_t e = threadIdx.x; e < (int64_t)d.r * d.r; e += blockDim.x) LU[e] = X[e];
  __syncthreads();
  lu_inplace(LU, d.r, d.r, g.fi + fi_piv(d), g.err);
}

// Solve X_RR Uc = [X_RS X_RN] and X_RR^T LcT = [X_SR^T X_NR^T] (one thread per column).
constexpr int CW = 128;
struct CntLuRhs {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    return 2 * cdv(d.kp + d.n, CW) + cdv(d.r, CW);
  }
};
__device__ void lu_solve_col(const double* LU, const int32_t* piv, int64_t n, double* x, int64_t stride,
                             bool trans) {
  if (!trans) {
    for (int64_t j = 0; j < n; ++j) {
      int p = piv[j];
      if (p != j) {
        double t = x[j * stride];
        x[j * stride] = x[(int64_t)p * stride];
        x[(int64_t)p * stride] = t;
      }
    }
    for (int64_t i = 1; i < n; ++i) {
      double v = x[i * stride];
      for (int64_t q = 0; q < i; ++q) v -= LU[i * n + q] * x[q * stride];
      x[i * stride] = v;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double v = x[i * stride];
      for (int64_t q = i + 1; q < n; ++q) v -= LU[i * n + q] * x[q * stride];
      x[i * stride] = v / LU[i * n + i];
    }
  } else {
    for (int64_t i = 0; i < n; ++i) {  // U^T y = b
      double v = x[i * stride];
      for (int64_t q = 0; q < i; ++q) v -= LU[q * n + i] * x[q * stride];
      x[i * stride] = v / LU[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {  // L^T z = y
      double v = x[i * stride];
      for (int64_t q = i + 1; q < n; ++q) v -= LU[q * n + i] * x[q * stride];
      x[i * stride] = v;
    }
    for (int64_t j = n - 1; j >= 0; --j) {
      int p = piv[j];
      if (p != j) {
        double t = x[j * stride];
        x[j * stride] = x[(int64_t)p * stride];
        x[(int64_t)p * stride] = t;
      }
    }
  }
}
__global__ void __launch_bounds__(CW) k_lu_rhs(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntLuRhs(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t w = (int64_t)d.kp + d.n;
  int64_t per = cdv(w, CW);
  const double* LU = g.fd + fd_LU(d);
  const int32_t* piv = g.fi + fi_piv(d);
  if (loc >= 2 * per) {  // columns of X_RR^-1: solve against the identity
    int64_t col = (loc - 2 * per) * CW + threadIdx.x;
    if (col >= d.r) return;
    double* B = g.fd + fd_Xinv(d);
    for (int64_t i = 0; i < d.r; ++i) B[i * d.r + col] = (i == col) ? 1.0 : 0.0;
    lu_solve_col(LU, piv, d.r, B + col, d.r, false);
    return;
  }
  int side = (int)(loc / per);
  int64_t col = (loc % per) * CW + threadIdx.x;
  if (col >= w) return;
  double* B = g.fd + (side == 0 ? fd_Uc(d) : fd_LcT(d));
  lu_solve_col(LU, piv, d.r, B + col, w, side == 1);
}

// Mixed path: only X_RR^-1 by substitution (one thread per column); Uc and Lc^T then come from
// tensor-core products with it (k_tc_grouped<LcUcJob>), staged by k_lcuc_prep and written back to the
// factor by k_lcuc_store.
struct CntLuInv {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return cdv(d.r, CW); }
};
__global__ void __launch_bounds__(CW) k_lu_inv(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntLuInv(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t col = loc * CW + threadIdx.x;
  if (col >= d.r) return;
  double* B = g.fd + fd_Xinv(d);
  for (int64_t i = 0; i < d.r; ++i) B[i * d.r + col] = (i == col) ? 1.0 : 0.0;
  lu_solve_col(g.fd + fd_LU(d), g.fi + fi_piv(d), d.r, B + col, d.r, false);
}

// Mixed path: X_RR^-1 by in-place Gauss-Jordan elimination with partial pivoting (ties to the lower
// row) in FP32 shared memory, one CTA of 1024 threads per box (r <= GJ_MAX_R).  Per step k: the
// pivot row p (largest |A_ik|, i >= k), the multipliers of column k, then row k <- row p / pivot with
// A_kk replaced by 1 before the division, row p <- old row k, and every other row minus its
// multiplier times row k with its column-k entry replaced by 0.  The row interchanges become column
// interchanges of the result, applied in reverse step order.  Writes X_RR^-1 to the factor (FP64
// copy of the FP32 values) and X_RR^-1, X_RR^-T (FP32) to the head of the box's near-field test-row
// area for the products that make Uc and Lc^T.  A zero or non-finite pivot records kDevSingular or
// kDevNonfinite (and continues with 1).  The result carries FP32 rounding times cond(X_RR), the
// accuracy of the FP32 products and sweeps that use it.
constexpr int GJ_MAX_R = kGaussJordanMaxR;
__host__ __device__ inline size_t gj_smem_bytes(int r) { return ((size_t)r * r + (size_t)3 * r) * 4; }
__global__ void __launch_bounds__(1024, 1) k_gj_inv32(GroupArgs g) {
  const BoxDesc d = g.desc[blockIdx.x];
  const int r = d.r;
  if (r <= 0) return;
  extern __shared__ __align__(16) unsigned char gj_raw[];
  float* A = reinterpret_cast<float*>(gj_raw);  // r x r, row-major
  float* col = A + (size_t)r * r;                // multipliers of the step's column
  int* ipiv = reinterpret_cast<int*>(col + r);   // pivot row of each step
  int* idx = ipiv + r;                           // column order of the result
  __shared__ int s_p;
  __shared__ float s_inv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  const double* X = g.fd + fd_XRR(d);
  for (int e = tid; e < r * r; e += nt) A[e] = (float)X[e];
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (warp == 0) {  // pivot search in column k, rows k..r-1
      float bv = -1.f;
      int bp = -1;
      for (int i = k + lane; i < r; i += 32) {
        const float v = fabsf(A[(size_t)i * r + k]);
        if (v > bv) {  // ascending i per lane: ties keep the lower row
          bv = v;
          bp = i;
        }
      }
      for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (op >= 0 && (ov > bv || (ov == bv && (bp < 0 || op < bp)))) {
          bv = ov;
          bp = op;
        }
      }
      if (lane == 0) {
        int p = bp < 0 ? k : bp;
        float pv = A[(size_t)p * r + k];
        if (!(bv > 0.f)) set_err(g.err, kDevSingular);
        else if (!isfinite(bv)) set_err(g.err, kDevNonfinite);
        if (!(bv > 0.f) || !isfinite(bv)) pv = 1.f;
        s_p = p;
        s_inv = 1.f / pv;
        ipiv[k] = p;
      }
    }
    __syncthreads();
    const int p = s_p;
    const float inv = s_inv;
    // multipliers of column k after the interchange (old row k moves to p); none for row k
    for (int i = tid; i < r; i += nt) col[i] = (i == k) ? 0.f : (i == p ? A[(size_t)k * r + k] : A[(size_t)i * r + k]);
    __syncthreads();
    for (int j = tid; j < r; j += nt) {
      const float vk = A[(size_t)k * r + j], vp = A[(size_t)p * r + j];
      A[(size_t)p * r + j] = vk;                     // (a no-op when p == k, overwritten just below)
      A[(size_t)k * r + j] = (j == k ? 1.f : vp) * inv;
    }
    __syncthreads();
    for (int i = warp; i < r; i += nt >> 5) {  // a warp per row, lanes along it
      if (i == k) continue;
      const float m = col[i];
      float* Ai = A + (size_t)i * r;
      for (int j = lane; j < r; j += 32) Ai[j] = fmaf(-m, A[(size_t)k * r + j], j == k ? 0.f : Ai[j]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int j = 0; j < r; ++j) idx[j] = j;
    for (int k = r - 1; k >= 0; --k) {
      const int q = ipiv[k];
      const int t = idx[k];
      idx[k] = idx[q];
      idx[q] = t;
    }
  }
  __syncthreads();
  double* Xi = g.fd + fd_Xinv(d);
  float* P = reinterpret_cast<float*>(g.workc) + d.w_off;
  const size_t rr = (size_t)r * r;
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e - i * r;
    const float v = A[(size_t)i * r + idx[j]];
    Xi[e] = (double)v;
    P[e] = v;
    P[rr + (size_t)j * r + i] = v;
  }
}

// FP32 operands of the products Uc = X_RR^-1 [X_RS X_RN] and Lc^T = X_RR^-T [X_SR^T X_NR^T], in the
// box's near-field test-row area (free once the projections are done): [X_RR^-1 | X_RR^-T | the
// right-hand blocks of Uc | of Lc^T], r x r, r x r, r x w, r x w (w = k' + n).
struct CntLcUcPrep {
  int with_inv;  // also stage X_RR^-1 (not when k_gj_inv32 has staged it)
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    const int64_t w = (int64_t)d.kp + d.n;
    return cdv((with_inv ? (int64_t)d.r * d.r : 0) + 2 * (int64_t)d.r * w, 256);
  }
};
__global__ void __launch_bounds__(256) k_lcuc_prep(GroupArgs g, int with_inv) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntLcUcPrep{with_inv}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t r = d.r, w = (int64_t)d.kp + d.n, rr = r * r, rw = r * w;
  const int64_t e = loc * 256 + threadIdx.x + (with_inv ? 0 : rr);
  float* P = reinterpret_cast<float*>(g.workc) + d.w_off;
  if (e < rr) {
    const float v = (float)g.fd[fd_Xinv(d) + e];
    P[e] = v;
    P[rr + (e % r) * r + e / r] = v;
  } else if (e < rr + rw) {
    P[2 * rr + (e - rr)] = (float)g.fd[fd_Uc(d) + (e - rr)];
  } else if (e < rr + 2 * rw) {
    P[2 * rr + rw + (e - rr - rw)] = (float)g.fd[fd_LcT(d) + (e - rr - rw)];
  }
}

// The products' FP32 results (Lc^T then Uc in the extraction area, the Schur update's operands)
// back into the factor in FP64.
struct CntLcUcStore {
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    return cdv(2 * (int64_t)d.r * ((int64_t)d.kp + d.n), 256);
  }
};
__global__ void __launch_bounds__(256) k_lcuc_store(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntLcUcStore(), loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t e = loc * 256 + threadIdx.x;
  if (e >= 2 * (int64_t)d.r * ((int64_t)d.kp + d.n)) return;
  g.fd[fd_LcT(d) + e] = (double)reinterpret_cast<const float*>(g.workc)[d.e_off + e];
}

// Block elimination on the sketches: Y_SN -= Lc Y_R, Om_R += Uc Om_SN, Z_SN -= Uc^T Z_R,
// Ps_R += Lc^T Ps_SN, with Lc = LcT^T stored r x (kp+n).
struct CntSchur {
  int64_t s;
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    return (2 * cdv(d.kp + d.n, TB) + 2 * cdv(d.r, TB)) * cdv(s, TB);
  }
};
template <typename CT>
__global__ void __launch_bounds__(NT) k_schur(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntSchur{g.s}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t nt = cdv(g.s, TB);
  const int64_t w = (int64_t)d.kp + d.n;
  const int64_t tw = cdv(w, TB), tr = cdv(d.r, TB);
  int64_t row_tile = loc / nt, tt = loc % nt;
  const int32_t* Rl = g.fi + fi_R(d);
  const int32_t* SN = g.fi + fi_S(d);
  const double* LcT = g.fd + fd_LcT(d);
  const double* Uc = g.fd + fd_Uc(d);
  if (row_tile < tw) {
    tile_acc<CT>(-1.0, MatA{LcT, w, true}, w, d.r, Rows{g.Y, g.s, Rl}, 0, RowsW{g.Y, g.s, SN}, 0, g.s,
             row_tile * TB, tt * TB);
  } else if (row_tile < tw + tr) {
    row_tile -= tw;
    tile_acc<CT>(1.0, MatA{Uc, w, false}, d.r, w, Rows{g.Om, g.s, SN}, 0, RowsW{g.Om, g.s, Rl}, 0, g.s,
             row_tile * TB, tt * TB);
  } else if (row_tile < 2 * tw + tr) {
    row_tile -= tw + tr;
    tile_acc<CT>(-1.0, MatA{Uc, w, true}, w, d.r, Rows{g.Z, g.s, Rl}, 0, RowsW{g.Z, g.s, SN}, 0, g.s,
             row_tile * TB, tt * TB);
  } else {
    row_tile -= 2 * tw + tr;
    tile_acc<CT>(1.0, MatA{LcT, w, false}, d.r, w, Rows{g.Ps, g.s, SN}, 0, RowsW{g.Ps, g.s, Rl}, 0, g.s,
             row_tile * TB, tt * TB);
  }
}

// Mixed path: FP32 copies of the Schur products' reused operands, made once per group (FP64 ->
// FP32 conversions run at the FP64 rate on this part, and a tile product converts every operand
// element it loads, i.e. once per tile that reads it): LcT and Uc (r x (k'+n) each) into the box's
// extraction workspace, Y_R and Z_R (r x s each) into its sketch workspace (both free after the
// extraction and the CPQR).
struct CntSchurPrep {
  int64_t s;
  int yz_only;  // Lc^T and Uc are already in the workspace (made there by tensor-core products)
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    return cdv((yz_only ? 0 : 2 * (int64_t)d.r * ((int64_t)d.kp + d.n)) + 2 * (int64_t)d.r * s, 256);
  }
};
__global__ void __launch_bounds__(256) k_schur_prep(GroupArgs g, int yz_only) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntSchurPrep{g.s, yz_only}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t w = (int64_t)d.kp + d.n, rw = (int64_t)d.r * w, rs = (int64_t)d.r * g.s;
  int64_t e = loc * 256 + threadIdx.x;
  float* wc = reinterpret_cast<float*>(g.workc);
  if (!yz_only) {
    if (e < 2 * rw) {
      const double* src = g.fd + (e < rw ? fd_LcT(d) : fd_Uc(d));
      wc[d.e_off + e] = (float)src[e < rw ? e : e - rw];
      return;
    }
    e -= 2 * rw;
  }
  if (e >= 2 * rs) return;
  const int side = (int)(e / rs);
  const int64_t i = (e % rs) / g.s, t = (e % rs) % g.s;
  const int32_t* Rl = g.fi + fi_R(d);
  const double* src = side == 0 ? g.Y : g.Z;
  wc[d.mc_off + e] = from_f64<float>(src[(int64_t)Rl[i] * g.s + t]);
}
__global__ void __launch_bounds__(NT) k_schur32(GroupArgs g) {
  int64_t loc;
  int bi = find_item(g.desc, g.nbox, blockIdx.x, CntSchur{g.s}, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int64_t nt = cdv(g.s, TB);
  const int64_t w = (int64_t)d.kp + d.n;
  const int64_t tw = cdv(w, TB), tr = cdv(d.r, TB);
  int64_t row_tile = loc / nt, tt = loc % nt;
  const int32_t* Rl = g.fi + fi_R(d);
  const int32_t* SN = g.fi + fi_S(d);
  const float* wc = reinterpret_cast<const float*>(g.workc);
  const float* LcT = wc + d.e_off;
  const float* Uc = LcT + (int64_t)d.r * w;
  const float* YR = wc + d.mc_off;
  const float* ZR = YR + (int64_t)d.r * g.s;
  if (row_tile < tw) {
    tile_acc<float>(-1.0, MatAT<float>{LcT, w, true}, w, d.r, RowsT<float>{YR, g.s, nullptr}, 0,
                    RowsW{g.Y, g.s, SN}, 0, g.s, row_tile * TB, tt * TB);
  } else if (row_tile < tw + tr) {
    row_tile -= tw;
    tile_acc<float>(1.0, MatAT<float>{Uc, w, false}, d.r, w, Rows{g.Om, g.s, SN}, 0, RowsW{g.Om, g.s, Rl}, 0, g.s,
                    row_tile * TB, tt * TB);
  } else if (row_tile < 2 * tw + tr) {
    row_tile -= tw + tr;
    tile_acc<float>(-1.0, MatAT<float>{Uc, w, true}, w, d.r, RowsT<float>{ZR, g.s, nullptr}, 0,
                    RowsW{g.Z, g.s, SN}, 0, g.s, row_tile * TB, tt * TB);
  } else {
    row_tile -= 2 * tw + tr;
    tile_acc<float>(1.0, MatAT<float>{LcT, w, false}, d.r, w, Rows{g.Ps, g.s, SN}, 0, RowsW{g.Ps, g.s, Rl}, 0, g.s,
                    row_tile * TB, tt * TB);
  }
}

// Dense LU of the root block (single CTA) and its solve on gathered rows of F.
__global__ void __launch_bounds__(1024) k_dense_lu(double* A, int64_t n, int32_t* piv, int* err) {
  lu_inplace(A, n, n, piv, err);
}
__global__ void k_dense_lu_solve(const double* LU, const int32_t* piv, int64_t n, const int32_t* rows,
                                 double* F, int nrhs, int adjoint) {
  // one CTA per right-hand side; the column is staged in shared memory
  extern __shared__ double col[];
  const int c = blockIdx.x;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) col[i] = F[(int64_t)rows[i] * nrhs + c];
  __syncthreads();
  if (threadIdx.x == 0) lu_solve_col(LU, piv, n, col, 1, adjoint != 0);
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) F[(int64_t)rows[i] * nrhs + c] = col[i];
}

// ---- solve / apply sweeps ------------------------------------------------------
// C rows += alpha * A(i, q) * B rows, nrhs columns of the row-major (tree order) block F.
// Row sets: 0 = R, 1 = S, 2 = SN (S followed by N); matrices: 0 = T, 1 = LcT, 2 = Uc.
struct SweepOp {
  int cset, mat, trans, bset;
  double alpha;
};
__device__ inline void sweep_set(const BoxDesc& d, const int32_t* fi, int set, const int32_t*& idx, int64_t& m) {
  if (set == 0) { idx = fi + fi_R(d); m = d.r; }
  else if (set == 1) { idx = fi + fi_S(d); m = d.kp; }
  else { idx = fi + fi_S(d); m = (int64_t)d.kp + d.n; }
}
// Output rows per CTA of the sweep products: op(A) = A^T (A stored K x m) takes a thread per
// output row, op(A) = A (row-major m x K) a warp per two rows.
constexpr int SW_T_ROWS = 128, SW_N_ROWS = 16;
struct CntSweep {
  int cset, rows;  // output row set, output rows per item
  __host__ __device__ int64_t operator()(const BoxDesc& d) const {
    int64_t m = cset == 0 ? d.r : (cset == 1 ? d.kp : (int64_t)d.kp + d.n);
    return cdv(m, rows);
  }
};
// The factor's blocks and the right-hand sides in the sweep's arithmetic: FP64, or the FP32 copies
// a mixed-precision factor keeps for its solves.
template <typename T>
__device__ inline const T* sweep_fd(const SweepArgs& a);
template <>
__device__ inline const double* sweep_fd<double>(const SweepArgs& a) { return a.fd; }
template <>
__device__ inline const float* sweep_fd<float>(const SweepArgs& a) { return a.fd32; }
template <typename T>
__device__ inline T* sweep_F(const SweepArgs& a);
template <>
__device__ inline double* sweep_F<double>(const SweepArgs& a) { return a.F; }
template <>
__device__ inline float* sweep_F<float>(const SweepArgs& a) { return a.F32; }

// C rows += alpha op(A) B rows for 16 right-hand sides at a time, B staged in shared memory in
// chunks of K.  Transposed form (A stored K x m): thread i of the CTA owns output row i and its 16
// sums; the threads read consecutive elements of each K row of A.
template <typename T>
__device__ inline void sweep_operands(const SweepArgs& a, const SweepOp& op, const BoxDesc& d, const int32_t*& cidx,
                                      int64_t& m, const int32_t*& bidx, int64_t& K, const T*& A, int64_t& lda) {
  sweep_set(d, a.fi, op.cset, cidx, m);
  sweep_set(d, a.fi, op.bset, bidx, K);
  const T* fd = sweep_fd<T>(a);
  if (op.mat == 0) { A = fd + fd_T(d); lda = d.r; }
  else if (op.mat == 1) { A = fd + fd_LcT(d); lda = (int64_t)d.kp + d.n; }
  else { A = fd + fd_Uc(d); lda = (int64_t)d.kp + d.n; }
}
template <typename T, int ROWS>
__device__ void sweep_t_item(const SweepArgs& a, const SweepOp& op, int64_t item, const int2* map = nullptr) {
  int64_t loc;
  int bi;
  if (map) {
    const int2 bl = map[item];
    bi = bl.x;
    loc = bl.y;
  } else {
    bi = find_item(a.desc, a.nbox, item, CntSweep{op.cset, ROWS}, loc);
  }
  if (bi < 0) return;
  const BoxDesc d = a.desc[bi];
  const int32_t *cidx, *bidx;
  int64_t m, K, lda;
  const T* A;
  sweep_operands<T>(a, op, d, cidx, m, bidx, K, A, lda);
  T* F = sweep_F<T>(a);
  constexpr int QC = 64;
  __shared__ __align__(16) T Bs[QC][16];
  const int64_t i = loc * ROWS + threadIdx.x;
  for (int c0 = 0; c0 < a.nrhs; c0 += 16) {
    T acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0;
    for (int64_t q0 = 0; q0 < K; q0 += QC) {
      for (int e = threadIdx.x; e < QC * 16; e += ROWS) {
        const int qq = e >> 4, cc = e & 15;
        const int64_t q = q0 + qq;
        Bs[qq][cc] = (q < K && c0 + cc < a.nrhs) ? F[((int64_t)bidx[q] - a.row_base) * a.nrhs + c0 + cc] : (T)0;
      }
      __syncthreads();
      if (i < m) {
        const int qn = (int)imin64(QC, K - q0);
        const T* Ai = A + q0 * lda + i;
        for (int qq = 0; qq < qn; qq += 16) {  // 16 loads of A in flight, then their products
          T av[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) av[u] = qq + u < qn ? Ai[(int64_t)(qq + u) * lda] : (T)0;
#pragma unroll
          for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = mad(av[u], Bs[qq + u][c], acc[c]);
        }
      }
      __syncthreads();
    }
    if (i < m) {
      T* out = F + ((int64_t)cidx[i] - a.row_base) * a.nrhs + c0;
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c0 + c < a.nrhs) out[c] += (T)op.alpha * acc[c];
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(SW_T_ROWS) k_sweep_t(SweepArgs a, SweepOp op) {
  sweep_t_item<T, SW_T_ROWS>(a, op, blockIdx.x);
}

// Row-major form (A m x K): warp w of the CTA owns output rows 2w and 2w + 1, its lanes stride
// along K (consecutive elements of the A rows) with 16 partial sums per row, then reduce.
template <typename T>
__device__ void sweep_n_item(const SweepArgs& a, const SweepOp& op, int64_t item, const int2* map = nullptr) {
  int64_t loc;
  int bi;
  if (map) {
    const int2 bl = map[item];
    bi = bl.x;
    loc = bl.y;
  } else {
    bi = find_item(a.desc, a.nbox, item, CntSweep{op.cset, SW_N_ROWS}, loc);
  }
  if (bi < 0) return;
  const BoxDesc d = a.desc[bi];
  const int32_t *cidx, *bidx;
  int64_t m, K, lda;
  const T* A;
  sweep_operands<T>(a, op, d, cidx, m, bidx, K, A, lda);
  T* F = sweep_F<T>(a);
  constexpr int QC = 128;
  __shared__ T Bs[QC][17];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i0 = loc * SW_N_ROWS + 2 * warp;
  for (int c0 = 0; c0 < a.nrhs; c0 += 16) {
    T acc[2][16];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int c = 0; c < 16; ++c) acc[u][c] = 0;
    for (int64_t q0 = 0; q0 < K; q0 += QC) {
      for (int e = threadIdx.x; e < QC * 16; e += 256) {
        const int qq = e >> 4, cc = e & 15;
        const int64_t q = q0 + qq;
        Bs[qq][cc] = (q < K && c0 + cc < a.nrhs) ? F[((int64_t)bidx[q] - a.row_base) * a.nrhs + c0 + cc] : (T)0;
      }
      __syncthreads();
      const int qn = (int)imin64(QC, K - q0);
      T av[2][QC / 32];  // the chunk's A values of both rows, all loads in flight together
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int t = 0; t < QC / 32; ++t) {
          const int qq = lane + 32 * t;
          av[u][t] = (i0 + u < m && qq < qn) ? A[(i0 + u) * lda + q0 + qq] : (T)0;
        }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int t = 0; t < QC / 32; ++t) {
          const int qq = lane + 32 * t;
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[u][c] = mad(av[u][t], Bs[qq][c], acc[u][c]);
        }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
#pragma unroll
      for (int c = 0; c < 16; ++c)
#pragma unroll
        for (int o = 16; o; o >>= 1) acc[u][c] += __shfl_xor_sync(0xffffffffu, acc[u][c], o);
      T v = acc[u][0];
#pragma unroll
      for (int c = 1; c < 16; ++c)
        if (lane == c) v = acc[u][c];
      if (i0 + u < m && lane < 16 && c0 + lane < a.nrhs)
        F[((int64_t)cidx[i0 + u] - a.row_base) * a.nrhs + c0 + lane] += (T)op.alpha * v;
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_n(SweepArgs a, SweepOp op) {
  sweep_n_item<T>(a, op, blockIdx.x);
}

// f_R <- M f_R with M = X_RR^-1 (solve) or X_RR (apply), or M^T for the adjoint; one CTA per
// (box, group of DC columns): the rows R of F are staged in shared memory.
constexpr int DC = 4;
struct CntDiag {
  int nrhs;
  __host__ __device__ int64_t operator()(const BoxDesc& d) const { return cdv(nrhs, DC); }
};
template <typename T>
__device__ void sweep_diag_item(const SweepArgs& a, int solve, int64_t item, unsigned char* dsm_raw,
                                bool by_division = false) {
  int64_t loc;
  int bi;
  if (by_division) {  // every box has cdv(nrhs, DC) items
    const int64_t per = cdv(a.nrhs, DC);
    bi = (int)(item / per);
    loc = item % per;
  } else {
    bi = find_item(a.desc, a.nbox, item, CntDiag{a.nrhs}, loc);
  }
  if (bi < 0) return;
  const BoxDesc d = a.desc[bi];
  const int c0 = (int)loc * DC;
  const int nc = min(DC, a.nrhs - c0);
  const int64_t r = d.r;
  const int32_t* R = a.fi + fi_R(d);
  const T* M = sweep_fd<T>(a) + (solve ? fd_Xinv(d) : fd_XRR(d));
  T* F = sweep_F<T>(a);
  T* in = reinterpret_cast<T*>(dsm_raw);  // r x DC
  for (int64_t e = threadIdx.x; e < r * DC; e += blockDim.x) {
    int64_t i = e / DC;
    int c = (int)(e % DC);
    in[e] = (c < nc) ? F[((int64_t)R[i] - a.row_base) * a.nrhs + c0 + c] : (T)0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T out[DC];
  if (!a.adjoint) {  // warp per row, lanes along the row (coalesced)
    for (int64_t i = warp; i < r; i += nw) {
#pragma unroll
      for (int c = 0; c < DC; ++c) out[c] = 0;
      for (int64_t q = lane; q < r; q += 32) {
        T m = M[i * r + q];
#pragma unroll
        for (int c = 0; c < DC; ++c) out[c] = mad(m, in[q * DC + c], out[c]);
      }
#pragma unroll
      for (int c = 0; c < DC; ++c)
        for (int o = 16; o; o >>= 1) out[c] += __shfl_xor_sync(0xffffffffu, out[c], o);
      if (lane < nc) {
        T v = out[0];
#pragma unroll
        for (int c = 1; c < DC; ++c)
          if (lane == c) v = out[c];
        F[((int64_t)R[i] - a.row_base) * a.nrhs + c0 + lane] = v;
      }
    }
  } else {  // thread per row, reading column i of M (coalesced across threads)
    for (int64_t i = threadIdx.x; i < r; i += blockDim.x) {
#pragma unroll
      for (int c = 0; c < DC; ++c) out[c] = 0;
      for (int64_t q = 0; q < r; ++q) {
        T m = M[q * r + i];
#pragma unroll
        for (int c = 0; c < DC; ++c) out[c] = mad(m, in[q * DC + c], out[c]);
      }
      for (int c = 0; c < nc; ++c) F[((int64_t)R[i] - a.row_base) * a.nrhs + c0 + c] = out[c];
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_diag(SweepArgs a, int solve) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  sweep_diag_item<T>(a, solve, blockIdx.x, dsm_raw);
}

// ---- fused solve sweeps -----------------------------------------------------------------------
// Barrier of all CTAs of a cooperative launch (all resident at once), in global memory: bar[0]
// counts arrivals, bar[1] is the generation.  Thread 0 of each CTA makes its arrival without
// waiting for the atomic's result; CTA 0 waits until every CTA has arrived, resets the count and
// opens the next generation, which the other CTAs wait for.  Every wait gives up after max_polls
// polls: it records kDevTimeout in bar[2] and returns false, and the CTA leaves the kernel (the
// others then give up too).
constexpr long long kGridPolls = 1ll << 25;
__device__ bool grid_sync(unsigned* bar, long long max_polls = kGridPolls) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vcnt = bar;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    atomicAdd(bar, 1u);  // result unused: a reduction, no round trip
    int ok = 1;
    long long polls = 0;
    if (blockIdx.x == 0) {
      while (*vcnt < gridDim.x) {
        if (++polls > max_polls) {
          ok = 0;
          break;
        }
        if (polls > 256) __nanosleep(32);
      }
      if (ok) {
        *vcnt = 0u;
        __threadfence();
        atomicAdd(bar + 1, 1u);
      }
    } else {
      while (*vgen == gen) {
        if (++polls > max_polls) {
          ok = 0;
          break;
        }
        if (polls > 256) __nanosleep(32);
      }
    }
    if (!ok) atomicCAS(reinterpret_cast<int*>(bar + 2), 0, (int)kDevTimeout);
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}
template <typename T>
__global__ void __launch_bounds__(kSweepFusedThreads) k_sweep_fused(SweepArgs a, const SweepPhase* ph, int nph,
                                                                   unsigned* bar) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  for (int p = 0; p < nph; ++p) {
    const SweepPhase P = ph[p];
    SweepArgs b = a;
    b.desc = P.desc;
    b.nbox = P.nbox;
    const SweepOp op{P.cset, P.mat, P.kind == 0 ? 1 : 0, P.bset, P.alpha};
    const int64_t items = P.kind == 2 ? (int64_t)P.nbox * ((a.nrhs + DC - 1) / DC) : P.items;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      if (P.kind == 0) sweep_t_item<T, kSweepFusedRowsT>(b, op, it, P.map);
      else if (P.kind == 1) sweep_n_item<T>(b, op, it, P.map);
      else sweep_diag_item<T>(b, P.solve, it, dsm_raw, true);
      __syncthreads();  // shared memory is reused by the next item
    }
    if (P.sync && p + 1 < nph && !grid_sync(bar)) return;
  }
}

// Column of the inverse of an LU-factored matrix, staged in shared memory, solved cooperatively:
// each substitution step updates the remaining entries in parallel.
__global__ void __launch_bounds__(256) k_dense_inverse(const double* LU, const int32_t* piv, int64_t n,
                                                       double* inv) {
  extern __shared__ double x[];
  const int64_t col = blockIdx.x;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = (i == col) ? 1.0 : 0.0;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int64_t j = 0; j < n; ++j) {
      int p = piv[j];
      if (p != j) {
        double t = x[j];
        x[j] = x[p];
        x[p] = t;
      }
    }
  __syncthreads();
  for (int64_t j = 0; j < n; ++j) {  // unit lower
    double xj = x[j];
    for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) x[i] -= LU[i * n + j] * xj;
    __syncthreads();
  }
  for (int64_t j = n - 1; j >= 0; --j) {  // upper
    if (threadIdx.x == 0) x[j] /= LU[j * n + j];
    __syncthreads();
    double xj = x[j];
    for (int64_t i = threadIdx.x; i < j; i += blockDim.x) x[i] -= LU[i * n + j] * xj;
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) inv[i * n + col] = x[i];
}
// Dense root block times rows of F: F[rows] <- A F[rows] (or A^T), one CTA per column.
template <typename T>
__global__ void k_dense_apply(const T* A, int64_t n, const int32_t* rows, int64_t row_base, T* F, int nrhs,
                              int adjoint) {
  extern __shared__ __align__(16) unsigned char col_raw[];
  T* col = reinterpret_cast<T*>(col_raw);
  T* out = col + n;
  const int c = blockIdx.x;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) col[i] = F[((int64_t)rows[i] - row_base) * nrhs + c];
  __syncthreads();
  if (adjoint) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      T v = 0;
      for (int64_t q = 0; q < n; ++q) v = mad(A[q * n + i], col[q], v);
      out[i] = v;
    }
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t i = warp; i < n; i += nw) {
      T v = 0;
      for (int64_t q = lane; q < n; q += 32) v = mad(A[i * n + q], col[q], v);
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) out[i] = v;
    }
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) F[((int64_t)rows[i] - row_base) * nrhs + c] = out[i];
}

// FP32 -> FP64, elementwise.
__global__ void k_f32_to_f64(const float* __restrict__ in, int64_t count, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = (double)in[e];
}

template <class K, class Cnt>
int64_t items_of(const std::vector<BoxDesc>& h, Cnt cnt) {
  int64_t t = 0;
  for (const auto& d : h) t += cnt(d);
  return t;
}

}  // namespace

// ---- host wrappers -------------------------------------------------------------
static inline void count_launch(Launch L) {
  if (L.counter) ++*L.counter;
}
static inline unsigned grid1(int64_t items) { return (unsigned)items; }

void launch_copy_segments(Launch L, const Seg* segs, int nseg, const int32_t* src, int32_t* dst) {
  if (nseg <= 0) return;
  k_copy_segments<<<nseg, 128, 0, L.st>>>(segs, nseg, src, dst);
  count_launch(L);
}
void launch_gather_rows(Launch L, const double* in, int64_t ld_in, const int32_t* rows, int64_t m,
                        int64_t ncols, double* out, int64_t ld_out) {
  if (m <= 0) return;
  k_gather_rows<<<(unsigned)m, 256, 0, L.st>>>(in, ld_in, rows, m, ncols, out, ld_out);
  count_launch(L);
}
void launch_gram(Launch L, const GroupArgs& g, int64_t items) {
  if (items <= 0) return;
  if (g.fp32) k_gram<float><<<grid1(items), NT, 0, L.st>>>(g);
  else k_gram<double><<<grid1(items), NT, 0, L.st>>>(g);
  count_launch(L);
}
void launch_chol_panel(Launch L, const GroupArgs& g, int panel) {
  // items = number of (box, side) with l > panel*64; the caller passes it through nbox scan
  if (g.fp32) k_chol_panel<float><<<(unsigned)(2 * g.nbox), NT, 0, L.st>>>(g, panel);
  else k_chol_panel<double><<<(unsigned)(2 * g.nbox), NT, 0, L.st>>>(g, panel);
  count_launch(L);
}
void launch_chol_trsm(Launch L, const GroupArgs& g, int panel, int64_t items) {
  if (items <= 0) return;
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(k_chol_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * TB * (TB + 1) * sizeof(double)));
    cudaFuncSetAttribute(k_chol_trsm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * TB * (TB + 1) * sizeof(float)));
  });
  if (g.fp32) k_chol_trsm<float><<<grid1(items), NT, 2 * TB * (TB + 1) * sizeof(float), L.st>>>(g, panel);
  else k_chol_trsm<double><<<grid1(items), NT, 2 * TB * (TB + 1) * sizeof(double), L.st>>>(g, panel);
  count_launch(L);
}
void launch_chol_update(Launch L, const GroupArgs& g, int panel, int64_t items) {
  if (items <= 0) return;
  if (g.fp32) k_chol_update<float><<<grid1(items), NT, 0, L.st>>>(g, panel);
  else k_chol_update<double><<<grid1(items), NT, 0, L.st>>>(g, panel);
  count_launch(L);
}
void launch_gather_box(Launch L, const GroupArgs& g, int64_t items) {
  if (g.fp32) k_gather_box<float><<<grid1(items), 256, 0, L.st>>>(g);
  else k_gather_box<double><<<grid1(items), 256, 0, L.st>>>(g);
  count_launch(L);
}
void launch_m_finalize(Launch L, const GroupArgs& g, int64_t items) {
  if (items <= 0) return;
  if (g.fp32) k_m_finalize<float><<<grid1(items), 256, 0, L.st>>>(g);
  else k_m_finalize<double><<<grid1(items), 256, 0, L.st>>>(g);
  count_launch(L);
}
void launch_proj_nt(Launch L, const GroupArgs& g, int pass, int64_t items) {
  if (g.fp32) k_proj_nt<float><<<grid1(items), NT, 0, L.st>>>(g, pass);
  else k_proj_nt<double><<<grid1(items), NT, 0, L.st>>>(g, pass);
  count_launch(L);
}
void launch_proj_solve(Launch L, const GroupArgs& g, int pass, int64_t items) {
  if (g.fp32) k_proj_solve<float><<<grid1(items), NT, 0, L.st>>>(g, pass);
  else k_proj_solve<double><<<grid1(items), NT, 0, L.st>>>(g, pass);
  count_launch(L);
}
void launch_proj_acc(Launch L, const GroupArgs& g, int pass, int64_t items) {
  if (g.fp32) k_proj_acc<float><<<grid1(items), NT, 0, L.st>>>(g, pass);
  else k_proj_acc<double><<<grid1(items), NT, 0, L.st>>>(g, pass);
  count_launch(L);
}
void launch_cpqr(Launch L, const GroupArgs& g, int max_b) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(g.nbox * CPQR_C));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = (size_t)max_b * (3 * sizeof(double) + sizeof(int));
  cfg.stream = L.st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CPQR_C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_cpqr_cluster, g);
  count_launch(L);
}
// Shared memory of k_cpqr32_cluster for boxes of up to max_b rows, C CTAs and slices of cs columns.
static size_t cpqr32_smem(int max_b, int cs, int C) {
  return cpqr32_head_bytes(max_b, C) + (size_t)max_b * cs * sizeof(float);
}
constexpr size_t kCpqr32MaxSmem = 220 * 1024;
bool launch_cpqr32(Launch L, const GroupArgs& g, int max_b, int cluster, int threads) {
  const int64_t c = 2 * g.s;
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(k_cpqr32_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_cpqr32_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCpqr32MaxSmem);
  });
  auto slice = [c](int q) { return (int)((cdiv(c, q) + 3) / 4 * 4); };
  // smallest cluster whose shared memory holds the slices; otherwise 16 CTAs on slices in place
  int C = 16, in_global = 1;
  for (int q = 1; q <= 16; q *= 2)
    if (cpqr32_smem(max_b, slice(q), q) <= kCpqr32MaxSmem) {
      C = q;
      in_global = 0;
      break;
    }
  if (!in_global && cluster > C && cluster <= 16 && (cluster & (cluster - 1)) == 0 &&
      cpqr32_smem(max_b, slice(cluster), cluster) <= kCpqr32MaxSmem)
    C = cluster;
  const int cs = slice(C);
  const size_t smem = in_global ? cpqr32_smem(max_b, 0, C) : cpqr32_smem(max_b, cs, C);
  if (smem > kCpqr32MaxSmem) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(g.nbox * C));
  // one CTA per SM: many warps hide the shared-memory latency of each step
  cfg.blockDim = dim3((threads == 256 || threads == 512) ? (unsigned)threads : 1024u);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = L.st;
  cudaLaunchAttribute attr1[1];
  attr1[0].id = cudaLaunchAttributeClusterDimension;
  attr1[0].val.clusterDim.x = C;
  attr1[0].val.clusterDim.y = 1;
  attr1[0].val.clusterDim.z = 1;
  cfg.attrs = attr1;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_cpqr32_cluster, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchKernelEx(&cfg, k_cpqr32_cluster, g, cs, in_global);
  count_launch(L);
  return true;
}
void launch_cpqr_single(Launch L, const GroupArgs& g, int max_b) {
  size_t smem = (size_t)max_b * (sizeof(double) + sizeof(int));
  k_cpqr<<<(unsigned)g.nbox, 512, smem, L.st>>>(g);
  count_launch(L);
}
void launch_id_finish(Launch L, const GroupArgs& g, int max_b) {
  size_t smem = (size_t)(2 * max_b + max_b) * sizeof(int);
  k_id_finish<<<(unsigned)g.nbox, 256, smem, L.st>>>(g);
  count_launch(L);
}
void launch_ef_update(Launch L, const GroupArgs& g, int64_t items) {
  if (items <= 0) return;
  if (g.fp32) k_ef_update<float><<<grid1(items), NT, 0, L.st>>>(g);
  else k_ef_update<double><<<grid1(items), NT, 0, L.st>>>(g);
  count_launch(L);
}
void launch_extract(Launch L, const GroupArgs& g, int64_t items) {
  if (items <= 0) return;
  if (g.fp32) k_extract<float><<<grid1(items), 256, 0, L.st>>>(g);
  else k_extract<double><<<grid1(items), 256, 0, L.st>>>(g);
  count_launch(L);
}
void launch_lu(Launch L, const GroupArgs& g) {
  k_lu<<<(unsigned)g.nbox, 512, 0, L.st>>>(g);
  count_launch(L);
}
void launch_lu_rhs(Launch L, const GroupArgs& g, int64_t items) {
  if (items <= 0) return;
  k_lu_rhs<<<grid1(items), CW, 0, L.st>>>(g);
  count_launch(L);
}
void launch_lu_inv(Launch L, const GroupArgs& g, int64_t items) {
  if (items <= 0) return;
  k_lu_inv<<<grid1(items), CW, 0, L.st>>>(g);
  count_launch(L);
}
void launch_lcuc_prep(Launch L, const GroupArgs& g, int64_t items, int with_inv) {
  if (items <= 0) return;
  k_lcuc_prep<<<grid1(items), 256, 0, L.st>>>(g, with_inv);
  count_launch(L);
}
bool launch_gj_inv32(Launch L, const GroupArgs& g, int max_r) {
  if (max_r > GJ_MAX_R) return false;
  if (max_r <= 0 || g.nbox <= 0) return true;
  const size_t smem = gj_smem_bytes(max_r);
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(k_gj_inv32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gj_smem_bytes(GJ_MAX_R));
  });
  k_gj_inv32<<<(unsigned)g.nbox, 1024, smem, L.st>>>(g);
  count_launch(L);
  return true;
}
void launch_lcuc_store(Launch L, const GroupArgs& g, int64_t items) {
  if (items <= 0) return;
  k_lcuc_store<<<grid1(items), 256, 0, L.st>>>(g);
  count_launch(L);
}
void launch_schur(Launch L, const GroupArgs& g, int64_t items, int64_t prep_items, int yz_only,
                  const std::vector<BoxDesc>* tc) {
  if (items <= 0) return;
  if (g.fp32) {
    if (prep_items > 0) {
      k_schur_prep<<<grid1(prep_items), 256, 0, L.st>>>(g, yz_only);
      count_launch(L);
    }
    if (tc) {
      launch_schur_tc(L, g, *tc);
      return;
    }
    k_schur32<<<grid1(items), NT, 0, L.st>>>(g);
  } else {
    k_schur<double><<<grid1(items), NT, 0, L.st>>>(g);
  }
  count_launch(L);
}
void launch_dense_lu(Launch L, double* A, int64_t n, int32_t* piv, int* err) {
  k_dense_lu<<<1, 1024, 0, L.st>>>(A, n, piv, err);
  count_launch(L);
}
void launch_dense_lu_solve(Launch L, const double* LU, const int32_t* piv, int64_t n, const int32_t* rows,
                           double* F, int nrhs, int adjoint) {
  k_dense_lu_solve<<<nrhs, 256, n * sizeof(double), L.st>>>(LU, piv, n, rows, F, nrhs, adjoint);
  count_launch(L);
}

void launch_sweep_op(Launch L, const SweepArgs& a, int cset, int mat, int trans, int bset, double alpha,
                     const std::vector<BoxDesc>& h) {
  const int64_t items = items_of<void>(h, CntSweep{cset, trans ? SW_T_ROWS : SW_N_ROWS});
  if (items <= 0) return;
  const SweepOp op{cset, mat, trans, bset, alpha};
  if (trans) {
    if (a.F32) k_sweep_t<float><<<grid1(items), SW_T_ROWS, 0, L.st>>>(a, op);
    else k_sweep_t<double><<<grid1(items), SW_T_ROWS, 0, L.st>>>(a, op);
  } else {
    if (a.F32) k_sweep_n<float><<<grid1(items), 256, 0, L.st>>>(a, op);
    else k_sweep_n<double><<<grid1(items), 256, 0, L.st>>>(a, op);
  }
  count_launch(L);
}
// Self-test of the grid barrier's bounded wait: two CTAs of a cooperative launch; CTA 1 takes part
// only when `arrive` is set, so without it CTA 0's wait must expire after `polls` polls and record
// kDevTimeout in bar[2].
__global__ void k_grid_wait_selftest(unsigned* bar, long long polls, int arrive) {
  if (blockIdx.x == 1 && !arrive) return;
  (void)grid_sync(bar, polls);
}
bool launch_grid_wait_selftest(Launch L, unsigned* bar, long long polls, int arrive) {
  void* kargs[] = {&bar, &polls, &arrive};
  if (cudaLaunchCooperativeKernel((const void*)k_grid_wait_selftest, dim3(2), dim3(32), kargs, 0, L.st) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  count_launch(L);
  return true;
}
int64_t sweep_phase_tiles(const BoxDesc& d, int kind, int cset) {
  return CntSweep{cset, kind == 0 ? kSweepFusedRowsT : kSweepFusedRowsN}(d);
}
int64_t sweep_phase_items(const std::vector<BoxDesc>& h, int kind, int cset, int nrhs) {
  if (kind == 2) return items_of<void>(h, CntDiag{nrhs});
  return items_of<void>(h, CntSweep{cset, kind == 0 ? kSweepFusedRowsT : kSweepFusedRowsN});
}
bool launch_sweep_fused(Launch L, const SweepArgs& a, const SweepPhase* ph, int nph, int max_r, unsigned* bar) {
  if (nph <= 0) return true;
  static_assert(kSweepFusedRowsN == SW_N_ROWS, "row-major items of the fused and the separate sweeps agree");
  const size_t es = a.F32 ? sizeof(float) : sizeof(double);
  const size_t smem = (size_t)std::max(max_r, 1) * DC * es;
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  const void* fn = a.F32 ? (const void*)k_sweep_fused<float> : (const void*)k_sweep_fused<double>;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kSweepFusedThreads, smem) != cudaSuccess || per < 1) {
    (void)cudaGetLastError();
    return false;
  }
  const unsigned grid = (unsigned)(std::min(per, 2) * nsm);  // fewer arrivals per barrier
  SweepArgs args = a;
  const SweepPhase* php = ph;
  int n = nph;
  unsigned* b = bar;
  void* kargs[] = {&args, &php, &n, &b};
  if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kSweepFusedThreads), kargs, smem, L.st) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  count_launch(L);
  return true;
}
void launch_sweep_diag(Launch L, const SweepArgs& a, int solve, int64_t items, int max_r) {
  if (items <= 0) return;
  if (a.F32) k_sweep_diag<float><<<grid1(items), 256, (size_t)max_r * DC * sizeof(float), L.st>>>(a, solve);
  else k_sweep_diag<double><<<grid1(items), 256, (size_t)max_r * DC * sizeof(double), L.st>>>(a, solve);
  count_launch(L);
}
void launch_to_f64(Launch L, const float* in, int64_t count, double* out) {
  if (count <= 0) return;
  k_f32_to_f64<<<(unsigned)cdv(count, 256), 256, 0, L.st>>>(in, count, out);
  count_launch(L);
}
void launch_dense_inverse(Launch L, const double* LU, const int32_t* piv, int64_t n, double* inv) {
  if (n <= 0) return;
  const size_t smem = (size_t)n * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_dense_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_dense_inverse<<<(unsigned)n, 256, smem, L.st>>>(LU, piv, n, inv);
  count_launch(L);
}
template <typename T>
void dense_apply_t(Launch L, const T* A, int64_t n, const int32_t* rows, int64_t row_base, T* F, int nrhs,
                   int adjoint) {
  const size_t smem = 2 * (size_t)n * sizeof(T);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_dense_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_dense_apply<T><<<nrhs, 256, smem, L.st>>>(A, n, rows, row_base, F, nrhs, adjoint);
  count_launch(L);
}
void launch_dense_apply(Launch L, const double* A, int64_t n, const int32_t* rows, int64_t row_base, double* F,
                        int nrhs, int adjoint) {
  dense_apply_t(L, A, n, rows, row_base, F, nrhs, adjoint);
}
void launch_dense_apply(Launch L, const float* A, int64_t n, const int32_t* rows, int64_t row_base, float* F,
                        int nrhs, int adjoint) {
  dense_apply_t(L, A, n, rows, row_base, F, nrhs, adjoint);
}

// Item counts for host planning (same functors as the device decoding).
int64_t items_diag(const std::vector<BoxDesc>& h, int nrhs) { return items_of<void>(h, CntDiag{nrhs}); }
int64_t items_lu_inv(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntLuInv()); }
int64_t items_lcuc_prep(const std::vector<BoxDesc>& h, int with_inv) {
  return items_of<void>(h, CntLcUcPrep{with_inv});
}
int64_t items_lcuc_store(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntLcUcStore()); }
int64_t items_gram(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntGram()); }
int64_t items_chol_trsm(const std::vector<BoxDesc>& h, int p) { return items_of<void>(h, CntPanelRows{p}); }
int64_t items_chol_update(const std::vector<BoxDesc>& h, int p) { return items_of<void>(h, CntUpdate{p}); }
int64_t items_gather(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntGather()); }
int64_t items_finalize(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntFinal()); }
int64_t items_proj_nt(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntProjNT()); }
int64_t items_proj_solve(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntProjSolve()); }
int64_t items_proj_acc(const std::vector<BoxDesc>& h, int64_t s) { return items_of<void>(h, CntProjAcc{s}); }
int64_t items_ef(const std::vector<BoxDesc>& h, int64_t s) { return items_of<void>(h, CntEF{s}); }
int64_t items_extract(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntExtract()); }
int64_t items_lu_rhs(const std::vector<BoxDesc>& h) { return items_of<void>(h, CntLuRhs()); }
int64_t items_schur(const std::vector<BoxDesc>& h, int64_t s) { return items_of<void>(h, CntSchur{s}); }
int64_t items_schur_prep(const std::vector<BoxDesc>& h, int64_t s, int yz_only) {
  return items_of<void>(h, CntSchurPrep{s, yz_only});
}

}  // namespace rsrs
