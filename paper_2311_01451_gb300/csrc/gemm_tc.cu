// Grouped 3xTF32 products on the tensor cores for the mixed path's FP32 workspace, for every box
// of a (level, colour) group in one launch: the near-field Grams G = W W^T, their blocked
// Cholesky factors and U = L^-T (with the diagonal-block kernel below), the least-squares
// right-hand sides X = M W^T, the solves X G^-1 = (X U) U^T and the projection updates M -= X W of
// the nullification (Algorithm 1, the null-space projection of the sketches).
//
// One CTA computes a 128 x 128 tile of D = A B^T (A rows and B rows both K-contiguous) or
// D = A B (B stored K x N, N contiguous), with D <- alpha D_acc + beta D on store.  Eight producer
// warps load 32-deep K slices of both operands from global memory, split every FP32 value v into
// hi = v with 13 low mantissa bits cleared and lo = v - hi (Ootomo & Yokota 2022), and write them
// into the 128-byte-swizzled K-major layout the MMA reads (an N-contiguous B is transposed on the
// way); a ninth warp issues D += A_hi B_hi + A_hi B_lo + A_lo B_hi with tcgen05.mma into a 128-column
// TMEM accumulator.  Three stages; per stage an mbarrier for "operands written" (256 arrivals) and
// one for "stage free" (tcgen05.commit).  Every wait is bounded: on expiry the kernel records
// kDevTimeout and completes without hanging.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "tc_common.cuh"

namespace rsrs {
namespace {
using namespace tc;

constexpr int GM = 128, GN = 128, GK = 32;
constexpr int OP_BYTES = GM * GK * 4;  // 16 KB: one hi or lo operand tile
constexpr int GSTAGE = 4 * OP_BYTES;   // A_hi, A_lo, B_hi, B_lo
constexpr int GNST = 3;
constexpr int GSMEM = GNST * GSTAGE + 1024;
constexpr int GPROD = 256, GTHREADS = GPROD + 32;
constexpr uint32_t GTMEM = 128;
static_assert(GM == GN, "both operand tiles have 128 rows");

__host__ __device__ inline int64_t cdiv128(int64_t a) { return (a + 127) / 128; }
__host__ __device__ inline int64_t tri_n(int64_t t) { return t * (t + 1) / 2; }
__device__ inline void tri_idx(int64_t idx, int64_t& ti, int64_t& tj) {
  int64_t t = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
  while (tri_n(t) > idx) --t;
  while (tri_n(t + 1) <= idx) ++t;
  ti = t;
  tj = idx - tri_n(t);
}

struct TcTile {
  const float* A;  // row 0, k 0 of the tile's A rows (row i at A + i * lda)
  int64_t lda;
  int m;           // valid rows
  const float* B;  // bnm = 0: row j at B + j * ldb; bnm = 1: element (k, j) at B + k * ldb + j
  int64_t ldb;
  int n;           // valid columns
  int bnm;
  int64_t K;
  float* D;        // element (i, j) at D + i * ldd + j
  int64_t ldd;
  float alpha, beta;
  float* D2 = nullptr;  // when set, also D2(i, j) += alpha * acc (same ldd)
  // Operand forms of the Schur updates only (jobs with sketch_io<Job>::value):
  int anm = 0;                     // A stored K x M: element (i, k) at A + k * lda + i
  const double* B64 = nullptr;     // bnm = 1, FP64 rows gathered: (k, j) at B64 + bidx[k] * ldb + j
  const int32_t* bidx = nullptr;
  double* D64 = nullptr;           // FP64 rows gathered: D64(didx[i], j) += alpha * acc (in FP64)
  const int32_t* didx = nullptr;
};

// Job functors: tiles per box (count) and the tile for a box-local index (tile).
struct GramJob {  // G_side = W_side W_side^T, lower block triangle of 128 x 128 tiles (row pitch gram_ld(l))
  int64_t s;
  __device__ int64_t count(const BoxDesc& d) const { return 2 * tri_n(cdiv128(d.l)); }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t per = tri_n(cdiv128(d.l));
    const int side = (int)(loc / per);
    int64_t ti, tj;
    tri_idx(loc % per, ti, tj);
    float* wc = reinterpret_cast<float*>(g.workc);
    const float* W = wc + d.w_off + (int64_t)side * d.l * s;
    TcTile t;
    t.A = W + ti * GM * s;
    t.lda = s;
    t.m = (int)imin64(GM, d.l - ti * GM);
    t.B = W + tj * GN * s;
    t.ldb = s;
    t.n = (int)imin64(GN, d.l - tj * GN);
    t.bnm = 0;
    t.K = s;
    const int64_t lg = gram_ld(d.l);
    t.D = wc + d.g_off + (int64_t)side * d.l * lg + ti * GM * lg + tj * GN;
    t.ldd = lg;
    t.alpha = 1.f;
    t.beta = 0.f;
    return t;
  }
};
struct ProjNtJob {  // X_side(pass) = M_side W_side^T (b x l)
  int64_t s;
  int pass;
  __device__ int64_t count(const BoxDesc& d) const { return 2 * cdiv128(d.b) * cdiv128(d.l); }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t per = cdiv128(d.b) * cdiv128(d.l);
    const int side = (int)(loc / per);
    const int64_t ti = (loc % per) / cdiv128(d.l), tj = (loc % per) % cdiv128(d.l);
    float* wc = reinterpret_cast<float*>(g.workc);
    TcTile t;
    t.A = wc + d.mc_off + (int64_t)side * s + ti * GM * 2 * s;
    t.lda = 2 * s;
    t.m = (int)imin64(GM, d.b - ti * GM);
    t.B = wc + d.w_off + (int64_t)side * d.l * s + tj * GN * s;
    t.ldb = s;
    t.n = (int)imin64(GN, d.l - tj * GN);
    t.bnm = 0;
    t.K = s;
    t.D = wc + (pass ? d.x2_off : d.x_off) + (int64_t)side * d.b * d.l + ti * GM * d.l + tj * GN;
    t.ldd = d.l;
    t.alpha = 1.f;
    t.beta = 0.f;
    return t;
  }
};
struct ProjAccJob {  // M_side -= X_side(pass) W_side (b x s), B = W stored l x s
  int64_t s;
  int pass;
  __device__ int64_t count(const BoxDesc& d) const { return 2 * cdiv128(d.b) * cdiv128(s); }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t per = cdiv128(d.b) * cdiv128(s);
    const int side = (int)(loc / per);
    const int64_t ti = (loc % per) / cdiv128(s), tj = (loc % per) % cdiv128(s);
    float* wc = reinterpret_cast<float*>(g.workc);
    TcTile t;
    t.A = wc + (pass ? d.x2_off : d.x_off) + (int64_t)side * d.b * d.l + ti * GM * d.l;
    t.lda = d.l;
    t.m = (int)imin64(GM, d.b - ti * GM);
    t.B = wc + d.w_off + (int64_t)side * d.l * s + tj * GN;
    t.ldb = s;
    t.n = (int)imin64(GN, s - tj * GN);
    t.bnm = 1;
    t.K = d.l;
    t.D = wc + d.mc_off + (int64_t)side * s + ti * GM * 2 * s + tj * GN;
    t.ldd = 2 * s;
    t.alpha = -1.f;
    t.beta = 1.f;
    return t;
  }
};


// ---- blocked Cholesky and inverse on the tensor-core path (128-wide blocks, G row pitch lg) ----
// Block (i, j) of side `side` of the box's Gram area starts at gblk(...) + i*128*lg + j*128.
__device__ inline float* gram_side(const GroupArgs& g, const BoxDesc& d, int side) {
  return reinterpret_cast<float*>(g.workc) + d.g_off + (int64_t)side * d.l * gram_ld(d.l);
}
// Inverse of diagonal block p (128 x 128 row-major, zero padded).
__device__ inline float* dinv_blk(const GroupArgs& g, const BoxDesc& d, int side, int64_t p) {
  return reinterpret_cast<float*>(g.workc) + d.li_off + ((int64_t)side * cdiv128(d.l) + p) * GM * GM;
}
__device__ inline int rows_of(int64_t l, int64_t blk) { return (int)imin64(GM, l - blk * GM); }

struct CholPanelJob {  // L_ip = G_ip L_pp^-T for the blocks i > p below the diagonal block p
  int p;
  __device__ int64_t count(const BoxDesc& d) const {
    const int64_t t = cdiv128(d.l) - p - 1;
    return t > 0 ? 2 * t : 0;
  }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t per = cdiv128(d.l) - p - 1, lg = gram_ld(d.l);
    const int side = (int)(loc / per);
    const int64_t i = p + 1 + loc % per;
    float* G = gram_side(g, d, side);
    TcTile t;
    t.A = G + i * GM * lg + (int64_t)p * GM;
    t.lda = lg;
    t.m = rows_of(d.l, i);
    t.B = dinv_blk(g, d, side, p);
    t.ldb = GM;
    t.n = GM;
    t.bnm = 0;
    t.K = GM;
    t.D = G + i * GM * lg + (int64_t)p * GM;  // in place: the tile's own A, read before the epilogue
    t.ldd = lg;
    t.alpha = 1.f;
    t.beta = 0.f;
    return t;
  }
};
struct CholLeftJob {  // G_ip -= L_{i,0:p} L_{p,0:p}^T for i >= p (left-looking: column block p, K = 128 p)
  int p;
  __device__ int64_t count(const BoxDesc& d) const {
    const int64_t t = cdiv128(d.l) - p;
    return t > 0 ? 2 * t : 0;
  }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t per = cdiv128(d.l) - p, lg = gram_ld(d.l);
    const int side = (int)(loc / per);
    const int64_t i = p + loc % per;
    float* G = gram_side(g, d, side);
    TcTile t;
    t.A = G + i * GM * lg;
    t.lda = lg;
    t.m = rows_of(d.l, i);
    t.B = G + (int64_t)p * GM * lg;
    t.ldb = lg;
    t.n = rows_of(d.l, p);
    t.bnm = 0;
    t.K = (int64_t)p * GM;
    t.D = G + i * GM * lg + (int64_t)p * GM;  // column block p: disjoint from the columns read
    t.ldd = lg;
    t.alpha = -1.f;
    t.beta = 1.f;
    return t;
  }
};
struct LtildeJob {  // L~_ik = L_ii^-1 L_ik for k < i, in place
  __device__ int64_t count(const BoxDesc& d) const {
    const int64_t nb = cdiv128(d.l);
    return nb > 1 ? 2 * tri_n(nb - 1) : 0;
  }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t per = tri_n(cdiv128(d.l) - 1), lg = gram_ld(d.l);
    const int side = (int)(loc / per);
    int64_t ti, tj;
    tri_idx(loc % per, ti, tj);
    const int64_t i = ti + 1, k = tj;
    float* G = gram_side(g, d, side);
    TcTile t;
    t.A = dinv_blk(g, d, side, i);
    t.lda = GM;
    t.m = rows_of(d.l, i);
    t.B = G + i * GM * lg + k * GM;  // K x N = rows of block i x columns of block k, N contiguous
    t.ldb = lg;
    t.n = GM;
    t.bnm = 1;
    t.K = rows_of(d.l, i);
    t.D = G + i * GM * lg + k * GM;  // in place: the tile's own B, read before the epilogue
    t.ldd = lg;
    t.alpha = 1.f;
    t.beta = 0.f;
    return t;
  }
};
struct InvColJob {  // U_ji = -sum_{k=j}^{i-1} U_jk L~_ik^T for j < i (block column i of U = L^-T)
  int i;
  __device__ int64_t count(const BoxDesc& d) const { return cdiv128(d.l) > i ? 2 * (int64_t)i : 0; }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t lg = gram_ld(d.l);
    const int side = (int)(loc / i);
    const int64_t j = loc % i;
    float* G = gram_side(g, d, side);
    TcTile t;
    t.A = G + j * GM * lg + j * GM;  // row block j of U from column block j (U_jj on the diagonal)
    t.lda = lg;
    t.m = GM;
    t.B = G + (int64_t)i * GM * lg + j * GM;  // row block i of L~ from column block j
    t.ldb = lg;
    t.n = rows_of(d.l, i);
    t.bnm = 0;
    t.K = ((int64_t)i - j) * GM;
    t.D = G + j * GM * lg + (int64_t)i * GM;
    t.ldd = lg;
    t.alpha = -1.f;
    t.beta = 0.f;
    return t;
  }
};
struct SolveTJob {  // T = X U (U upper: column block j needs rows < 128 (j + 1))
  int pass;
  __device__ int64_t count(const BoxDesc& d) const { return 2 * cdiv128(d.b) * cdiv128(d.l); }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t nb = cdiv128(d.l), per = cdiv128(d.b) * nb, lg = gram_ld(d.l);
    const int side = (int)(loc / per);
    const int64_t a = (loc % per) / nb, j = (loc % per) % nb;
    float* wc = reinterpret_cast<float*>(g.workc);
    TcTile t;
    t.A = wc + (pass ? d.x2_off : d.x_off) + (int64_t)side * d.b * d.l + a * GM * d.l;
    t.lda = d.l;
    t.m = rows_of(d.b, a);
    t.B = gram_side(g, d, side) + j * GM;  // element (k, n) at B + k * lg + n
    t.ldb = lg;
    t.n = rows_of(d.l, j);
    t.bnm = 1;
    t.K = imin64(d.l, (j + 1) * GM);
    t.D = wc + d.t_off + (int64_t)side * d.b * lg + a * GM * lg + j * GM;
    t.ldd = lg;
    t.alpha = 1.f;
    t.beta = 0.f;
    return t;
  }
};
struct SolveCJob {  // X = T U^T (U upper: column block j needs columns >= 128 j of T); pass 1 adds into X_0
  int pass;
  __device__ int64_t count(const BoxDesc& d) const { return 2 * cdiv128(d.b) * cdiv128(d.l); }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t nb = cdiv128(d.l), per = cdiv128(d.b) * nb, lg = gram_ld(d.l);
    const int side = (int)(loc / per);
    const int64_t a = (loc % per) / nb, j = (loc % per) % nb;
    float* wc = reinterpret_cast<float*>(g.workc);
    float* G = gram_side(g, d, side);
    TcTile t;
    t.A = wc + d.t_off + (int64_t)side * d.b * lg + a * GM * lg + j * GM;
    t.lda = lg;
    t.m = rows_of(d.b, a);
    t.B = G + j * GM * lg + j * GM;
    t.ldb = lg;
    t.n = rows_of(d.l, j);
    t.bnm = 0;
    t.K = d.l - j * GM;
    const int64_t xo = (int64_t)side * d.b * d.l + a * GM * d.l + j * GM;
    t.D = wc + (pass ? d.x2_off : d.x_off) + xo;
    t.ldd = d.l;
    t.alpha = 1.f;
    t.beta = 0.f;
    if (pass) t.D2 = wc + d.x_off + xo;
    return t;
  }
};

struct LcUcJob {  // Uc = X_RR^-1 [X_RS X_RN] (side 0), Lc^T = X_RR^-T [X_SR^T X_NR^T] (side 1), r x w each
  __device__ int64_t count(const BoxDesc& d) const { return 2 * cdiv128(d.r) * cdiv128((int64_t)d.kp + d.n); }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t r = d.r, w = (int64_t)d.kp + d.n, nt = cdiv128(w), per = cdiv128(r) * nt;
    const int side = (int)(loc / per);
    const int64_t ti = (loc % per) / nt, tj = (loc % per) % nt;
    float* wc = reinterpret_cast<float*>(g.workc);
    const float* P = wc + d.w_off;  // [X_RR^-1 | X_RR^-T | Uc's right-hand block | Lc^T's] (k_lcuc_prep)
    TcTile t;
    t.A = P + (side == 0 ? 0 : r * r) + ti * GM * r;
    t.lda = r;
    t.m = rows_of(r, ti);
    t.B = P + 2 * r * r + (int64_t)side * r * w + tj * GN;  // element (k, n) at B + k w + n
    t.ldb = w;
    t.n = (int)imin64(GN, w - tj * GN);
    t.bnm = 1;
    t.K = r;
    t.D = wc + d.e_off + (side == 0 ? r * w : 0) + ti * GM * w + tj * GN;  // the Schur update's operands
    t.ldd = w;
    t.alpha = 1.f;
    t.beta = 0.f;
    return t;
  }
};

// Block elimination on the sketches (the Schur complement of X_RR, Algorithm 1): with Lc = LcT^T
// (w x r) and Uc (r x w), w = k' + n, stored FP32 in the extraction area, and Y_R, Z_R staged FP32
// in the sketch area (k_schur_prep):
//   product 0: Y_SN -= Lc Y_R        (A = LcT read K x M, B = Y_R)
//   product 1: Om_R += Uc Om_SN      (A = Uc,             B = Om rows SN, FP64)
//   product 2: Z_SN -= Uc^T Z_R      (A = Uc read K x M,  B = Z_R)
//   product 3: Ps_R += Lc^T Ps_SN    (A = LcT,            B = Ps rows SN, FP64)
// each into the FP64 sketch rows in place.  Same-colour boxes touch disjoint rows.
struct SchurJob {
  int64_t s;
  __device__ int64_t count(const BoxDesc& d) const {
    return 2 * (cdiv128((int64_t)d.kp + d.n) + cdiv128(d.r)) * cdiv128(s);
  }
  __device__ TcTile tile(const GroupArgs& g, const BoxDesc& d, int64_t loc) const {
    const int64_t r = d.r, w = (int64_t)d.kp + d.n, nt = cdiv128(s);
    const int64_t pw = cdiv128(w) * nt, pr = cdiv128(r) * nt;
    int prod;
    if (loc < pw) prod = 0;
    else if ((loc -= pw) < pr) prod = 1;
    else if ((loc -= pr) < pw) prod = 2;
    else {
      loc -= pw;
      prod = 3;
    }
    const int64_t ti = loc / nt, tj = loc % nt;
    const float* wc = reinterpret_cast<const float*>(g.workc);
    const float* LcT = wc + d.e_off;
    const float* Uc = LcT + r * w;
    const int32_t* R = g.fi + fi_R(d);
    const int32_t* SN = g.fi + fi_S(d);
    TcTile t;
    t.bnm = 1;
    t.ldb = s;
    t.n = (int)imin64(GN, s - tj * GN);
    t.D = nullptr;
    t.ldd = s;
    t.beta = 1.f;
    if (prod == 0 || prod == 2) {  // M = w (rows SN), K = r
      t.anm = 1;
      t.A = (prod == 0 ? LcT : Uc) + ti * GM;
      t.lda = w;
      t.m = rows_of(w, ti);
      t.B = wc + d.mc_off + (prod == 0 ? 0 : r * s) + tj * GN;
      t.K = r;
      t.D64 = (prod == 0 ? g.Y : g.Z) + tj * GN;
      t.didx = SN + ti * GM;
      t.alpha = -1.f;
    } else {  // M = r (rows R), K = w
      t.A = (prod == 1 ? Uc : LcT) + ti * GM * w;
      t.lda = w;
      t.m = rows_of(r, ti);
      t.B = nullptr;
      t.B64 = (prod == 1 ? g.Om : g.Ps) + tj * GN;
      t.bidx = SN;
      t.K = w;
      t.D64 = (prod == 1 ? g.Om : g.Ps) + tj * GN;
      t.didx = R + ti * GM;
      t.alpha = 1.f;
    }
    return t;
  }
};
template <class Job>
struct sketch_io {
  static constexpr bool value = false;
};
template <>
struct sketch_io<SchurJob> {
  static constexpr bool value = true;
};

template <class Job>
__device__ int find_box(const BoxDesc* desc, int nbox, int64_t item, const Job& job, int64_t& local) {
  // block-wide prefix sum over the boxes' tile counts, blockDim.x boxes at a time
  __shared__ int s_box;
  __shared__ int64_t s_local;
  __shared__ int64_t s_warp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (threadIdx.x == 0) s_box = -1;
  int64_t base = 0;
  for (int c0 = 0; c0 < nbox; c0 += blockDim.x) {
    const int i = c0 + (int)threadIdx.x;
    const int64_t c = i < nbox ? job.count(desc[i]) : 0;
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
    if (s_box >= 0 || item < base) break;
  }
  __syncthreads();
  local = s_local;
  return s_box;
}

// 16 consecutive K values of one K-contiguous row (zero outside the valid rows and K).
__device__ __forceinline__ void load_row16(float v[16], const float* src, bool row_ok, int64_t kleft, bool vec) {
  if (row_ok && vec && kleft >= 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 x = __ldg(reinterpret_cast<const float4*>(src) + q);
      v[4 * q] = x.x;
      v[4 * q + 1] = x.y;
      v[4 * q + 2] = x.z;
      v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = (row_ok && q < kleft) ? __ldg(src + q) : 0.f;
  }
}
// 16 consecutive columns of one K row of an N-contiguous operand (zero outside).
__device__ __forceinline__ void load_col16(float v[16], const float* src, bool k_ok, int nleft, bool vec) {
  if (k_ok && vec && nleft >= 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 x = __ldg(reinterpret_cast<const float4*>(src) + q);
      v[4 * q] = x.x;
      v[4 * q + 1] = x.y;
      v[4 * q + 2] = x.z;
      v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = (k_ok && q < nleft) ? __ldg(src + q) : 0.f;
  }
}
// 16 consecutive columns of one K row of an FP64 operand (zero outside), kept as the two 32-bit
// halves of each value (v[2q] low, v[2q+1] high) so that the loads of the next slice stay in flight
// until it is converted (a conversion here would wait for them).
__device__ __forceinline__ void load_col16_f64(float v[32], const double* src, bool k_ok, int nleft, bool vec) {
  auto put = [&](int q, double x) {
    v[2 * q] = __int_as_float(__double2loint(x));
    v[2 * q + 1] = __int_as_float(__double2hiint(x));
  };
  if (k_ok && vec && nleft >= 16) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double2 x = __ldg(reinterpret_cast<const double2*>(src) + q);
      put(2 * q, x.x);
      put(2 * q + 1, x.y);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) put(q, (k_ok && q < nleft) ? __ldg(src + q) : 0.0);
  }
}
// Split into TF32 hi/lo and store row `row`, K positions k0l .. k0l + 15, of the swizzled tiles.
__device__ __forceinline__ void store_row16(unsigned char* hi, unsigned char* lo, int row, int k0l, const float v[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float4 h, l;
    h.x = tf32_hi(v[4 * q]);
    h.y = tf32_hi(v[4 * q + 1]);
    h.z = tf32_hi(v[4 * q + 2]);
    h.w = tf32_hi(v[4 * q + 3]);
    l.x = v[4 * q] - h.x;
    l.y = v[4 * q + 1] - h.y;
    l.z = v[4 * q + 2] - h.z;
    l.w = v[4 * q + 3] - h.w;
    const uint32_t off = sw128(row, k0l + 4 * q);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}
// Split and store column k, rows n0 .. n0 + 15 (the transpose of an N-contiguous operand).
__device__ __forceinline__ void store_col16(unsigned char* hi, unsigned char* lo, int n0, int k, const float v[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float h = tf32_hi(v[q]);
    const uint32_t off = sw128(n0 + q, k);
    *reinterpret_cast<float*>(hi + off) = h;
    *reinterpret_cast<float*>(lo + off) = v[q] - h;
  }
}

// 16-byte asynchronous copy global -> shared (both 16-byte aligned); the bytes beyond src_bytes
// (0..16) are written as zeros and not read.
__device__ __forceinline__ void cp_async16(uint32_t dst, const float* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// barrier of the eight producer warps only (the MMA warp does not take part)
__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(GPROD) : "memory"); }

template <class Job>
__global__ void __launch_bounds__(GTHREADS, 1) k_tc_grouped(GroupArgs g, Job job) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[GNST], empty[GNST];
  __shared__ uint32_t s_tmem;
  __shared__ int s_timeout;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  int64_t loc;
  const int bi = find_box(g.desc, g.nbox, blockIdx.x, job, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const TcTile t = job.tile(g, d, loc);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nchunk = (t.K + GK - 1) / GK;
  constexpr bool kIO = sketch_io<Job>::value;
  if (tid == 0) {
    s_timeout = 0;
    for (int s = 0; s < GNST; ++s) {
      bar_init(smem_u32(&full[s]), GPROD);
      bar_init(smem_u32(&empty[s]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&s_tmem, GTMEM);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;

  // Asynchronous producers, for tiles whose A and B are both K-contiguous with 16-byte aligned rows:
  // slice ch's raw FP32 operands are copied in 16-byte pieces (eight lanes per 128-byte K row, four
  // rows per warp instruction) into the hi tiles of stage ch % 3, two slices ahead of the split;
  // once a slice has landed (cp.async.wait_group, then a barrier of the producer warps) each
  // thread splits 16 values of A and of B in place: hi = v with the low 13 mantissa bits cleared,
  // lo = v - hi.  Other tiles take the register path below.
  const bool async16 = !kIO && !t.bnm && ((t.lda & 3) == 0) && ((t.ldb & 3) == 0) &&
                       ((reinterpret_cast<uintptr_t>(t.A) & 15) == 0) && ((reinterpret_cast<uintptr_t>(t.B) & 15) == 0);
  if (warp < GPROD / 32 && async16) {
    auto issue = [&](int64_t ch) {
      const int st = (int)(ch % GNST);
      unsigned char* Ahi = smem + st * GSTAGE;
      unsigned char* Bhi = Ahi + 2 * OP_BYTES;
      const int64_t k0 = ch * GK;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = tid + GPROD * j, row = c >> 3, kc = (c & 7) * 4;
        const int64_t kl = t.K - k0 - kc;  // valid K values from this piece on
        const uint32_t kb = kl >= 4 ? 16u : (kl > 0 ? (uint32_t)kl * 4u : 0u);
        const uint32_t ab = row < t.m ? kb : 0u, bb = row < t.n ? kb : 0u;
        cp_async16(smem_u32(Ahi + sw128(row, kc)), ab ? t.A + (int64_t)row * t.lda + k0 + kc : t.A, ab);
        cp_async16(smem_u32(Bhi + sw128(row, kc)), bb ? t.B + (int64_t)row * t.ldb + k0 + kc : t.B, bb);
      }
    };
    const int srow = tid >> 1, skh = (tid & 1) * 16;
    auto split = [&](unsigned char* hi, unsigned char* lo) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t off = sw128(srow, skh + 4 * q);
        const float4 v = *reinterpret_cast<const float4*>(hi + off);
        float4 h, l;
        h.x = tf32_hi(v.x);
        h.y = tf32_hi(v.y);
        h.z = tf32_hi(v.z);
        h.w = tf32_hi(v.w);
        l.x = v.x - h.x;
        l.y = v.y - h.y;
        l.z = v.z - h.z;
        l.w = v.w - h.w;
        *reinterpret_cast<float4*>(hi + off) = h;
        *reinterpret_cast<float4*>(lo + off) = l;
      }
    };
    constexpr int64_t AHEAD = GNST - 1;
    for (int64_t p = 0; p < AHEAD; ++p) {
      if (p < nchunk) issue(p);
      cp_async_commit();
    }
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      const int st = (int)(ch % GNST);
      unsigned char* Ahi = smem + st * GSTAGE;
      cp_async_wait<GNST - 2>();  // this thread's copies of slice ch are done
      producer_sync();            // ... and every producer's
      split(Ahi, Ahi + OP_BYTES);
      split(Ahi + 2 * OP_BYTES, Ahi + 3 * OP_BYTES);
      fence_proxy_async();
      bar_arrive(smem_u32(&full[st]));
      const int64_t nx = ch + AHEAD;  // into the stage the MMA of slice ch - 1 frees
      if (nx < nchunk) {
        if (nx >= GNST && !bar_wait(smem_u32(&empty[nx % GNST]), (uint32_t)(((nx / GNST) - 1) & 1))) s_timeout = 1;
        issue(nx);
      }
      cp_async_commit();
    }
    cp_async_wait<0>();
  } else if (warp < GPROD / 32) {
    // A: row tid/2, K half (tid&1)*16.  B (K-contiguous): the same.  B (N-contiguous): k = tid%32,
    // columns (tid/32)*16 .. +15, transposed into rows n of the K-major tile.  The operands of the
    // next slice are loaded into registers while this slice is split and stored.
    // Sketch-update jobs: A may be stored K x M (loaded and stored like an N-contiguous B) and B
    // may be FP64 rows gathered through an index list.
    const int r = tid >> 1, kh = (tid & 1) * 16;
    const bool anm = kIO && t.anm;
    const bool avec = ((t.lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(t.A) & 15) == 0);
    const bool bvec = kIO && t.B64 ? (((t.ldb & 1) == 0) && ((reinterpret_cast<uintptr_t>(t.B64) & 15) == 0))
                                   : (((t.ldb & 3) == 0) && ((reinterpret_cast<uintptr_t>(t.B) & 15) == 0));
    const int bk = tid & 31, bn0 = (tid >> 5) * 16;
    constexpr int NB = kIO ? 32 : 16;  // next-slice B registers (FP64 halves for the sketch updates)
    auto load = [&](int64_t ch, float va[16], float vb[NB]) {
      const int64_t k0 = ch * GK;
      if (anm) load_col16(va, t.A + (k0 + bk) * t.lda + bn0, k0 + bk < t.K, t.m - bn0, avec);
      else load_row16(va, t.A + (int64_t)r * t.lda + k0 + kh, r < t.m, t.K - k0 - kh, avec);
      if (!t.bnm) {
        load_row16(vb, t.B + (int64_t)r * t.ldb + k0 + kh, r < t.n, t.K - k0 - kh, bvec);
      } else if (kIO && t.B64) {
        if constexpr (kIO) {
          const bool k_ok = k0 + bk < t.K;
          const double* src = k_ok ? t.B64 + (int64_t)t.bidx[k0 + bk] * t.ldb + bn0 : t.B64;
          load_col16_f64(vb, src, k_ok, t.n - bn0, bvec);
        }
      } else {
        load_col16(vb, t.B + (k0 + bk) * t.ldb + bn0, k0 + bk < t.K, t.n - bn0, bvec);
      }
    };
    float va[16], vb[16], na[16], nb[NB];
    // the current slice's B as FP32 from the raw registers
    auto take_b = [&](const float raw[NB]) {
      if constexpr (kIO) {
        if (t.B64) {
#pragma unroll
          for (int q = 0; q < 16; ++q) vb[q] = f64_bits_to_f32(__float_as_uint(raw[2 * q + 1]), __float_as_uint(raw[2 * q]));
          return;
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) vb[q] = raw[q];
    };
    if (nchunk > 0) {
      load(0, va, nb);
      take_b(nb);
    }
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      const int st = (int)(ch % GNST);
      const int64_t u = ch / GNST;
      unsigned char* Ahi = smem + st * GSTAGE;
      unsigned char* Alo = Ahi + OP_BYTES;
      unsigned char* Bhi = Alo + OP_BYTES;
      unsigned char* Blo = Bhi + OP_BYTES;
      if (ch + 1 < nchunk) load(ch + 1, na, nb);
      if (ch >= GNST && !bar_wait(smem_u32(&empty[st]), (uint32_t)((u - 1) & 1))) s_timeout = 1;
      if (anm) store_col16(Ahi, Alo, bn0, bk, va);
      else store_row16(Ahi, Alo, r, kh, va);
      if (!t.bnm) store_row16(Bhi, Blo, r, kh, vb);
      else store_col16(Bhi, Blo, bn0, bk, vb);
      fence_proxy_async();
      bar_arrive(smem_u32(&full[st]));
#pragma unroll
      for (int q = 0; q < 16; ++q) va[q] = na[q];
      take_b(nb);
    }
  } else if (lane == 0) {
    const uint32_t idesc = idesc_tf32(GM, GN);
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      const int st = (int)(ch % GNST);
      if (!bar_wait(smem_u32(&full[st]), (uint32_t)((ch / GNST) & 1))) s_timeout = 1;
      fence_after();
      const uint32_t a_hi = smem_u32(smem + st * GSTAGE);
      mma_3xtf32_chunk(tmem, a_hi, a_hi + OP_BYTES, a_hi + 2 * OP_BYTES, a_hi + 3 * OP_BYTES, idesc, ch == 0);
      mma_commit(smem_u32(&empty[st]));
    }
  }
  if (warp == GPROD / 32) __syncwarp();
  if (nchunk > 0) {
    const int64_t last = nchunk - 1;
    if (!bar_wait(smem_u32(&empty[last % GNST]), (uint32_t)((last / GNST) & 1))) s_timeout = 1;
  }
  fence_after();
  if (warp < GPROD / 32) {
    // epilogue: warp w reads TMEM lanes 32*(w%4).. (its rows), columns (w/4)*64 .. +64
    const int row = 32 * (warp & 3) + lane;
    const int colbase = (warp >> 2) * 64;
    if constexpr (kIO) {
      if (t.D64) {  // FP64 sketch rows, read-modify-write in FP64; the next 16 values load meanwhile
        const bool rok = row < t.m;
        double* drow = rok ? t.D64 + (int64_t)t.didx[row] * t.ldd + colbase : t.D64;
        const bool dvec = ((t.ldd & 1) == 0) && ((reinterpret_cast<uintptr_t>(t.D64) & 15) == 0);
        const float al = t.alpha;  // +-1: the product's sign, exact in FP32
        auto ld16 = [&](int cc, double v[16]) {
          const int nleft = t.n - colbase - cc;
          if (dvec && nleft >= 16) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const double2 x = reinterpret_cast<const double2*>(drow + cc)[q];
              v[2 * q] = x.x;
              v[2 * q + 1] = x.y;
            }
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = q < nleft ? drow[cc + q] : 0.0;
          }
        };
        double cur[16], nxt[16];
        if (rok && colbase < t.n) ld16(0, cur);
        for (int cc = 0; cc < 64; cc += 16) {
          if (colbase + cc >= t.n) break;  // warp-uniform
          uint32_t rr[16];
          tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(colbase + cc), rr);
          const bool more = cc + 16 < 64 && colbase + cc + 16 < t.n;
          if (rok && more) ld16(cc + 16, nxt);
          if (rok) {
            const int nleft = t.n - colbase - cc;
#pragma unroll
            for (int q = 0; q < 16; ++q) cur[q] += f32_to_f64_exact(nchunk > 0 ? al * __uint_as_float(rr[q]) : 0.f);
            if (dvec && nleft >= 16) {
#pragma unroll
              for (int q = 0; q < 8; ++q) reinterpret_cast<double2*>(drow + cc)[q] = make_double2(cur[2 * q], cur[2 * q + 1]);
            } else {
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (q < nleft) drow[cc + q] = cur[q];
            }
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) cur[q] = nxt[q];
        }
      }
    }
    for (int cc = 0; cc < 64; cc += 16) {
      if (kIO && t.D64) break;
      if (colbase + cc >= t.n) break;  // warp-uniform
      uint32_t rr[16];
      tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(colbase + cc), rr);
      if (row < t.m) {
        float* drow = t.D + (int64_t)row * t.ldd + colbase + cc;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (colbase + cc + q < t.n) {
            const float acc = nchunk > 0 ? __uint_as_float(rr[q]) : 0.f;
            drow[q] = t.beta == 0.f ? t.alpha * acc : fmaf(t.alpha, acc, t.beta * drow[q]);
            if (t.D2) t.D2[(int64_t)row * t.ldd + colbase + cc + q] += t.alpha * acc;
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, GTMEM);
  if (tid == 0 && s_timeout && g.err) atomicCAS(g.err, 0, kDevTimeout);
}


// Diagonal block p of the blocked Cholesky, one CTA per (box, side) with l > 128 p: G_pp = L L^T
// and X = L^-1, both blocked by 16.  Cholesky, right-looking over eight 16-column panels: one warp
// factors the panel (rows in registers, 16 column steps with shuffles, no block barrier), then all
// warps apply its rank-16 update to the trailing lower triangle.  Inverse: the eight 16 x 16
// diagonal blocks by one warp each (a column of X per lane, forward substitution), then block row
// by block row X_ij = -X_ii sum_{j<=k<i} L_ik X_kj.  Rows beyond the box's l are padded with the
// identity.  Writes X (lower, zero padded) to the block's inverse area and U_pp = X^T (upper, zeros
// below) to the diagonal block of G.  A pivot that is not positive and finite records
// kDevNonfinite (and is replaced by 1 so that the factorisation completes).
constexpr int DB = 128, DLD = DB + 1, DTHREADS = 512, DW = 16;
constexpr int DSMEM = (2 * DB * DLD + DW * DB) * 4;
struct DiagCount {
  int p;
  __device__ int64_t count(const BoxDesc& d) const { return d.l > (int64_t)p * DB ? 2 : 0; }
};
__global__ void __launch_bounds__(DTHREADS, 1) k_chol_diag_tc(GroupArgs g, int p) {
  extern __shared__ float dsm[];
  float* S = dsm;                // DB x DLD: G_pp, then L (lower)
  float* Xs = S + DB * DLD;      // DB x DLD: X = L^-1 (lower)
  float* Tb = Xs + DB * DLD;     // DW x DB: partial products of one block row
  __shared__ int s_bad;
  int64_t loc;
  const DiagCount cnt{p};
  const int bi = find_box(g.desc, g.nbox, blockIdx.x, cnt, loc);
  if (bi < 0) return;
  const BoxDesc d = g.desc[bi];
  const int side = (int)loc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t lg = gram_ld(d.l), o = (int64_t)p * DB;
  const int nbp = (int)imin64(DB, d.l - o);
  float* G = gram_side(g, d, side) + o * lg + o;
  if (tid == 0) s_bad = 0;
  for (int e = tid; e < DB * DB; e += DTHREADS) {
    const int i = e / DB, j = e % DB;
    float v = (i == j) ? 1.f : 0.f;
    if (j <= i && i < nbp) v = G[(int64_t)i * lg + j];
    S[i * DLD + j] = v;
  }
  __syncthreads();
  // ---- Cholesky ----
  for (int c0 = 0; c0 < DB; c0 += DW) {
    if (warp == 0) {
      // panel rows c0 + lane + 32 q, columns c0 .. c0 + 15
      float P[4][DW];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int cc = 0; cc < DW; ++cc) {
          const int r = c0 + lane + 32 * q;
          P[q][cc] = r < DB ? S[r * DLD + c0 + cc] : 0.f;
        }
      bool bad = false;
#pragma unroll
      for (int cc = 0; cc < DW; ++cc) {
        float a = __shfl_sync(0xffffffffu, P[0][cc], cc);  // row c0 + cc lives in lane cc, q = 0
        if (!(a > 0.f) || !isfinite(a)) {
          bad = true;
          a = 1.f;
        }
        const float dg = __fsqrt_rn(a), rd = __frcp_rn(dg);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int ri = lane + 32 * q;
          P[q][cc] = ri == cc ? dg : (ri > cc ? P[q][cc] * rd : P[q][cc]);
        }
#pragma unroll
        for (int c2 = 1; c2 < DW; ++c2) {
          if (c2 <= cc) continue;  // compile-time
          const float lc = __shfl_sync(0xffffffffu, P[0][cc], c2);  // L[c0 + c2][c0 + cc]
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (lane + 32 * q >= c2) P[q][c2] = fmaf(-P[q][cc], lc, P[q][c2]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int cc = 0; cc < DW; ++cc) {
          const int r = c0 + lane + 32 * q;
          if (r < DB) {
            S[r * DLD + c0 + cc] = P[q][cc];
            Tb[cc * DB + r] = P[q][cc];  // the panel transposed, for the update below
          }
        }
      if (lane == 0 && bad) s_bad = 1;
    }
    __syncthreads();
    // rank-16 update of the trailing lower triangle, a 4 x 4 block (bi, bj <= bi) per thread
    const int c1 = c0 + DW;
    if (c1 < DB) {
      const int nb4 = (DB - c1) / 4, nblk = nb4 * (nb4 + 1) / 2;  // at most 406 < DTHREADS
      if (tid < nblk) {
        int bi = (int)((sqrtf(8.f * (float)tid + 1.f) - 1.f) * 0.5f);
        while (bi * (bi + 1) / 2 > tid) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= tid) ++bi;
        const int bj = tid - bi * (bi + 1) / 2;
        const int i0 = c1 + 4 * bi, j0 = c1 + 4 * bj;
        float acc[4][4] = {};
#pragma unroll
        for (int k = 0; k < DW; ++k) {
          const float4 a = *reinterpret_cast<const float4*>(Tb + k * DB + i0);
          const float4 b = *reinterpret_cast<const float4*>(Tb + k * DB + j0);
          const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (j0 + v <= i0 + u) S[(i0 + u) * DLD + j0 + v] -= acc[u][v];
      }
    }
    __syncthreads();
  }
  // ---- X = L^-1: diagonal 16 x 16 blocks, one warp each, a column per lane ----
  if (warp < DB / DW && lane < DW) {
    const int k0 = warp * DW, j = lane;
    float x[DW];
#pragma unroll
    for (int r = 0; r < DW; ++r) {
      float acc = (r == j) ? 1.f : 0.f;
#pragma unroll
      for (int t = 0; t < r; ++t) acc = fmaf(-S[(k0 + r) * DLD + k0 + t], x[t], acc);
      x[r] = r >= j ? acc / S[(k0 + r) * DLD + k0 + r] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < DW; ++r) Xs[(k0 + r) * DLD + k0 + j] = x[r];
  }
  __syncthreads();
  // block rows i = 1..7: T_ij = sum_{j<=k<i} L_ik X_kj, then X_ij = -X_ii T_ij
  for (int ib = 1; ib < DB / DW; ++ib) {
    const int i0 = ib * DW;
    for (int e = tid; e < DW * i0; e += DTHREADS) {  // T: DW rows x (columns of blocks j < i)
      const int a = e / i0, col = e % i0, jb = col / DW;
      float acc = 0.f;
      for (int k = jb * DW; k < i0; ++k) acc = fmaf(S[(i0 + a) * DLD + k], Xs[k * DLD + col], acc);
      Tb[a * DB + col] = acc;
    }
    __syncthreads();
    for (int e = tid; e < DW * i0; e += DTHREADS) {
      const int a = e / i0, col = e % i0;
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < DW; ++c) acc = fmaf(Xs[(i0 + a) * DLD + i0 + c], Tb[c * DB + col], acc);
      Xs[(i0 + a) * DLD + col] = -acc;
    }
    __syncthreads();
  }
  float* Xo = dinv_blk(g, d, side, p);
  for (int e = tid; e < DB * DB; e += DTHREADS) {
    const int i = e / DB, j = e % DB;
    Xo[e] = (i < nbp && j < nbp && j <= i) ? Xs[i * DLD + j] : 0.f;
  }
  for (int e = tid; e < nbp * nbp; e += DTHREADS) {
    const int i = e / nbp, j = e % nbp;
    G[(int64_t)i * lg + j] = (j >= i) ? Xs[j * DLD + i] : 0.f;  // U = X^T
  }
  if (tid == 0 && s_bad && g.err) atomicCAS(g.err, 0, (int)kDevNonfinite);
}

template <class Job>
void launch_job(Launch L, const GroupArgs& g, const Job& job, int64_t items) {
  if (items <= 0) return;
  static PerDeviceOnce attr;
  attr([] { cudaFuncSetAttribute(k_tc_grouped<Job>, cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM); });
  k_tc_grouped<Job><<<(unsigned)items, GTHREADS, GSMEM, L.st>>>(g, job);
  if (L.counter) ++*L.counter;
}

template <class Count>
int64_t items_of_h(const std::vector<BoxDesc>& h, Count c) {
  int64_t n = 0;
  for (const BoxDesc& d : h) n += c(d);
  return n;
}

// Self-test of the bounded mbarrier wait every kernel here uses: one CTA initialises a barrier
// that expects one arrival, makes that arrival only when `arrive` is set, and waits for the phase
// with at most `polls` polls.  With no arrival the wait must expire and record kDevTimeout; the
// kernel then returns normally, so the context stays usable.
__global__ void __launch_bounds__(32) k_wait_selftest(long long polls, int arrive, int* err) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = tc::smem_u32(&bar);
  if (threadIdx.x == 0) tc::bar_init(b, 1);
  __syncthreads();
  if (threadIdx.x == 0 && arrive) tc::bar_arrive(b);
  __syncthreads();
  if (threadIdx.x == 0 && !tc::bar_wait(b, 0, polls)) atomicCAS(err, 0, (int)kDevTimeout);
}

}  // namespace

namespace {
__global__ void k_convert_selftest(const double* x, int64_t n, float* f, double* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const float r = f64_bits_to_f32((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v));
  f[i] = r;
  g[i] = f32_to_f64_exact(r);
}
}  // namespace
void launch_convert_selftest(Launch L, const double* x, int64_t n, float* f, double* g) {
  if (n <= 0) return;
  k_convert_selftest<<<(unsigned)((n + 255) / 256), 256, 0, L.st>>>(x, n, f, g);
  if (L.counter) ++*L.counter;
}
void launch_wait_selftest(Launch L, long long polls, int arrive, int* err) {
  polls = std::min(std::max(polls, 1ll), tc::kWaitLimit);
  k_wait_selftest<<<1, 32, 0, L.st>>>(polls, arrive, err);
  if (L.counter) ++*L.counter;
}

void launch_gram_tc(Launch L, const GroupArgs& g, const std::vector<BoxDesc>& h) {
  launch_job(L, g, GramJob{g.s}, items_of_h(h, [](const BoxDesc& d) { return 2 * tri_n(cdiv128(d.l)); }));
}
void launch_proj_nt_tc(Launch L, const GroupArgs& g, int pass, const std::vector<BoxDesc>& h) {
  launch_job(L, g, ProjNtJob{g.s, pass},
             items_of_h(h, [](const BoxDesc& d) { return 2 * cdiv128(d.b) * cdiv128(d.l); }));
}
void launch_proj_acc_tc(Launch L, const GroupArgs& g, int pass, const std::vector<BoxDesc>& h) {
  const int64_t s = g.s;
  launch_job(L, g, ProjAccJob{g.s, pass},
             items_of_h(h, [s](const BoxDesc& d) { return 2 * cdiv128(d.b) * cdiv128(s); }));
}

void launch_chol_tc(Launch L, const GroupArgs& g, const std::vector<BoxDesc>& h) {
  int64_t nbmax = 0;
  for (const BoxDesc& d : h) nbmax = std::max<int64_t>(nbmax, cdiv128(d.l));
  static PerDeviceOnce attr;
  attr([] { cudaFuncSetAttribute(k_chol_diag_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, DSMEM); });
  // left-looking: column block p takes all earlier panels in one product (K = 128 p), then its
  // diagonal block is factored and inverted and the blocks below it are scaled
  for (int p = 0; p < (int)nbmax; ++p) {
    if (p > 0)
      launch_job(L, g, CholLeftJob{p}, items_of_h(h, [p](const BoxDesc& d) {
                   const int64_t t = cdiv128(d.l) - p;
                   return t > 0 ? 2 * t : (int64_t)0;
                 }));
    const int64_t nd = items_of_h(h, [p](const BoxDesc& d) { return d.l > (int64_t)p * DB ? 2 : 0; });
    if (nd > 0) {
      k_chol_diag_tc<<<(unsigned)nd, DTHREADS, DSMEM, L.st>>>(g, p);
      if (L.counter) ++*L.counter;
    }
    launch_job(L, g, CholPanelJob{p}, items_of_h(h, [p](const BoxDesc& d) {
                 const int64_t t = cdiv128(d.l) - p - 1;
                 return t > 0 ? 2 * t : (int64_t)0;
               }));
  }
  launch_job(L, g, LtildeJob{}, items_of_h(h, [](const BoxDesc& d) {
               const int64_t nb = cdiv128(d.l);
               return nb > 1 ? 2 * tri_n(nb - 1) : (int64_t)0;
             }));
  for (int i = 1; i < (int)nbmax; ++i)
    launch_job(L, g, InvColJob{i},
               items_of_h(h, [i](const BoxDesc& d) { return cdiv128(d.l) > i ? 2 * (int64_t)i : (int64_t)0; }));
}
void launch_lcuc_tc(Launch L, const GroupArgs& g, const std::vector<BoxDesc>& h) {
  launch_job(L, g, LcUcJob{}, items_of_h(h, [](const BoxDesc& d) {
               return 2 * cdiv128(d.r) * cdiv128((int64_t)d.kp + d.n);
             }));
}
void launch_schur_tc(Launch L, const GroupArgs& g, const std::vector<BoxDesc>& h) {
  const int64_t s = g.s;
  launch_job(L, g, SchurJob{s}, items_of_h(h, [s](const BoxDesc& d) {
               return 2 * (cdiv128((int64_t)d.kp + d.n) + cdiv128(d.r)) * cdiv128(s);
             }));
}
void launch_solve_tc(Launch L, const GroupArgs& g, int pass, const std::vector<BoxDesc>& h) {
  const int64_t items = items_of_h(h, [](const BoxDesc& d) { return 2 * cdiv128(d.b) * cdiv128(d.l); });
  launch_job(L, g, SolveTJob{pass}, items);
  launch_job(L, g, SolveCJob{pass}, items);
}

}  // namespace rsrs
