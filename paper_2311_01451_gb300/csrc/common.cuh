// Internal declarations shared by the CUDA translation units of librsrs.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/rsrs.h"
#include "tree.h"

namespace rsrs {

// Device error word: set (first writer wins) by kernels that meet a bad pivot.
enum DevErr : int { kDevOk = 0, kDevSingular = 1, kDevNonfinite = 2, kDevTimeout = 3 };

// One compressed box of a (level, colour) group, as the device kernels see it.
// All offsets are element offsets into the buffers named in the comments.
// Workspaces: `work` is FP64 (the CPQR input and R rows); `workc` holds the blocks of the
// compute type (FP32 in the mixed path, FP64 otherwise); offsets count elements of each type.
struct BoxDesc {
  int32_t b, n, l, kp, r, pad_;
  int64_t bn_off;   // int32 work: l tree positions [B_act | N_act]
  int64_t g_off;    // workc: two l x l Grams / Cholesky factors (Omega side, then Psi side); row
                    //   pitch and side stride l and l * l on the SIMT path, gram_ld(l) and
                    //   l * gram_ld(l) on the tensor-core path (room for 2 l gram_ld(l))
  int64_t t_off;    // workc (tensor-core path): two b x gram_ld(l) blocks X L^-T of the projection
  int64_t x_off;    // workc: two b x l least-squares coefficient blocks (Y, Z)
  int64_t x2_off;   // workc: two b x l correction-pass blocks
  int64_t mc_off;   // workc: b x 2s sketches [Y_B | Z_B], projected in place
  int64_t w_off;    // workc: near-field test rows W = Om[B u N], then V = Ps[B u N], l x s each
  int64_t e_off;    // workc: extraction blocks, 2 x r x l
  int64_t m_off;    // work (FP64): b x 2s projected sketches for the CPQR
  int64_t cp_off;   // work (FP64): CPQR R rows, kp x b
  int64_t sn_off;   // work (FP64): b squared row norms of [Y_B | Z_B] before nullification
  int64_t li_off;   // workc: inverses (and their transposes) of the 64 x 64 diagonal Cholesky
                    //   blocks, 2 sides x nblk x 2 x 64 x 64 (SIMT path); inverses of the
                    //   128 x 128 diagonal blocks, 2 sides x nblk128 x 128 x 128 (tensor-core path)
  int64_t pv_off;   // int32 work: b CPQR local permutation, then the first dependent step
  int64_t fi_off;   // int32 factor: R (r), S (kp), N (n), LU pivots (r)
  int64_t fd_off;   // double factor: T (kp x r), XRR (r x r), LU (r x r), LcT (r x (kp+n)), Uc (r x (kp+n)),
                    //   XRR^-1 (r x r)
  int64_t act_off;  // int32 active-list pool slot of the box
};

// Offsets inside a box's factor blocks.
__host__ __device__ inline int64_t fd_T(const BoxDesc& d) { return d.fd_off; }
__host__ __device__ inline int64_t fd_XRR(const BoxDesc& d) { return d.fd_off + (int64_t)d.kp * d.r; }
__host__ __device__ inline int64_t fd_LU(const BoxDesc& d) { return fd_XRR(d) + (int64_t)d.r * d.r; }
__host__ __device__ inline int64_t fd_LcT(const BoxDesc& d) { return fd_LU(d) + (int64_t)d.r * d.r; }
__host__ __device__ inline int64_t fd_Uc(const BoxDesc& d) { return fd_LcT(d) + (int64_t)d.r * (d.kp + d.n); }
__host__ __device__ inline int64_t fd_Xinv(const BoxDesc& d) { return fd_Uc(d) + (int64_t)d.r * (d.kp + d.n); }
__host__ __device__ inline int64_t fd_size(int64_t kp, int64_t r, int64_t n) {
  return kp * r + 3 * r * r + 2 * r * (kp + n);
}
__host__ __device__ inline int64_t fi_R(const BoxDesc& d) { return d.fi_off; }
__host__ __device__ inline int64_t fi_S(const BoxDesc& d) { return d.fi_off + d.r; }   // S then N: the "SN" list
__host__ __device__ inline int64_t fi_N(const BoxDesc& d) { return d.fi_off + d.r + d.kp; }
__host__ __device__ inline int64_t fi_piv(const BoxDesc& d) { return d.fi_off + d.r + d.kp + d.n; }
__host__ __device__ inline int64_t fi_size(int64_t kp, int64_t r, int64_t n) { return 2 * r + kp + n; }

// Segment copy of int32 lists (active-list assembly, neighbour gathers).
struct Seg {
  int64_t src, dst, len;
};

// ---- launch wrappers (defined in kernels.cu) --------------------------------
// Runs f once per device: kernel attributes (dynamic shared memory, cluster sizes) belong to a
// device's context, so a process that launches on several devices sets them on each.
struct PerDeviceOnce {
  static constexpr int kDevices = 64;
  std::once_flag flags[kDevices];
  template <class F>
  void operator()(F&& f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) {
      (void)cudaGetLastError();
      f();
      return;
    }
    std::call_once(flags[dev], f);
  }
};

struct Launch {
  cudaStream_t st;
  int64_t* counter;  // kernels launched (for stats), may be null
};

void launch_copy_segments(Launch L, const Seg* segs, int nseg, const int32_t* src, int32_t* dst);

// Gather rows: out[i][c] = in[rows[i]][c] for i < m, c < ncols.
void launch_gather_rows(Launch L, const double* in, int64_t ld_in, const int32_t* rows, int64_t m,
                        int64_t ncols, double* out, int64_t ld_out);

// Kernel-matrix product on the fly (tree order): out = shift*in + scale*K*in.
void launch_kernel_matvec(Launch L, int kind, const double* pts, int d, int64_t n, double shift,
                          double scale, const double* in, int64_t ld_in, double* out, int64_t ld_out,
                          int64_t ncols);
// Same, with the kernel part in FP32 (fp32 != 0) from in32, an FP32 copy of `in` (same layout);
// the identity term uses the FP64 `in`.
void launch_kernel_matvec_prec(Launch L, int kind, const double* pts, int d, int64_t n, double shift,
                               double scale, const double* in, int64_t ld_in, double* out, int64_t ld_out,
                               int64_t ncols, int fp32, const float* in32);
// FP32 copy; and TF32 hi/lo split of an n x s row-major block transposed to s x n planes with
// row pitch ldp (>= n).
void launch_to_f32(Launch L, const double* in, int64_t count, float* out);
void launch_split_transpose(Launch L, const double* in, int64_t n, int64_t s, float* hi, float* lo, int64_t ldp);

// Same product in 3xTF32 on the tensor cores (tcgen05, TMEM accumulators, TMA-fed B operand).
// p32: points in FP32 from launch_points_f32 (tc_points_len(n, d) floats); bhi/blo: TF32 hi/lo
// planes of the input columns (ncols x n, row pitch ldp = tc_plane_ld(n), 16-byte aligned).
// Columns [0, ncols0) come from in0 / go to out0, [ncols0, ncols) from in1 / to out1, all row-major
// with leading dimension ld.  Returns false when the tensor maps cannot be made (no launch);
// a bounded wait that expires records kDevTimeout in *err.
// FP64-accurate residual product in float-float arithmetic on the FP32 pipe (refinement):
// out = shift*in + scale*K*in, rows in tree order (ld_in, ld_out), any number of columns;
// scratch: ff_scratch_floats(n, d, ncols, split) floats.  split: point-range splits of the sums
// (partials added in a second kernel), 0 = enough CTAs for four per SM, else 1..16.
int64_t ff_scratch_floats(int64_t n, int d, int ncols, int split);
void launch_kernel_matvec_ff(Launch L, int kind, const double* pts, int d, int64_t n, double shift, double scale,
                             const double* in, int64_t ld_in, double* out, int64_t ld_out, int64_t ncols,
                             float* scratch, int split);

// The same product on the bf16 tensor cores by the Ozaki scheme (residual_oz.cu): a store of K's
// slices made once (oz_store_bytes bytes, launch_oz_prepare; its status word records a coincident
// point as kDevNonfinite and an expired wait as kDevTimeout), then any number of products, each with
// oz_scratch_bytes(n) bytes of scratch per call.  Rows in tree order; ncols any.
int64_t oz_store_bytes(int64_t n, int d);
int* oz_status_word(void* store, int64_t n, int d);
void launch_oz_prepare(Launch L, int kind, const double* pts, int d, int64_t n, void* store);
int64_t oz_scratch_bytes(int64_t n);
void launch_oz_matvec(Launch L, int64_t n, int d, const void* store, double shift, double scale, const double* in,
                      int64_t ld_in, double* out, int64_t ld_out, int64_t ncols, void* scratch);

int64_t tc_plane_ld(int64_t n);
int64_t tc_points_len(int64_t n, int d);
void launch_points_f32(Launch L, const double* pts, int64_t n, int d, float* out);
// variant: RSRS_SAMPLE_TILE_* (column tile x stages).
bool launch_kernel_matvec_tc(Launch L, int kind, const float* p32, int64_t n, double shift, double scale,
                             const double* in0, const double* in1, double* out0, double* out1, int64_t ld,
                             int64_t ncols0, int64_t ncols, const float* bhi, const float* blo, int64_t ldp, int* err,
                             int variant);


// Group-batched kernels (descriptors of one (level, colour) group).
struct GroupArgs {
  const BoxDesc* desc;  // device array, nbox entries
  int nbox;
  int64_t s;
  double* Y;
  double* Z;
  double* Om;
  double* Ps;
  double* work;
  void* workc;
  int32_t* iwork;
  double* fd;
  int32_t* fi;
  int32_t* act;
  int* err;
  int fp32;  // arithmetic of the Gram, Cholesky, projection, E/F and Schur kernels: FP32 (1) or FP64 (0)
};

void launch_gram(Launch L, const GroupArgs& g, int64_t items);                    // G = W W^T
void launch_chol_panel(Launch L, const GroupArgs& g, int panel);                   // diag block
void launch_chol_trsm(Launch L, const GroupArgs& g, int panel, int64_t items);     // below-diag panel
void launch_chol_update(Launch L, const GroupArgs& g, int panel, int64_t items);   // trailing update
void launch_gather_box(Launch L, const GroupArgs& g, int64_t items);               // M, W, V rows
void launch_m_finalize(Launch L, const GroupArgs& g, int64_t items);               // FP64 M for the CPQR
void launch_proj_nt(Launch L, const GroupArgs& g, int pass, int64_t items);        // X = M W^T
void launch_proj_solve(Launch L, const GroupArgs& g, int pass, int64_t items);     // X <- X G^-1
void launch_proj_acc(Launch L, const GroupArgs& g, int pass, int64_t items);       // M -= X W
// Mixed path (FP32 workspace): the group's Grams, least-squares right-hand sides and projection
// updates as 3xTF32 tcgen05 products (one launch each); the same results as launch_gram,
// launch_proj_nt and launch_proj_acc with CT = float, to FP32 accuracy.
void launch_gram_tc(Launch L, const GroupArgs& g, const std::vector<BoxDesc>& h);
void launch_proj_nt_tc(Launch L, const GroupArgs& g, int pass, const std::vector<BoxDesc>& h);
void launch_proj_acc_tc(Launch L, const GroupArgs& g, int pass, const std::vector<BoxDesc>& h);
// Tensor-core path of the Gram factorisation and the projection solve (FP32 workspace, Gram from
// launch_gram_tc): left-looking blocked Cholesky G = L L^T with 128-wide panels (diagonal blocks
// factored and inverted by one CTA each, column-block and panel products in 3xTF32), then U = L^-T by blocked
// substitution, stored in the upper block triangle of G (lower: L~_ik = L_ii^-1 L_ik).
// launch_solve_tc: X <- X G^-1 = (X U) U^T for the pass's coefficients (pass 1 also adds the
// result into the pass-0 coefficients).
void launch_chol_tc(Launch L, const GroupArgs& g, const std::vector<BoxDesc>& h);
void launch_solve_tc(Launch L, const GroupArgs& g, int pass, const std::vector<BoxDesc>& h);
// One CTA waits, through the tcgen05 kernels' bounded mbarrier wait, for a barrier that receives
// its arrival only when `arrive` is set; at most `polls` polls (clamped to 1..2^26).  An expired
// wait records kDevTimeout in *err (device int) and the kernel returns.
void launch_wait_selftest(Launch L, long long polls, int arrive, int* err);
// f = f64_bits_to_f32(x), g = f32_to_f64_exact(f), elementwise (device arrays of n)
void launch_convert_selftest(Launch L, const double* x, int64_t n, float* f, double* g);

// FP64 <-> FP32 conversions on the integer pipes, from the IEEE 754 binary64 / binary32 layouts
// (sign, biased exponent 11 / 8 bits, fraction 52 / 23 bits; biases 1023 / 127): this part's FP64
// pipe, which the hardware conversions use, is the mixed path's scarcest unit.  No FP64
// instruction appears in either routine (a rarely taken hardware-conversion branch would still be
// issued under predication).  They equal the hardware conversions bit for bit (NaN payloads aside).
// Round to nearest even of the binary64 value with high word hi and low word lo.
__device__ inline float f64_bits_to_f32(uint32_t hi, uint32_t lo) {
  const uint32_t sign = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {  // 897 <= e <= 1150: normal in binary32
    uint32_t r = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;  // a carry may reach the exponent
    return __uint_as_float(sign | r);
  }
  if (e >= 1151u) {  // beyond the binary32 range: infinity, or a quiet NaN
    const bool nan = e == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
    return __uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u));
  }
  if (e < 873u) return __uint_as_float(sign);  // below 2^-150: rounds to zero
  // 873 <= e <= 896: a binary32 subnormal (or the smallest normal after rounding), in units of
  // 2^-149: the 53-bit significand shifted right by 926 - e (30..53), rounded to nearest even
  const uint64_t m = ((uint64_t)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
  const uint32_t sh = 926u - e;
  uint64_t q = m >> sh;
  const uint64_t rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1u);
  q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  return __uint_as_float(sign | (uint32_t)q);
}
// The binary64 value of a binary32 (exact).
__device__ inline double f32_to_f64_exact(float f) {
  const uint32_t u = __float_as_uint(f), sign = u & 0x80000000u, mag = u & 0x7fffffffu;
  uint32_t hi, lo;
  if (mag - 0x00800000u < 0x7f000000u) {  // normal: widen the fraction, rebias the exponent by 896
    hi = sign | ((mag >> 3) + 0x38000000u);
    lo = mag << 29;
  } else if (mag >= 0x7f800000u) {  // infinity or NaN (payload kept)
    hi = sign | 0x7ff00000u | ((mag & 0x7fffffu) >> 3);
    lo = mag << 29;
  } else if (mag == 0u) {
    hi = sign;
    lo = 0u;
  } else {  // subnormal: normalise the leading one to bit 23, exponent 1 - sh in binary32 terms
    const uint32_t sh = (uint32_t)__clz(mag) - 8u;
    const uint32_t m = mag << sh;
    hi = sign | ((897u - sh) << 20) | ((m & 0x7fffffu) >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}



// Root blocks of a build: LU with partial pivoting in place in A (LAPACK interchange record in
// piv) and the explicit inverse in inv, all problems at once, FP64.
struct RootLU {
  double* A;
  int64_t n;
  int32_t* piv;
  double* inv;
};
void launch_root_lu_inverse(Launch L, const RootLU* R_dev, int nprob, int64_t max_n, int* err);

void launch_cpqr(Launch L, const GroupArgs& g, int max_b);                         // ID pivots + R
// FP32 CPQR on the compute-type sketch held in distributed shared memory (mixed path); false when
// the group's boxes do not fit a cluster of at most 16 CTAs (nothing launched).
// cluster: CTAs per box (0 = the fewest that hold the sketch; never fewer); threads: per CTA (0 = 1024).
bool launch_cpqr32(Launch L, const GroupArgs& g, int max_b, int cluster, int threads);
void launch_id_finish(Launch L, const GroupArgs& g, int max_b);                    // T, R/S/N lists
void launch_ef_update(Launch L, const GroupArgs& g, int64_t items);                // E, F on sketches
void launch_extract(Launch L, const GroupArgs& g, int64_t items);                  // X blocks
void launch_lu(Launch L, const GroupArgs& g);                                      // LU(X_RR)
void launch_lu_rhs(Launch L, const GroupArgs& g, int64_t items);                   // Lc, Uc
// Mixed path with tensor cores: X_RR^-1 alone by substitution, FP32 staging of it (and its
// transpose) and of the right-hand blocks, Uc and Lc^T as 3xTF32 products straight into the Schur
// update's FP32 operands, and those results written back to the factor in FP64.
void launch_lu_inv(Launch L, const GroupArgs& g, int64_t items);
// ... or, for groups whose boxes have r <= 224, X_RR^-1 by FP32 Gauss-Jordan in shared memory (one
// CTA per box; no LU needed), which also stages it: false (nothing launched) when max_r is larger.
bool launch_gj_inv32(Launch L, const GroupArgs& g, int max_r);
constexpr int kGaussJordanMaxR = 224;
void launch_lcuc_prep(Launch L, const GroupArgs& g, int64_t items, int with_inv);
void launch_lcuc_tc(Launch L, const GroupArgs& g, const std::vector<BoxDesc>& h);
void launch_lcuc_store(Launch L, const GroupArgs& g, int64_t items);
// L, U on the sketches; the mixed path first makes FP32 copies of LcT, Uc (unless yz_only: already
// there), Y_R, Z_R (prep_items blocks)
// tc: the group's boxes, to run the updates as 3xTF32 tensor-core products (mixed path only)
void launch_schur(Launch L, const GroupArgs& g, int64_t items, int64_t prep_items, int yz_only = 0,
                  const std::vector<BoxDesc>* tc = nullptr);
// The four block-elimination updates of the FP64 sketches as grouped 3xTF32 tcgen05 products (FP32
// operands staged by k_schur_prep / the Lc-Uc products, FP64 read-modify-write of the sketch rows).
void launch_schur_tc(Launch L, const GroupArgs& g, const std::vector<BoxDesc>& h);

// Number of 64-row x 64-col tiles for the group kernels (host-side planning).
constexpr int kT = 64;
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
// Tensor-core path: 128-wide Cholesky panels; the Gram's row pitch is padded to 4 elements so that
// its rows start 16-byte aligned for the operand loads.
constexpr int kTB = 128;
__host__ __device__ inline int64_t gram_ld(int64_t l) { return (l + 3) & ~(int64_t)3; }
// Compute-type elements of one box's diagonal-inverse area (both sides), either path.
inline int64_t li_elems(int64_t l) {
  const int64_t a = 2 * cdiv(l, kT) * 2 * kT * kT, b = 2 * cdiv(l, kTB) * kTB * kTB;
  return a > b ? a : b;
}
__host__ __device__ inline int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

// Solve / apply sweeps over one group (defined in solve.cu).
struct SweepArgs {
  const BoxDesc* desc;
  int nbox;
  const double* fd;
  const int32_t* fi;
  double* F;  // N x nrhs row-major, tree order of one problem
  int nrhs;
  int adjoint;
  int64_t row_base;  // index lists hold rows of the build's shared index space: row - row_base in F
  // FP32 sweeps (a mixed-precision factor's solve): FP32 copies of the blocks and of F; F32 set
  // selects them
  const float* fd32 = nullptr;
  float* F32 = nullptr;
};
// One phase of the fused solve sweeps (k_sweep_fused): a group's sweep product or the diagonal
// step over a range of boxes.  kind 0: C rows += alpha A^T B rows (A stored K x m, a thread per
// output row, 256 rows per item); 1: C rows += alpha A B rows (A row-major, 16 rows per item);
// 2: f_R <- X_RR^-1 f_R (solve = 1) or X_RR f_R, DC columns per item.  sync: a grid-wide barrier
// follows the phase (the next phase reads rows this one writes).
struct SweepPhase {
  const BoxDesc* desc;
  int nbox, kind, cset, mat, bset, solve, sync;
  double alpha;
  int64_t items;
  const int2* map;  // kinds 0 and 1: item -> (box, tile of the box); kind 2 maps by division
};
constexpr int kSweepFusedThreads = 256, kSweepFusedRowsT = 256, kSweepFusedRowsN = 16;
// Items of a sweep phase over boxes h (kind as above; nrhs for the diagonal step).
int64_t sweep_phase_items(const std::vector<BoxDesc>& h, int kind, int cset, int nrhs);
// Output-row tiles per box of a sweep product phase (kinds 0 and 1).
int64_t sweep_phase_tiles(const BoxDesc& d, int kind, int cset);
// The phases [ph, ph + nph) in one cooperative launch of persistent CTAs (all resident), with a
// bounded grid-wide barrier after each phase marked sync: bar holds the barrier's arrival counter
// and generation (zero on entry) and a status word (bar[2], kDevTimeout when a barrier wait gave
// up).  Returns false, launching nothing, when a cooperative launch is not possible.
bool launch_sweep_fused(Launch L, const SweepArgs& a, const SweepPhase* ph, int nph, int max_r, unsigned* bar);
// Two CTAs meet at the fused sweeps' grid barrier (with at most `polls` polls per wait), CTA 1 only
// when arrive is set; false when the cooperative launch is refused.
bool launch_grid_wait_selftest(Launch L, unsigned* bar, long long polls, int arrive);

// C rows += alpha * op(A) * B rows; row sets 0 = R, 1 = S, 2 = SN; matrices 0 = T, 1 = LcT, 2 = Uc.
void launch_sweep_op(Launch L, const SweepArgs& a, int cset, int mat, int trans, int bset, double alpha,
                     const std::vector<BoxDesc>& h);
// f_R <- X_RR^-1 f_R (solve, from the stored inverse) or X_RR f_R (apply), adjoint as requested.
void launch_sweep_diag(Launch L, const SweepArgs& a, int solve, int64_t items, int max_r);
void launch_dense_apply(Launch L, const double* A, int64_t n, const int32_t* rows, int64_t row_base, double* F,
                        int nrhs, int adjoint);
void launch_dense_apply(Launch L, const float* A, int64_t n, const int32_t* rows, int64_t row_base, float* F,
                        int nrhs, int adjoint);
void launch_to_f64(Launch L, const float* in, int64_t count, double* out);

// Item counts (host planning) matching the device decoding of each kernel.
int64_t items_gram(const std::vector<BoxDesc>& h);
int64_t items_chol_trsm(const std::vector<BoxDesc>& h, int p);
int64_t items_chol_update(const std::vector<BoxDesc>& h, int p);
int64_t items_gather(const std::vector<BoxDesc>& h);
int64_t items_finalize(const std::vector<BoxDesc>& h);
int64_t items_proj_nt(const std::vector<BoxDesc>& h);
int64_t items_proj_solve(const std::vector<BoxDesc>& h);
int64_t items_proj_acc(const std::vector<BoxDesc>& h, int64_t s);
int64_t items_ef(const std::vector<BoxDesc>& h, int64_t s);
int64_t items_extract(const std::vector<BoxDesc>& h);
int64_t items_lu_rhs(const std::vector<BoxDesc>& h);
int64_t items_schur(const std::vector<BoxDesc>& h, int64_t s);
int64_t items_schur_prep(const std::vector<BoxDesc>& h, int64_t s, int yz_only = 0);
int64_t items_lu_inv(const std::vector<BoxDesc>& h);
int64_t items_lcuc_prep(const std::vector<BoxDesc>& h, int with_inv);
int64_t items_lcuc_store(const std::vector<BoxDesc>& h);
int64_t items_diag(const std::vector<BoxDesc>& h, int nrhs);

// Root block (dense): LU in place with partial pivoting, single CTA.
void launch_dense_lu(Launch L, double* A, int64_t n, int32_t* piv, int* err);
void launch_dense_lu_solve(Launch L, const double* LU, const int32_t* piv, int64_t n,
                           const int32_t* rows, double* F, int nrhs, int adjoint);
// Explicit inverse of an LU-factored n x n matrix (one CTA per column).
void launch_dense_inverse(Launch L, const double* LU, const int32_t* piv, int64_t n, double* inv);

}  // namespace rsrs
