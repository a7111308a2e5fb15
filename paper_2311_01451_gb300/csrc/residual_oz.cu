// Refinement residual product out = shift*in + scale*K*in for the built-in kernels, to FP64-level
// accuracy on the bf16 tensor cores by the Ozaki scheme (Ozaki, Ogita, Oishi & Rump 2012; Ootomo,
// Ozaki & Yokota 2024): both operands are split into slices of small integers times powers of two,
// every product of slices is exact on the tensor cores, and the slice products are summed exactly in
// integers.
//
// Splitting.  Row i of K is scaled by sigma_i = 2^E_i >= 2 max_j |K_ij| and column c of the
// right-hand sides by tau_c = 2^F_c >= 2 max_j |X_jc|, so both scaled values lie in [-1/2, 1/2].  A
// value v in that range is written as sum_{t=0}^{9} a_t 2^(-7(t+1)) with integer digits from
// rounding to nearest: y = 128 v, a_t = rint(y), v <- y - a_t (exact steps); |a_t| <= 64.  K's
// entries are float-float (48 bits, as in the float-float residual), so its digits are those of the
// high part plus those of the low part (|a_t| <= 128); X's are taken from the FP64 value.  Ten
// digits resolve 2^-70 of the scale.
//
// Product.  K X / (sigma_i tau_c) = sum_{t,u} 2^(-7(t+u+2)) sum_j a_t(i,j) b_u(j,c).  Pairs with
// t + u <= 9 are kept (the products of 55 digit pairs per 16 points, issued as 10 MMAs); the dropped pairs and the digits beyond the
// tenth contribute below 2^-67 of sigma_i tau_c per point.  Since sigma_i <= 4 max_j |K_ij| and
// tau_c <= 4 max_j |X_jc|, that is below 2e-15 of sum_j |K_ij X_jc| for a row whose largest entry
// is 1e4 times its mean (a 3D point with a neighbour at 1e-4) and columns whose largest entry is 5
// times their mean.  All pairs of one level L = t + u accumulate into one FP32 TMEM accumulator (128
// rows x 16 columns); a product is at most 128 x 64 = 2^13, so over a block of 128 points a level
// holds an integer below 10 x 2^13 x 128 < 2^24 and FP32 accumulation is exact.  After every block
// the ten levels are read out and added into three int64 sums per output (levels 0-2, 3-5, 6-9 with
// their relative powers of two), exact for up to 2^16 blocks (8 million points); the final FP64
// value is formed once.
//
// Storage.  K's slices are made once per factor (k_oz_rowscale for E_i from the closest and the
// farthest point of each row, in float-float; k_oz_slices for the digits) and stored in the exact
// shared-memory image the MMA reads: per block of 128 rows and chunk of 32 points, ten 8 KB tiles
// (K-major rows of 32 bf16 values, 64-byte swizzle), 20 bytes per matrix entry.  A residual then
// streams them once from HBM (k_oz_mma: bulk copies into a two-stage ring, one thread issuing 20
// MMAs of N = 160 per 32 points, a warpgroup draining the accumulators into integers, two TMEM sets
// so that draining overlaps the next block's products), which makes it HBM-bound instead of bound
// by the float-float arithmetic of every kernel value and product.  Every wait is bounded: on
// expiry the kernel records kDevTimeout, waits (bounded) for its copies in flight, frees its TMEM and
// returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "ff.cuh"
#include "tc_common.cuh"

namespace rsrs {
namespace {
using namespace tc;

constexpr int OZ_S = 10;                            // digits (slices) per operand
constexpr int OZ_LV = 10;                           // levels t + u = 0 .. 9 kept
constexpr int OZ_M = 128;                           // rows per block (MMA M)
constexpr int OZ_KC = 32;                           // points per chunk: two bf16 K-steps of 16
constexpr int OZ_N = 16;                            // right-hand sides per pass (MMA N)
constexpr int OZ_BLK = 4;                           // chunks per exactly accumulated block (128 points)
constexpr int OZ_ATILE = OZ_M * OZ_KC * 2;          // 8192 bytes: one slice of one chunk of K
constexpr int OZ_BTILE = OZ_N * OZ_KC * 2;          // 1024 bytes: one slice of one chunk of X
constexpr int OZ_ACHUNK = OZ_S * OZ_ATILE;          // 81920
constexpr int OZ_BCHUNK = OZ_S * OZ_BTILE;          // 10240
constexpr int OZ_ZBYTES = (OZ_S - 1) * OZ_BTILE;    // 9216: nine zero blocks in front of X's digits
constexpr int OZ_STAGE = OZ_ACHUNK + OZ_ZBYTES + OZ_BCHUNK;  // 101376 = 99 KB: [K digits | zeros | X digits]
constexpr int OZ_NST = 2;                           // stages
constexpr int OZ_SMEM = OZ_NST * OZ_STAGE + 1024;   // + alignment slack
constexpr int OZ_NW = OZ_S * OZ_N;                  // 160: MMA N, all levels of one set
constexpr uint32_t OZ_TMEM = 512;                   // two accumulator sets of 10 levels x 16 columns
constexpr uint32_t OZ_SET = 256;                    // column offset of the second set
constexpr int OZ_THREADS = 160;                     // warps 0-3 drain, warp 4 issues
constexpr int OZ_PARTS = 3;                         // int64 sums per output
static_assert(OZ_LV * OZ_N <= (int)OZ_SET, "a set of levels fits in its TMEM columns");
static_assert(OZ_STAGE % 1024 == 0 && OZ_ACHUNK % 1024 == 0 && OZ_ZBYTES % 1024 == 0, "1024-byte alignment");
static_assert(OZ_NW % 16 == 0 && OZ_NW <= 256, "MMA N for M = 128");

// Byte offset of bf16 element e (0..31, the point inside the chunk) of row `row` of a tile with
// 64-byte rows and the 64-byte swizzle: the 16-byte chunk index (bits 4..5) is XOR-ed with bits
// 7..8 of the row's start, i.e. (row / 2) mod 4; 8-row atoms of 512 bytes.
__host__ __device__ inline uint32_t oz_off(int row, int e) {
  return (uint32_t)(row * 64 + ((((e >> 3) ^ ((row >> 1) & 3)) & 3) << 4) + (e & 7) * 2);
}

// Shared-memory descriptor of such a tile: start >> 4, leading byte offset 1 (unused by swizzled
// K-major layouts), stride 512 bytes between 8-row atoms, version 1, 64-byte swizzle (4).
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4..5 = 1), A and B BF16 (bits 7..9, 10..12 = 1),
// both K-major, N >> 3 at bits 17..22 (N = 160: the ten levels), M >> 4 at bits 24..28.
__device__ __forceinline__ uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_NW >> 3) << 17) | ((uint32_t)(OZ_M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global memory into
// this CTA's shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
      : "memory");
}

// The ten round-to-nearest base-128 digits of v (|v| <= 1/2), v = sum a_t 2^(-7(t+1)) + O(2^-71).
// Every step is exact in FP32: y = 128 v scales by a power of two; for |y| < 2^22, (y + 1.5 2^23)
// - 1.5 2^23 is y rounded to the nearest integer (ties to even) by the FP32 adder, and y minus it
// is y's fractional part.
__device__ __forceinline__ void digits(float v, float a[OZ_S]) {
  constexpr float kRound = 12582912.f;  // 1.5 * 2^23
#pragma unroll
  for (int t = 0; t < OZ_S; ++t) {
    const float y = v * 128.f;
    a[t] = __fsub_rn(__fadd_rn(y, kRound), kRound);
    v = y - a[t];
  }
}

// Digits of the low part l of a normalised float-float value h + l (|l| <= 2^-24 |h|, |h| <= 1/2
// after the row scale): |l| <= 2^-25, so 128^3 |l| <= 2^-4 and its first three digits are zero;
// the remainder after them is 2^21 l exactly.
__device__ __forceinline__ void digits_lo(float v, float a[OZ_S]) {
  constexpr float kRound = 12582912.f;  // 1.5 * 2^23
  a[0] = a[1] = a[2] = 0.f;
  v *= 0x1p21f;
#pragma unroll
  for (int t = 3; t < OZ_S; ++t) {
    const float y = v * 128.f;
    a[t] = __fsub_rn(__fadd_rn(y, kRound), kRound);
    v = y - a[t];
  }
}

// Points as three floats each (exact), padded with zeros to npad points.
__global__ void k_oz_f3(const double* __restrict__ pts, int64_t n, int d, int64_t npad, float3* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npad * d) return;
  out[e] = e < n * d ? f64_to_f3(pts[e]) : make_float3(0.f, 0.f, 0.f);
}

constexpr int RS_T = 128;  // rows (threads) per CTA of the row-scale pass
constexpr int RS_J = 64;   // points per shared-memory tile

// E_i with 2^E_i >= 2 max_{j != i} |K_ij|, from the closest and the farthest point of row i; |log r|
// <= max |log r^2| / 2 over the two extremes, 1/r <= 1/r_min.  r^2 of a pair from the high parts of
// the coordinates in FP32: each difference is then within 2^-24 (|x_i| + |x_j|) of the true one, so
// r^2 is within 2^-22 r S of the truth (S = sum over the axes of |x_i| + |x_j|), i.e. within 2^-10 of
// itself once r >= 2^-12 S; closer pairs take r^2 in float-float (accurate to 2^-46, the arithmetic
// of the kernel values).  The bounds carry the matching slack.  A row with a coincident point
// (r = 0) has no finite bound: err records kDevNonfinite and E_i = 0.
template <int KIND, int D>
__global__ void __launch_bounds__(RS_T) k_oz_rowscale(const float3* __restrict__ pff, int64_t n,
                                                        int* __restrict__ row_exp, int* err) {
  __shared__ float3 ps[RS_J][D];
  const int64_t i = (int64_t)blockIdx.x * RS_T + threadIdx.x;
  float3 pi[D];
#pragma unroll
  for (int k = 0; k < D; ++k) pi[k] = i < n ? pff[i * D + k] : make_float3(0.f, 0.f, 0.f);
  float rmin = INFINITY, rmax = 0.f;  // bracketing the true extremes from below / above
  for (int64_t j0 = 0; j0 < n; j0 += RS_J) {
    __syncthreads();
    for (int q = threadIdx.x; q < RS_J * D; q += RS_T) {
      const int64_t j = j0 + q / D;
      ps[q / D][q % D] = j < n ? pff[j * D + q % D] : make_float3(0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int jn = (int)imin64(RS_J, n - j0);
    for (int jj = 0; jj < jn; ++jj) {
      if (j0 + jj == i) continue;
      float r2 = 0.f, sc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float dd = pi[k].x - ps[jj][k].x;
        r2 = fmaf(dd, dd, r2);
        sc += fabsf(pi[k].x) + fabsf(ps[jj][k].x);
      }
      const float lim = 0x1p-12f * sc;
      if (r2 >= lim * lim) {
        rmin = fminf(rmin, r2 * (1.f - 0x1p-9f));
        rmax = fmaxf(rmax, r2 * (1.f + 0x1p-9f));
      } else {  // close pair: float-float r^2
        ffv q2 = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < D; ++k) q2 = ff_add_pos(q2, ff_sqr(coord_diff(pi[k], ps[jj][k])));
        rmin = fminf(rmin, q2.h * (1.f - 0x1p-22f));
        rmax = fmaxf(rmax, q2.h * (1.f + 0x1p-22f));
      }
    }
  }
  if (i >= n) return;
  double bound = 0.0;
  if (n > 1) {
    const double lo = (double)rmin, hi = (double)rmax;
    if (!(lo > 0.0) || !isfinite(hi)) {
      if (err) atomicCAS(err, 0, kDevNonfinite);
      row_exp[i] = 0;
      return;
    }
    bound = KIND == RSRS_OP_LOG2D ? 0.5 * fmax(fabs(log(lo)), fabs(log(hi))) : 1.0 / sqrt(lo);
  }
  int e = 0;
  if (bound > 0.0) {
    (void)frexp(2.0 * bound * (1.0 + 0x1p-20), &e);  // 2 bound (1 + 2^-20) < 2^e
  }
  row_exp[i] = e;
}

constexpr int SL_T = 256;  // threads of the slicing pass: two per row, 16 points each

// Digits of K_ij / sigma_i for row block I and chunks [c_begin, c_end), written as the MMA's
// shared-memory image: tile (I, ch, t) at store + ((I nch + ch) 10 + t) 8192 bytes.  K_ii = 0 and
// entries beyond n are zero.
template <int KIND, int D>
__global__ void __launch_bounds__(SL_T) k_oz_slices(const float3* __restrict__ pff, int64_t n, int64_t nch,
                                                     int64_t chunks_per_cta, const int* __restrict__ row_exp,
                                                     uint8_t* __restrict__ store, const LogTable tab) {
  __shared__ LogTable T;
  __shared__ float3 ps[OZ_KC][D];
  const int tid = threadIdx.x;
  for (int q = tid; q < kLogTab; q += SL_T) {
    T.ic[q] = tab.ic[q];
    T.lch[q] = tab.lch[q];
    T.lcl[q] = tab.lcl[q];
  }
  const int64_t I = blockIdx.y;
  const int row = tid >> 1, half = tid & 1;
  const int64_t gi = I * OZ_M + row;
  float3 pi[D];
#pragma unroll
  for (int k = 0; k < D; ++k) pi[k] = gi < n ? pff[gi * D + k] : make_float3(0.f, 0.f, 0.f);
  const int ex = gi < n ? row_exp[gi] : 0;
  const float inv = __int_as_float((127 - ex) << 23);  // 2^-E_i exactly (|E_i| < 127)
  const int sw = (row >> 1) & 3;
  const int64_t c_begin = (int64_t)blockIdx.x * chunks_per_cta, c_end = imin64(c_begin + chunks_per_cta, nch);
  for (int64_t ch = c_begin; ch < c_end; ++ch) {
    __syncthreads();
    for (int q = tid; q < OZ_KC * D; q += SL_T) {
      const int64_t j = ch * OZ_KC + q / D;
      ps[q / D][q % D] = j < n ? pff[j * D + q % D] : make_float3(0.f, 0.f, 0.f);
    }
    __syncthreads();
    uint8_t* base = store + (size_t)(I * nch + ch) * OZ_ACHUNK;
#pragma unroll 1
    for (int c8 = 0; c8 < 2; ++c8) {  // the thread's two 16-byte chunks of 8 points
      const int e0 = half * 16 + c8 * 8;
      uint32_t w[OZ_S][4];
#pragma unroll
      for (int pr = 0; pr < 4; ++pr) {
        float dg[2][OZ_S];
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          const int e = e0 + 2 * pr + q2;
          const int64_t gj = ch * OZ_KC + e;
          ffv r2 = {0.f, 0.f};
#pragma unroll
          for (int k = 0; k < D; ++k) r2 = ff_add_pos(r2, ff_sqr(coord_diff(pi[k], ps[e][k])));
          ffv kv;
          if (KIND == RSRS_OP_LOG2D) {
            kv = ff_log(r2, T);
            kv.h *= 0.5f;
            kv.l *= 0.5f;
          } else {
            kv = ff_rsqrt(r2);
          }
          if (gi >= n || gj >= n || gj == gi) kv = {0.f, 0.f};
          float dh[OZ_S], dl[OZ_S];
          digits(kv.h * inv, dh);
          digits_lo(kv.l * inv, dl);
#pragma unroll
          for (int t = 0; t < OZ_S; ++t) dg[q2][t] = t < 3 ? dh[t] : dh[t] + dl[t];
        }
#pragma unroll
        for (int t = 0; t < OZ_S; ++t) {
          const __nv_bfloat162 b2 = __floats2bfloat162_rn(dg[0][t], dg[1][t]);  // .x: even point (low half)
          w[t][pr] = *reinterpret_cast<const uint32_t*>(&b2);
        }
      }
      const uint32_t off = (uint32_t)(row * 64 + ((((e0 >> 3) ^ sw) & 3) << 4));
#pragma unroll
      for (int t = 0; t < OZ_S; ++t)
        *reinterpret_cast<uint4*>(base + (size_t)t * OZ_ATILE + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
  }
}

// F_c with 2^F_c >= 2 max_j |X_jc| for column c0 + c of in (row-major, ld_in); 0 for a zero column.
// One CTA per column.
__global__ void __launch_bounds__(256) k_oz_colscale(const double* __restrict__ in, int64_t n, int64_t ld_in,
                                                      int64_t c0, int nsrc, int* __restrict__ col_exp) {
  __shared__ double red[8];
  const int c = blockIdx.x;
  double m = 0.0;
  if (c < nsrc)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) m = fmax(m, fabs(in[j * ld_in + c0 + c]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
    int e = 0;
    if (m > 0.0) (void)frexp(2.0 * m * (1.0 + 0x1p-40), &e);
    col_exp[c] = e;
  }
}

// Digits of X_jc / tau_c for columns c0 .. c0 + 15 (zero beyond nsrc and beyond n), as the MMA's
// shared-memory image of B: chunk ch at xs + ch 10240 bytes, digit u of column c in row 16 u + c
// (block u at byte 1024 u), element j - 32 ch.
// FP64 steps: 128 v and v - rint(v) are exact.
__global__ void k_oz_xslices(const double* __restrict__ in, int64_t n, int64_t ld_in, int64_t c0, int nsrc,
                             int64_t nch, const int* __restrict__ col_exp, uint8_t* __restrict__ xs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (point, column) pairs
  if (e >= nch * OZ_KC * OZ_N) return;
  const int64_t j = e / OZ_N;
  const int c = (int)(e % OZ_N);
  double v = 0.0;
  if (j < n && c < nsrc) v = ldexp(in[j * ld_in + c0 + c], -col_exp[c]);
  const int64_t ch = j / OZ_KC;
  const int jj = (int)(j % OZ_KC);
  uint8_t* base = xs + (size_t)ch * OZ_BCHUNK + oz_off(c, jj);
#pragma unroll
  for (int u = 0; u < OZ_S; ++u) {
    const double y = v * 128.0;
    const double a = rint(y);
    v = y - a;
    *reinterpret_cast<__nv_bfloat16*>(base + (size_t)u * OZ_BTILE) = __float2bfloat16_rn((float)a);
  }
}

// The product for row block blockIdx.x, point range of split blockIdx.y, right-hand-side group of
// xs: ten level sums per output folded exactly into three int64, written to part[(ks n + i) 48 + ...].
// A stage holds one chunk: K's ten digit tiles, then nine zero blocks of 16 rows and X's ten digit
// blocks (row 16 u + c = digit u of column c).  For K digit t one MMA with N = 160 reads the ten
// blocks starting at block 9 - t of [zeros | X digits], so output block L receives a_t b_(L-t)
// (nothing for L < t): all pairs t + u <= 9 land in their level's accumulator, 20 MMAs per chunk.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_mma(const uint8_t* __restrict__ store, const uint8_t* __restrict__ xs, int64_t n, int64_t nch,
             int64_t chunks_per_split, long long* __restrict__ part, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[OZ_NST], empty[OZ_NST], accf[2], accfree[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_timeout;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t I = blockIdx.x, ks = blockIdx.y;
  const int64_t cb = ks * chunks_per_split, ce = imin64(cb + chunks_per_split, nch);
  const int64_t nc = ce > cb ? ce - cb : 0;
  const int64_t nblk = (nc + OZ_BLK - 1) / OZ_BLK;
  if (tid == 0) {
    s_timeout = 0;
    for (int st = 0; st < OZ_NST; ++st) {
      bar_init(smem_u32(&full[st]), 1);
      bar_init(smem_u32(&empty[st]), 1);
    }
    for (int p = 0; p < 2; ++p) {
      bar_init(smem_u32(&accf[p]), 1);
      bar_init(smem_u32(&accfree[p]), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the zero blocks of both stages (never written by a copy)
  for (int e = tid; e < OZ_NST * OZ_ZBYTES / 16; e += OZ_THREADS) {
    const int st = e / (OZ_ZBYTES / 16), o = e % (OZ_ZBYTES / 16);
    *reinterpret_cast<uint4*>(smem + st * OZ_STAGE + OZ_ACHUNK + o * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_proxy_async();
  if (warp == 0) tmem_alloc(&s_tmem, OZ_TMEM);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 4) {
    if (lane == 0) {
      // ---- copies and MMAs ----
      const uint32_t idesc = oz_idesc();
      bool armed[OZ_NST] = {};
      uint32_t armed_par[OZ_NST] = {};
      bool ok = true;
      auto arm = [&](int64_t c) {
        const int st = (int)(c % OZ_NST);
        unsigned char* sa = smem + st * OZ_STAGE;
        const uint32_t bar = smem_u32(&full[st]);
        bar_expect_tx(bar, (uint32_t)(OZ_ACHUNK + OZ_BCHUNK));
        const uint8_t* a = store + (size_t)(I * nch + cb + c) * OZ_ACHUNK;
#pragma unroll 1
        for (int t = 0; t < OZ_S; ++t) bulk_g2s(smem_u32(sa + t * OZ_ATILE), a + (size_t)t * OZ_ATILE, OZ_ATILE, bar);
        bulk_g2s(smem_u32(sa + OZ_ACHUNK + OZ_ZBYTES), xs + (size_t)(cb + c) * OZ_BCHUNK, OZ_BCHUNK, bar);
        armed[st] = true;
        armed_par[st] = (uint32_t)((c / OZ_NST) & 1);
      };
      for (int64_t c = 0; c < OZ_NST && c < nc; ++c) arm(c);
      for (int64_t c = 0; c < nc && ok; ++c) {
        const int st = (int)(c % OZ_NST);
        const uint32_t par = (uint32_t)((c / OZ_NST) & 1);
        const int64_t blk = c / OZ_BLK;
        const int p = (int)(blk & 1);
        const bool first = (c % OZ_BLK) == 0;
        // the accumulator set of block blk - 2 must have been read out
        if (first && blk >= 2 && !bar_wait(smem_u32(&accfree[p]), (uint32_t)(((blk - 2) / 2) & 1))) ok = false;
        if (ok && !bar_wait(smem_u32(&full[st]), par)) ok = false;
        if (!ok) break;
        armed[st] = false;
        fence_after();
        const uint32_t a0 = smem_u32(smem + st * OZ_STAGE), z0 = a0 + OZ_ACHUNK;
        const uint32_t acc = tmem + (uint32_t)p * OZ_SET;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {  // K = 16 bf16 values (32 bytes) per instruction
#pragma unroll
          for (int t = 0; t < OZ_S; ++t)
            mma_bf16(acc, oz_desc(a0 + t * OZ_ATILE + kk * 32), oz_desc(z0 + (OZ_S - 1 - t) * OZ_BTILE + kk * 32),
                     idesc, (first && kk == 0 && t == 0) ? 0u : 1u);
        }
        mma_commit(smem_u32(&empty[st]));
        if ((c % OZ_BLK) == OZ_BLK - 1 || c == nc - 1) mma_commit(smem_u32(&accf[p]));
        if (c + OZ_NST < nc) {
          if (!bar_wait(smem_u32(&empty[st]), par)) {
            ok = false;
            break;
          }
          arm(c + OZ_NST);
        }
      }
      if (!ok) {
        s_timeout = 1;
        for (int st = 0; st < OZ_NST; ++st)  // copies still in flight must land before the CTA exits
          if (armed[st]) bar_wait(smem_u32(&full[st]), armed_par[st]);
      }
    }
    __syncwarp();
  } else {
    // ---- drain: thread = row 32 warp + lane; exact level sums into three int64 per column ----
    long long H[OZ_N], Mi[OZ_N], Lo[OZ_N];
#pragma unroll
    for (int c = 0; c < OZ_N; ++c) H[c] = Mi[c] = Lo[c] = 0;
    bool ok = true;
    for (int64_t blk = 0; blk < nblk; ++blk) {
      const int p = (int)(blk & 1);
      if (!bar_wait(smem_u32(&accf[p]), (uint32_t)((blk / 2) & 1))) {
        ok = false;
        break;
      }
      fence_after();
#pragma unroll
      for (int L = 0; L < OZ_LV; ++L) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)p * OZ_SET + (uint32_t)L * OZ_N, r);
        const long long w = 1ll << (7 * ((L < 3 ? 2 : L < 6 ? 5 : 9) - L));  // weight inside its group
#pragma unroll
        for (int c = 0; c < OZ_N; ++c) {
          const long long v = (long long)__float2int_rn(__uint_as_float(r[c])) * w;
          if (L < 3) H[c] += v;
          else if (L < 6) Mi[c] += v;
          else Lo[c] += v;
        }
      }
      fence_before();
      bar_arrive(smem_u32(&accfree[p]));
    }
    if (!ok) s_timeout = 1;
    const int64_t i = I * OZ_M + tid;
    if (i < n) {
      long long* o = part + ((size_t)ks * n + i) * (OZ_PARTS * OZ_N);
#pragma unroll
      for (int c = 0; c < OZ_N; ++c) {
        o[c] = H[c];
        o[OZ_N + c] = Mi[c];
        o[2 * OZ_N + c] = Lo[c];
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, OZ_TMEM);
  if (tid == 0 && s_timeout && err) atomicCAS(err, 0, kDevTimeout);
}

// out = shift in + scale 2^(E_i + F_c) (H 2^-28 + M 2^-49 + Lo 2^-77), the int64 sums over the
// splits added exactly first (group g with top level h_g is in units of 2^-7(h_g + 2)).
__global__ void k_oz_finish(const long long* __restrict__ part, int ksplit, int64_t n, const int* __restrict__ row_exp,
                            const int* __restrict__ col_exp, int64_t c0, int nsrc, double shift, double scale,
                            const double* __restrict__ in, int64_t ld_in, double* __restrict__ out, int64_t ld_out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nsrc) return;
  const int64_t i = e / nsrc;
  const int c = (int)(e % nsrc);
  long long h = 0, m = 0, l = 0;
  for (int k = 0; k < ksplit; ++k) {
    const long long* o = part + ((size_t)k * n + i) * (OZ_PARTS * OZ_N);
    h += o[c];
    m += o[OZ_N + c];
    l += o[2 * OZ_N + c];
  }
  const double v = ((double)h * 0x1p-28 + (double)m * 0x1p-49) + (double)l * 0x1p-77;
  const double kx = ldexp(v, row_exp[i] + col_exp[c]);
  out[i * ld_out + c0 + c] = shift * in[i * ld_in + c0 + c] + scale * kx;
}

}  // namespace
}  // namespace rsrs

namespace rsrs {
namespace {

int64_t oz_nrb(int64_t n) { return (n + OZ_M - 1) / OZ_M; }
int64_t oz_nch(int64_t n) { return (n + OZ_KC - 1) / OZ_KC; }
size_t oz_align(size_t x) { return (x + 255) & ~(size_t)255; }

// Store layout: [K slices | E_i (n int) | points as float3 (n d) | status word].
size_t oz_slices_bytes(int64_t n) { return oz_align((size_t)oz_nrb(n) * oz_nch(n) * OZ_ACHUNK); }
size_t oz_rowexp_off(int64_t n) { return oz_slices_bytes(n); }
size_t oz_pff_off(int64_t n) { return oz_rowexp_off(n) + oz_align((size_t)n * sizeof(int)); }
size_t oz_err_off(int64_t n, int d) { return oz_pff_off(n) + oz_align((size_t)n * d * sizeof(float3)); }

// Point-range splits: enough CTAs (one per SM at a time) to fill the GPU in near-whole waves.
int oz_splits(int64_t n) {
  const int64_t nrb = oz_nrb(n), nblk = (oz_nch(n) + OZ_BLK - 1) / OZ_BLK;
  int best = 1;
  double best_eff = 0.0;
  for (int ks = 1; ks <= 8 && ks <= nblk; ++ks) {
    const int64_t ctas = nrb * ks, waves = (ctas + 151) / 152;
    const double eff = (double)ctas / (double)(waves * 152);
    if (ctas >= 2 * 152 && eff >= 0.9) return ks;
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = ks;
    }
  }
  return best;
}

// Scratch layout per residual: [X slices | F_c (16 int) | int64 partial sums].
size_t oz_xs_bytes(int64_t n) { return oz_align((size_t)oz_nch(n) * OZ_BCHUNK); }

}  // namespace

int64_t oz_store_bytes(int64_t n, int d) { return (int64_t)(oz_err_off(n, d) + 256); }

int* oz_status_word(void* store, int64_t n, int d) {
  return reinterpret_cast<int*>(static_cast<uint8_t*>(store) + oz_err_off(n, d));
}

void launch_oz_prepare(Launch L, int kind, const double* pts, int d, int64_t n, void* store) {
  if (n <= 0) return;
  uint8_t* base = static_cast<uint8_t*>(store);
  int* row_exp = reinterpret_cast<int*>(base + oz_rowexp_off(n));
  float3* pff = reinterpret_cast<float3*>(base + oz_pff_off(n));
  int* err = oz_status_word(store, n, d);
  cudaMemsetAsync(err, 0, sizeof(int), L.st);
  k_oz_f3<<<(unsigned)cdiv(n * d, 256), 256, 0, L.st>>>(pts, n, d, n, pff);
  const int64_t nrb = oz_nrb(n), nch = oz_nch(n);
  // slices: about 16 CTAs of 256 threads per SM in total, each a run of chunks of one row block
  const int64_t per = std::max<int64_t>(1, cdiv(nch * nrb, (int64_t)152 * 16));
  const dim3 sgrid((unsigned)cdiv(nch, per), (unsigned)nrb);
  const LogTable& tab = log_table();
  if (kind == RSRS_OP_LOG2D) {
    k_oz_rowscale<RSRS_OP_LOG2D, 2><<<(unsigned)cdiv(n, RS_T), RS_T, 0, L.st>>>(pff, n, row_exp, err);
    k_oz_slices<RSRS_OP_LOG2D, 2><<<sgrid, SL_T, 0, L.st>>>(pff, n, nch, per, row_exp, base, tab);
  } else {
    k_oz_rowscale<RSRS_OP_INVR3D, 3><<<(unsigned)cdiv(n, RS_T), RS_T, 0, L.st>>>(pff, n, row_exp, err);
    k_oz_slices<RSRS_OP_INVR3D, 3><<<sgrid, SL_T, 0, L.st>>>(pff, n, nch, per, row_exp, base, tab);
  }
  if (L.counter) *L.counter += 3;
}

int64_t oz_scratch_bytes(int64_t n) {
  return (int64_t)(oz_xs_bytes(n) + 256 + oz_align((size_t)oz_splits(n) * n * OZ_PARTS * OZ_N * sizeof(long long)));
}

void launch_oz_matvec(Launch L, int64_t n, int d, const void* store, double shift, double scale, const double* in,
                      int64_t ld_in, double* out, int64_t ld_out, int64_t ncols, void* scratch) {
  if (n <= 0 || ncols <= 0) return;
  static PerDeviceOnce attr;
  attr([] { cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM); });
  const uint8_t* base = static_cast<const uint8_t*>(store);
  const int* row_exp = reinterpret_cast<const int*>(base + oz_rowexp_off(n));
  int* err = oz_status_word(const_cast<void*>(store), n, d);
  uint8_t* xs = static_cast<uint8_t*>(scratch);
  int* col_exp = reinterpret_cast<int*>(xs + oz_xs_bytes(n));
  long long* part = reinterpret_cast<long long*>(xs + oz_xs_bytes(n) + 256);
  const int64_t nrb = oz_nrb(n), nch = oz_nch(n);
  const int ks = oz_splits(n);
  const int64_t per = cdiv(cdiv(nch, ks), (int64_t)OZ_BLK) * OZ_BLK;  // chunks per split, whole blocks
  for (int64_t c0 = 0; c0 < ncols; c0 += OZ_N) {
    const int nsrc = (int)imin64(OZ_N, ncols - c0);
    k_oz_colscale<<<OZ_N, 256, 0, L.st>>>(in, n, ld_in, c0, nsrc, col_exp);
    k_oz_xslices<<<(unsigned)cdiv(nch * OZ_KC * OZ_N, 256), 256, 0, L.st>>>(in, n, ld_in, c0, nsrc, nch, col_exp, xs);
    k_oz_mma<<<dim3((unsigned)nrb, (unsigned)ks), OZ_THREADS, OZ_SMEM, L.st>>>(base, xs, n, nch, per, part, err);
    k_oz_finish<<<(unsigned)cdiv(n * nsrc, 256), 256, 0, L.st>>>(part, ks, n, row_exp, col_exp, c0, nsrc, shift, scale,
                                                                  in, ld_in, out, ld_out);
    if (L.counter) *L.counter += 4;
  }
}

}  // namespace rsrs
