// Mixed-precision sampling product on the 5th-generation tensor cores (tcgen05, TMEM accumulators):
//   out = shift * in + scale * K * in,   K_ij = log|x_i - x_j| (2D) or 1/|x_i - x_j| (3D), K_ii = 0,
// in 3xTF32: every FP32 operand value v is split into hi = v with the 13 low mantissa bits cleared
// (exact in TF32) and lo = v - hi, and D += A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 in
// tensor memory.  The split follows Ootomo & Yokota (2022); products are then accurate to about
// 2^-21 relative, the level of the FP32 arithmetic of the rest of the mixed path.
//
// Tile: RH accumulators of 128 rows (TMEM lanes) x TN <= 256 columns (TMEM columns) per CTA, i.e.
// RH*128 rows that share every B stage; KT points j per stage.
//   A_hi, A_lo: K(x_i, x_j) for the RH*128 rows, generated by 16 producer warps (K-major rows of KT
//               TF32 values: 128-byte rows with the 128-byte swizzle for KT = 32, 64-byte rows
//               with the 64-byte swizzle for KT = 16; the 128-row halves are consecutive atoms);
//   B_hi, B_lo: in[j][c] for the tile's columns, from hi/lo planes split and transposed once
//               before the product (FP64 -> FP32 conversion runs at FP64 rate on this part, so it
//               must not sit in the inner loop), fetched by one TMA copy per plane and stage
//               straight into the same swizzled layout (the tensor map's swizzle is the canonical
//               K-major one).  Each CTA loads its own B tile from this GPU's memory; with RH = 2
//               one B tile feeds 256 rows, which halves the B traffic per product.
// A seventeenth warp issues, from one thread, the TMA copies and the KT/8 K-steps x 3 x RH products
// per stage.  NST stages (default: RH = 2, TN = 256, KT = 16, three stages); per stage three
// mbarriers: A written (512 arrivals), B landed (TMA transaction bytes) and stage free
// (tcgen05.commit of the products that read it).  The copies of chunk c + NST - 1 are armed once
// the products of chunk c - 1 are done, so the B tiles arrive NST - 1 products ahead.  Chunks that
// overlap the row tile (K_ii = 0) or hold the last points test indices; the others do not.  Every
// wait is bounded: on expiry the kernel records kDevTimeout, waits (bounded) for its own copies
// still in flight, frees its TMEM and returns.
#include <cuda.h>

#include <cstdint>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace rsrs {
namespace {

constexpr int TM = 128;
constexpr int TK = 32;                                    // point padding of p32 (a multiple of every KT)
constexpr int NPROD = 512;                                // producer threads (warps 0..15)
// K-major operand tiles with KT TF32 values (4 KT bytes) per row: KT = 32 uses the 128-byte swizzle
// (8-row atoms of 1024 bytes), KT = 16 the 64-byte swizzle (8-row atoms of 512 bytes).  In both, the
// 16-byte chunk index of a row is XOR-ed with address bits 7.. of the row start, which is what
// the TMA writes with the matching tensor-map swizzle and the MMA reads with the matching
// descriptor layout.
template <int KT>
struct Lay;
template <>
struct Lay<32> {
  static constexpr uint32_t SBO = 1024, MODE = 2;  // descriptor layout: 128-byte swizzle
  static constexpr CUtensorMapSwizzle TMA_SWIZZLE = CU_TENSOR_MAP_SWIZZLE_128B;
  __device__ static uint32_t off(int row, int k) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + (((k >> 2) ^ (row & 7)) << 4) + (k & 3) * 4);
  }
};
template <>
struct Lay<16> {
  static constexpr uint32_t SBO = 512, MODE = 4;  // descriptor layout: 64-byte swizzle
  static constexpr CUtensorMapSwizzle TMA_SWIZZLE = CU_TENSOR_MAP_SWIZZLE_64B;
  __device__ static uint32_t off(int row, int k) {
    return (uint32_t)(row * 64 + (((k >> 2) ^ ((row >> 1) & 3)) << 4) + (k & 3) * 4);
  }
};
// One variant: column tile TN, points per stage KT, pipeline depth NST and RH accumulators of 128
// rows: stages of A_hi, A_lo (RH*128 x KT) and B_hi, B_lo (TN x KT); each accumulator takes the next
// power of two >= TN TMEM columns.
template <int TN, int KT, int NST, int RH>
struct Tile {
  static constexpr int MR = RH * TM;  // rows per CTA
  static constexpr int AH_BYTES = TM * KT * 4;  // one 128-row half of one A plane
  static constexpr int A_BYTES = RH * AH_BYTES;
  static constexpr int B_BYTES = TN * KT * 4;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int SMEM_BYTES = NST * STAGE_BYTES + 1024;  // + alignment slack
  static constexpr uint32_t ACC_COLS = TN <= 32 ? 32 : TN <= 64 ? 64 : TN <= 128 ? 128 : 256;
  static constexpr uint32_t TMEM_COLS = RH * ACC_COLS;
  static constexpr int VPT = MR * KT / 512;  // kernel values per producer thread and stage
  static_assert(TN % 32 == 0 && TN >= 32 && TN <= 256, "MMA N and the TMA box height");
  static_assert(KT == 16 || KT == 32, "K-slice of one stage");
  static_assert(RH == 1 || RH == 2, "one or two 128-row accumulators");
  static_assert(TMEM_COLS <= 512, "tensor memory columns");
  static_assert(VPT % 4 == 0 && KT % VPT == 0, "producer values per thread");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
};
constexpr int NTHREADS = NPROD + 32;                      // + the TMA / MMA warp
constexpr long long WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address >> 4 (bits 0..13), leading byte offset (bits
// 16..29, not used by swizzled K-major layouts), stride byte offset >> 4 between 8-row atoms
// (bits 32..45), descriptor version 1 (bits 46..47), base offset 0, layout type (bits 61..63).
template <int KT>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(Lay<KT>::SBO >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)Lay<KT>::MODE << 61;
  return d;
}

// Instruction descriptor, kind::tf32: D FP32 (bits 4..5 = 1), A and B TF32 (bits 7..9, 10..12 = 2),
// both K-major, N >> 3 at bits 17..22, M >> 4 at bits 24..28.
__device__ __forceinline__ uint32_t idesc_tf32(int nmma) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void bar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the completion of the mbarrier phase with the given parity; false on expiry.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 2D tiled TMA load of box (KT points x TN columns) at (x = first point, y = first column) into
// this CTA's shared memory, completing on this CTA's mbarrier.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

template <int KIND>
__device__ __forceinline__ float kvalf_tc(float r2) {
  if (KIND == RSRS_OP_LOG2D) return 0.5f * __logf(r2);
  return rsqrtf(r2);
}

// p32: the points in FP32, n rounded up to a multiple of TK and zero padded (so that every
// producer load of a chunk stays in bounds).  Columns [0, ncols0) read in0 / write out0, columns
// [ncols0, ncols) read in1 / write out1 (column c - ncols0); all four are row-major with ld.
template <int KIND, int D, int TN, int KT, int NST, int RH>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_kmv_tc(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
             const float* __restrict__ p32, int64_t n, double shift, double scale, const double* __restrict__ in0,
             const double* __restrict__ in1, double* __restrict__ out0, double* __restrict__ out1, int64_t ld,
             int64_t ncols0, int64_t ncols, int* err) {
  using C = Tile<TN, KT, NST, RH>;
  constexpr int MR = C::MR, AH_BYTES = C::AH_BYTES, A_BYTES = C::A_BYTES, B_BYTES = C::B_BYTES;
  constexpr int STAGE_BYTES = C::STAGE_BYTES;
  constexpr int VPT = C::VPT;       // kernel values per producer thread and stage
  constexpr int TPR = KT / VPT;     // producer threads per row
  constexpr uint32_t TMEM_COLS = C::TMEM_COLS, ACC_COLS = C::ACC_COLS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_a[NST], full_b[NST], empty[NST];
  __shared__ uint32_t s_tmem;
  __shared__ int s_timeout;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = (int64_t)blockIdx.x * MR, c0 = (int64_t)blockIdx.y * TN;
  const int ntile = (int)(ncols - c0 < TN ? ncols - c0 : TN);
  const int nmma = (ntile + 15) & ~15;  // MMA N: a multiple of 16 in [16, TN]
  const int64_t nchunk = (n + KT - 1) / KT;

  if (tid == 0) {
    s_timeout = 0;
    for (int s = 0; s < NST; ++s) {
      bar_init(smem_u32(&full_a[s]), NPROD);
      bar_init(smem_u32(&full_b[s]), 1);
      bar_init(smem_u32(&empty[s]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp < NPROD / 32) {
    // ---- producers: kernel values of row arow, points akq..akq+VPT-1 of each chunk; the points of
    // the next chunk are loaded while this chunk's values are computed ----
    const int arow = tid / TPR, akq = (tid % TPR) * VPT;
    const int64_t gi = i0 + arow;
    const int gi32 = (int)gi;
    float pi[D];
#pragma unroll
    for (int k = 0; k < D; ++k) pi[k] = (gi < n) ? p32[gi * D + k] : 0.f;
    float pj[VPT * D], pn[VPT * D];
    auto load_pts = [&](int64_t ch, float* dst) {
      const float4* src = reinterpret_cast<const float4*>(p32 + (ch * KT + akq) * D);
#pragma unroll
      for (int q = 0; q < VPT * D / 4; ++q) {
        const float4 v = __ldg(src + q);
        dst[4 * q] = v.x;
        dst[4 * q + 1] = v.y;
        dst[4 * q + 2] = v.z;
        dst[4 * q + 3] = v.w;
      }
    };
    if (nchunk > 0) load_pts(0, pj);
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      const int st = (int)(ch % NST);
      const int64_t u = ch / NST;
      unsigned char* Ahi = smem + st * STAGE_BYTES;
      unsigned char* Alo = Ahi + A_BYTES;
      const int64_t j0 = ch * KT + akq;
      if (ch + 1 < nchunk) load_pts(ch + 1, pn);
      // the products of chunk ch - NST must be done with this stage
      if (ch >= NST && !bar_wait(smem_u32(&empty[st]), (uint32_t)((u - 1) & 1))) s_timeout = 1;
      // K_ii = 0 and the zero padding beyond n only concern the chunks that overlap the row tile
      // or hold the last points (block-uniform); rows beyond n are never stored, so their values
      // need no check
      const int64_t jc = ch * KT;
      const bool check = (jc < i0 + MR && jc + KT > i0) || jc + KT > n;
      auto gen = [&](auto check_tag) {
        constexpr bool CHECK = decltype(check_tag)::value;
#pragma unroll
        for (int q = 0; q < VPT / 4; ++q) {
          float hv[4], lv[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int kk = q * 4 + w;
            float r2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              const float dd = pi[k] - pj[kk * D + k];
              r2 = fmaf(dd, dd, r2);
            }
            float v = kvalf_tc<KIND>(r2);
            if (CHECK) {
              const int gj = (int)j0 + kk;
              if (gj >= (int)n || gj == gi32) v = 0.f;
            }
            hv[w] = tf32_hi(v);
            lv[w] = v - hv[w];
          }
          // rows 128.. of a stage are the next 128-row atoms of the same swizzled layout
          const uint32_t off = Lay<KT>::off(arow, akq + q * 4);
          *reinterpret_cast<float4*>(Ahi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<float4*>(Alo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
        }
      };
      if (check) gen(std::true_type{});
      else gen(std::false_type{});
      // generic-proxy writes must be visible to the tensor cores (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_arrive(smem_u32(&full_a[st]));
#pragma unroll
      for (int q = 0; q < VPT * D; ++q) pj[q] = pn[q];
    }
  } else if (lane == 0) {
    // ---- TMA + MMA issue ----
    const uint32_t idesc = idesc_tf32(nmma);
    bool armed[NST];
    uint32_t armed_par[NST];
#pragma unroll
    for (int q = 0; q < NST; ++q) {
      armed[q] = false;
      armed_par[q] = 0u;
    }
    bool ok = true;
    auto arm = [&](int64_t ch) {
      const int st = (int)(ch % NST);
      unsigned char* Bhi = smem + st * STAGE_BYTES + 2 * A_BYTES;
      const uint32_t bar = smem_u32(&full_b[st]);
      // the whole B tile of both planes, loaded by this CTA for its own products
      bar_expect_tx(bar, 2u * B_BYTES);
      tma_load_2d(smem_u32(Bhi), &tm_hi, (int)(ch * KT), (int)c0, bar);
      tma_load_2d(smem_u32(Bhi + B_BYTES), &tm_lo, (int)(ch * KT), (int)c0, bar);
      armed[st] = true;
      armed_par[st] = (uint32_t)((ch / NST) & 1);
    };
    for (int64_t c = 0; c < NST - 1 && c < nchunk; ++c) arm(c);
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      const int st = (int)(ch % NST);
      const uint32_t par = (uint32_t)((ch / NST) & 1);
      if (!bar_wait(smem_u32(&full_b[st]), par)) ok = false;
      else armed[st] = false;
      if (!bar_wait(smem_u32(&full_a[st]), par)) ok = false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* base = smem + st * STAGE_BYTES;
      const uint32_t a_hi = smem_u32(base), a_lo = a_hi + A_BYTES;
      const uint32_t b_hi = a_hi + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
#pragma unroll
      for (int kk = 0; kk < KT / 8; ++kk) {  // K = 8 TF32 values (32 bytes) per instruction
        const uint32_t ko = kk * 32;
        const uint64_t bh = smem_desc<KT>(b_hi + ko), bl = smem_desc<KT>(b_lo + ko);
#pragma unroll
        for (int h = 0; h < RH; ++h) {  // both accumulators read the same B stage
          const uint32_t td = tmem + (uint32_t)h * ACC_COLS, ho = (uint32_t)h * AH_BYTES + ko;
          mma_tf32(td, smem_desc<KT>(a_hi + ho), bh, idesc, (ch > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(td, smem_desc<KT>(a_hi + ho), bl, idesc, 1u);
          mma_tf32(td, smem_desc<KT>(a_lo + ho), bh, idesc, 1u);
        }
      }
      mma_commit(smem_u32(&empty[st]));
      const int64_t nxt = ch + NST - 1;
      if (nxt < nchunk) {
        // chunk nxt reuses the stage of chunk ch - 1: free once that chunk's products are done
        if (ch >= 1 && !bar_wait(smem_u32(&empty[(ch - 1) % NST]), (uint32_t)(((ch - 1) / NST) & 1))) ok = false;
        arm(nxt);
      }
    }
    if (!ok) {
      s_timeout = 1;
      for (int s = 0; s < NST; ++s)  // copies still in flight must land before the CTA exits
        if (armed[s]) bar_wait(smem_u32(&full_b[s]), armed_par[s]);
    }
  }
  if (warp == NPROD / 32) __syncwarp();  // lanes 1..31 of the issuing warp wait here, not spinning
  // every thread: the last commit completes after all earlier products
  if (nchunk > 0) {
    const int64_t last = nchunk - 1;
    if (!bar_wait(smem_u32(&empty[last % NST]), (uint32_t)((last / NST) & 1))) s_timeout = 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp < NPROD / 32 && nchunk > 0) {
    // epilogue: warp w reads TMEM lanes 32*(w%4).. (its rows), columns (w/4)*64 .. +64 of each
    // accumulator
    const int colbase = (warp >> 2) * 64;
#pragma unroll 1
    for (int h = 0; h < RH; ++h) {
      const int row = h * TM + 32 * (warp & 3) + lane;
      const int64_t gi = i0 + row;
      for (int cc = 0; cc < 64; cc += 16) {
        if (colbase + cc >= nmma) break;  // warp-uniform
        uint32_t r[16];
        const uint32_t taddr =
            tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)h * ACC_COLS + (uint32_t)(colbase + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (gi < n) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int64_t gc = c0 + colbase + cc + q;
            if (gc < ncols) {
              const bool first = gc < ncols0;
              const int64_t c = first ? gc : gc - ncols0;
              const double* in = first ? in0 : in1;
              double* out = first ? out0 : out1;
              out[gi * ld + c] = shift * in[gi * ld + c] + scale * (double)__uint_as_float(r[q]);
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  if (tid == 0 && s_timeout && err) atomicCAS(err, 0, kDevTimeout);
}

// Points in FP32, zero padded to a multiple of TK points.
__global__ void k_points_f32(const double* __restrict__ pts, int64_t n, int d, int64_t npad, float* __restrict__ out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npad * d) return;
  out[e] = e < n * d ? (float)pts[e] : 0.f;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// Tensor map of one plane: ncols rows of n FP32 values, row pitch ldp values (ldp % 4 == 0 so that
// the pitch is a multiple of 16 bytes); box = KT values x a whole column tile, the swizzle of the
// KT-point layout, zero fill outside [0, n) x [0, ncols).
bool plane_map(CUtensorMap* m, const float* base, int64_t n, int64_t ncols, int64_t ldp, int tn, int kt,
               CUtensorMapSwizzle swz) {
  EncodeTiled enc = encode_fn();
  if (!enc || (ldp & 3) || ((uintptr_t)base & 15)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)ncols};
  cuuint64_t strides[1] = {(cuuint64_t)ldp * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)kt, (cuuint32_t)tn};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TN, int KT, int NST, int RH>
bool launch_variant(cudaStream_t st, int kind, const float* p32, int64_t n, double shift, double scale,
                    const double* in0, const double* in1, double* out0, double* out1, int64_t ld, int64_t ncols0,
                    int64_t ncols, const float* bhi, const float* blo, int64_t ldp, int* err) {
  CUtensorMap mh, ml;
  if (!plane_map(&mh, bhi, n, ncols, ldp, TN, KT, Lay<KT>::TMA_SWIZZLE) ||
      !plane_map(&ml, blo, n, ncols, ldp, TN, KT, Lay<KT>::TMA_SWIZZLE))
    return false;
  using C = Tile<TN, KT, NST, RH>;
  constexpr int SMEM = C::SMEM_BYTES;
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(k_kmv_tc<RSRS_OP_LOG2D, 2, TN, KT, NST, RH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SMEM);
    cudaFuncSetAttribute(k_kmv_tc<RSRS_OP_INVR3D, 3, TN, KT, NST, RH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SMEM);
  });
  const dim3 grid((unsigned)((n + C::MR - 1) / C::MR), (unsigned)((ncols + TN - 1) / TN));
  if (kind == RSRS_OP_LOG2D)
    k_kmv_tc<RSRS_OP_LOG2D, 2, TN, KT, NST, RH><<<grid, NTHREADS, SMEM, st>>>(mh, ml, p32, n, shift, scale, in0, in1,
                                                                               out0, out1, ld, ncols0, ncols, err);
  else
    k_kmv_tc<RSRS_OP_INVR3D, 3, TN, KT, NST, RH><<<grid, NTHREADS, SMEM, st>>>(mh, ml, p32, n, shift, scale, in0, in1,
                                                                                out0, out1, ld, ncols0, ncols, err);
  return true;
}

}  // namespace

int64_t tc_plane_ld(int64_t n) { return (n + 3) & ~(int64_t)3; }
int64_t tc_points_len(int64_t n, int d) { return ((n + TK - 1) / TK) * TK * d; }

void launch_points_f32(Launch L, const double* pts, int64_t n, int d, float* out) {
  const int64_t npad = (n + TK - 1) / TK * TK;
  k_points_f32<<<(unsigned)((npad * d + 255) / 256), 256, 0, L.st>>>(pts, n, d, npad, out);
  if (L.counter) ++*L.counter;
}

bool launch_kernel_matvec_tc(Launch L, int kind, const float* p32, int64_t n, double shift, double scale,
                             const double* in0, const double* in1, double* out0, double* out1, int64_t ld,
                             int64_t ncols0, int64_t ncols, const float* bhi, const float* blo, int64_t ldp, int* err,
                             int variant) {
  if (n <= 0 || ncols <= 0) return true;
  bool ok;
#define RSRS_KMV_TC(TN, KT, NST, RH)                                                                              \
  launch_variant<TN, KT, NST, RH>(L.st, kind, p32, n, shift, scale, in0, in1, out0, out1, ld, ncols0, ncols, bhi, \
                                  blo, ldp, err)
  switch (variant) {
    case RSRS_SAMPLE_TILE_128x3: ok = RSRS_KMV_TC(128, 32, 3, 1); break;
    case RSRS_SAMPLE_TILE_192x2: ok = RSRS_KMV_TC(192, 32, 2, 1); break;
    case RSRS_SAMPLE_TILE_256x2: ok = RSRS_KMV_TC(256, 32, 2, 1); break;
    case RSRS_SAMPLE_TILE_256x4_K16: ok = RSRS_KMV_TC(256, 16, 4, 1); break;
    case RSRS_SAMPLE_TILE_192x5_K16: ok = RSRS_KMV_TC(192, 16, 5, 1); break;
    case RSRS_SAMPLE_TILE_2x192x4_K16: ok = RSRS_KMV_TC(192, 16, 4, 2); break;
    default:  // RSRS_SAMPLE_TILE_2x256x3_K16: two accumulators share each B stage
      ok = RSRS_KMV_TC(256, 16, 3, 2);
  }
#undef RSRS_KMV_TC
  if (ok && L.counter) ++*L.counter;
  return ok;
}

}  // namespace rsrs
