// Mixed-precision sampling product on the 5th-generation tensor cores (tcgen05, TMEM accumulators):
//   out = shift * in + scale * K * in,   K_ij = log|x_i - x_j| (2D) or 1/|x_i - x_j| (3D), K_ii = 0,
// in 3xTF32: every FP32 operand value v is split into hi = v with the 13 low mantissa bits cleared
// (exact in TF32) and lo = v - hi, and D += A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 in
// tensor memory.  The split follows Ootomo & Yokota (2022); products are then accurate to about
// 2^-21 relative, the level of the FP32 arithmetic of the rest of the mixed path.
//
// Tile: D = 128 rows (TMEM lanes) x 256 columns (TMEM columns).  Per stage, 32 points j:
//   A_hi, A_lo: K(x_i, x_j) for the 128 rows, generated by the CTA's threads (K-major, 128-byte
//               rows of 32 TF32 values, 128-byte swizzle, 8-row atoms 1024 bytes apart);
//   B_hi, B_lo: in[j][c] for the 256 columns, from hi/lo planes split and transposed once
//               before the product (FP64 -> FP32 conversion runs at FP64 rate on this part,
//               so it must not sit in the inner loop), copied into the same swizzled layout.
// One thread issues the 4 K-steps x 3 products per stage and commits them to the stage's
// mbarrier; two stages alternate so the threads fill one while the tensor cores read the other.
// Every wait is bounded: on expiry the kernel records kDevTimeout and finishes without hanging.
#include <cstdint>

#include "common.cuh"

namespace rsrs {
namespace {

constexpr int TM = 128, TN = 256, TK = 32;
constexpr int A_BYTES = TM * TK * 4;                      // 16 KB
constexpr int B_BYTES = TN * TK * 4;                      // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;     // 96 KB: A_hi, A_lo, B_hi, B_lo
constexpr int NSTAGE = 2;
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;   // + alignment slack
constexpr uint32_t TMEM_COLS = 256;
constexpr long long WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) of a K-major tile with 128-byte rows and the 128-byte swizzle:
// the 16-byte chunk index (bits 4..6) is XOR-ed with the row inside the 8-row atom (bits 7..9).
__device__ __forceinline__ uint32_t sw128(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + (((k >> 2) ^ (row & 7)) << 4) + (k & 3) * 4);
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0..13), leading byte offset (bits
// 16..29, not used by swizzled K-major layouts), stride byte offset >> 4 = 1024 B between 8-row
// atoms (bits 32..45), descriptor version 1 (bits 46..47), base offset 0, 128-byte swizzle (= 2,
// bits 61..63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::tf32: D FP32 (bits 4..5 = 1), A and B TF32 (bits 7..9, 10..12 = 2),
// both K-major, N >> 3 at bits 17..22, M >> 4 at bits 24..28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
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

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

template <int KIND>
__device__ __forceinline__ float kvalf_tc(float r2) {
  if (KIND == RSRS_OP_LOG2D) return 0.5f * __logf(r2);
  return rsqrtf(r2);
}

template <int KIND, int D>
__global__ void __launch_bounds__(256, 1) k_kmv_tc(const double* __restrict__ pts, int64_t n, double shift,
                                                   double scale, const double* __restrict__ in, int64_t ld_in,
                                                   const float* __restrict__ bhi, const float* __restrict__ blo,
                                                   double* __restrict__ out, int64_t ld_out, int64_t ncols,
                                                   int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[NSTAGE];
  __shared__ uint32_t s_tmem;
  __shared__ float Pj[TK][D];
  __shared__ int s_timeout;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = (int64_t)blockIdx.x * TM, c0 = (int64_t)blockIdx.y * TN;

  if (tid == 0) {
    s_timeout = 0;
    for (int s = 0; s < NSTAGE; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])) : "memory");
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

  // this thread's kernel row (A producer: row tid/2, 16 of the 32 points)
  const int arow = tid >> 1, akh = (tid & 1) * 16;
  float pi[D];
#pragma unroll
  for (int k = 0; k < D; ++k) pi[k] = (i0 + arow < n) ? (float)pts[(i0 + arow) * D + k] : 0.f;

  const int64_t nchunk = (n + TK - 1) / TK;
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    const int st = (int)(ch & 1);
    unsigned char* base = smem + st * STAGE_BYTES;
    unsigned char* Ahi = base;
    unsigned char* Alo = base + A_BYTES;
    unsigned char* Bhi = base + 2 * A_BYTES;
    unsigned char* Blo = base + 2 * A_BYTES + B_BYTES;
    const int64_t j0 = ch * TK;
    // B loads first: row c = tid of the 256, 32 consecutive points of the pre-split K-major planes
    // (128 contiguous bytes each), issued before the waits below so that their latency overlaps
    const int bc = tid;
    const int64_t gc = c0 + bc;
    float4 bh[TK / 4], bl[TK / 4];
    const bool full = (gc < ncols) && (j0 + TK <= n) && ((n & 3) == 0);
#pragma unroll
    for (int q = 0; q < TK / 4; ++q) {
      if (full) {
        bh[q] = __ldg(reinterpret_cast<const float4*>(bhi + gc * n + j0) + q);
        bl[q] = __ldg(reinterpret_cast<const float4*>(blo + gc * n + j0) + q);
      } else {
        float h[4], w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t gj = j0 + q * 4 + u;
          const bool ok = gc < ncols && gj < n;
          h[u] = ok ? bhi[gc * n + gj] : 0.f;
          w[u] = ok ? blo[gc * n + gj] : 0.f;
        }
        bh[q] = make_float4(h[0], h[1], h[2], h[3]);
        bl[q] = make_float4(w[0], w[1], w[2], w[3]);
      }
    }
    // the tensor cores must be done with this stage (its previous use, two chunks ago)
    if (ch >= NSTAGE) {
      if (!bar_wait(smem_u32(&bars[st]), (uint32_t)(((ch >> 1) - 1) & 1))) atomicExch(&s_timeout, 1);
    }
    if (tid < TK * D) {
      int j = tid / D, k = tid % D;
      Pj[j][k] = (j0 + j < n) ? (float)pts[(j0 + j) * D + k] : 0.f;
    }
    __syncthreads();
    // A: kernel values, 16 consecutive points per thread = 4 swizzle chunks of 4 values
    {
      const int64_t gi = i0 + arow;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float hv[4], lv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int kk = akh + q * 4 + u;
          const int64_t gj = j0 + kk;
          float v = 0.f;
          if (gi < n && gj < n && gi != gj) {
            float r2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              float dd = pi[k] - Pj[kk][k];
              r2 = fmaf(dd, dd, r2);
            }
            v = kvalf_tc<KIND>(r2);
          }
          hv[u] = tf32_hi(v);
          lv[u] = v - hv[u];
        }
        const uint32_t off = sw128(arow, akh + q * 4);
        *reinterpret_cast<float4*>(Ahi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<float4*>(Alo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
      }
    }
    // B: already split and K-major; 16-byte chunks into the swizzled rows
#pragma unroll
    for (int q = 0; q < TK / 4; ++q) {
      const uint32_t off = sw128(bc, q * 4);
      *reinterpret_cast<float4*>(Bhi + off) = bh[q];
      *reinterpret_cast<float4*>(Blo + off) = bl[q];
    }
    // generic-proxy writes must be visible to the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo), b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
#pragma unroll
      for (int kk = 0; kk < TK / 8; ++kk) {  // K = 8 TF32 values (32 bytes) per instruction
        const uint32_t ko = kk * 32;
        mma_tf32(tmem, smem_desc(a_hi + ko), smem_desc(b_hi + ko), (ch > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(a_hi + ko), smem_desc(b_lo + ko), 1u);
        mma_tf32(tmem, smem_desc(a_lo + ko), smem_desc(b_hi + ko), 1u);
      }
      mma_commit(smem_u32(&bars[st]));
    }
  }
  // wait for the last stage's products (commits complete in issue order)
  if (nchunk > 0) {
    const int64_t last = nchunk - 1;
    if (!bar_wait(smem_u32(&bars[last & 1]), (uint32_t)((last >> 1) & 1))) atomicExch(&s_timeout, 1);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warp w reads TMEM lanes 32*(w%4).. (its rows), columns (w/4)*128 .. +128
  {
    const int row = 32 * (warp & 3) + lane;
    const int64_t gi = i0 + row;
    const int colbase = (warp >> 2) * 128;
    for (int cc = 0; cc < 128; cc += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(colbase + cc);
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
          if (gc < ncols) out[gi * ld_out + gc] = shift * in[gi * ld_in + gc] + scale * (double)__uint_as_float(r[q]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  if (tid == 0 && s_timeout && err) atomicCAS(err, 0, kDevTimeout);
}

}  // namespace

void launch_kernel_matvec_tc(Launch L, int kind, const double* pts, int d, int64_t n, double shift, double scale,
                             const double* in, int64_t ld_in, const float* bhi, const float* blo, double* out,
                             int64_t ld_out, int64_t ncols, int* err) {
  if (n <= 0 || ncols <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_kmv_tc<RSRS_OP_LOG2D, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    cudaFuncSetAttribute(k_kmv_tc<RSRS_OP_INVR3D, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  dim3 grid((unsigned)((n + TM - 1) / TM), (unsigned)((ncols + TN - 1) / TN));
  if (kind == RSRS_OP_LOG2D)
    k_kmv_tc<RSRS_OP_LOG2D, 2><<<grid, 256, SMEM_BYTES, L.st>>>(pts, n, shift, scale, in, ld_in, bhi, blo, out, ld_out,
                                                                ncols, err);
  else
    k_kmv_tc<RSRS_OP_INVR3D, 3><<<grid, 256, SMEM_BYTES, L.st>>>(pts, n, shift, scale, in, ld_in, bhi, blo, out,
                                                                 ld_out, ncols, err);
  if (L.counter) ++*L.counter;
}

}  // namespace rsrs
