// Sampling matvec of eq. (rand_sample_setting) for the built-in kernel matrices,
// A = shift*I + scale*K with K_ij = log|x_i - x_j| (2D) or 1/|x_i - x_j| (3D),
// K_ii = 0, generated tile by tile on the fly (never stored).  The same kernel
// gives the FP64 residual product of iterative refinement.
//
// Each slice of K is evaluated once per CTA into shared memory and reused across
// the CTA's columns; the identity term is added exactly in FP64.  Three
// variants: FP64 for wide blocks (the FP64 sampling), FP64 for at most 32
// columns (refinement residuals), FP32 (mixed-precision sampling; FP32
// accumulation over N points gives about sqrt(N) eps_32 relative rounding,
// below the FP32 projection floor of the mixed path).
#include <cmath>

#include "common.cuh"

namespace rsrs {
namespace {

constexpr int RM = 64, CN = 128, JK64 = 16;

template <int KIND>
__device__ __forceinline__ double kval(double r2) {
  if (KIND == RSRS_OP_LOG2D) return 0.5 * log(r2);
  return rsqrt(r2);
}
template <int KIND>
__device__ __forceinline__ float kvalf(float r2) {
  if (KIND == RSRS_OP_LOG2D) return 0.5f * __logf(r2);
  return rsqrtf(r2);
}

template <int KIND, int D>
__global__ void __launch_bounds__(256) k_kmv64(const double* __restrict__ pts, int64_t n, double shift,
                                               double scale, const double* __restrict__ in, int64_t ld_in,
                                               double* __restrict__ out, int64_t ld_out, int64_t ncols) {
  __shared__ double Ks[JK64][RM];
  __shared__ double Xs[JK64][CN];
  __shared__ double Pi[RM][D];
  __shared__ double Pj[JK64][D];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * RM, c0 = (int64_t)blockIdx.y * CN;
  for (int e = tid; e < RM * D; e += 256) {
    int i = e / D, k = e % D;
    Pi[i][k] = (i0 + i < n) ? pts[(i0 + i) * D + k] : 0.0;
  }
  double acc[4][8] = {};
  for (int64_t j0 = 0; j0 < n; j0 += JK64) {
    if (tid < JK64 * D) {
      int j = tid / D, k = tid % D;
      Pj[j][k] = (j0 + j < n) ? pts[(j0 + j) * D + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < (RM * JK64) / 256; ++u) {
      int e = tid + 256 * u;
      int i = e & (RM - 1), jj = e / RM;
      int64_t gi = i0 + i, gj = j0 + jj;
      double v = 0.0;
      if (gi < n && gj < n && gi != gj) {
        double r2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          double dd = Pi[i][k] - Pj[jj][k];
          r2 = fma(dd, dd, r2);
        }
        v = kval<KIND>(r2);
      }
      Ks[jj][i] = v;
    }
#pragma unroll
    for (int u = 0; u < (JK64 * CN) / 256; ++u) {
      int e = tid + 256 * u;
      int jj = e / CN, c = e % CN;
      int64_t gj = j0 + jj, gc = c0 + c;
      Xs[jj][c] = (gj < n && gc < ncols) ? in[gj * ld_in + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < JK64; ++jj) {
      double a[4], b[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Ks[jj][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 8; ++v) b[v] = Xs[jj][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t gi = i0 + ty + 16 * u;
    if (gi >= n) continue;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      int64_t gc = c0 + tx + 16 * v;
      if (gc < ncols) out[gi * ld_out + gc] = shift * in[gi * ld_in + gc] + scale * acc[u][v];
    }
  }
}

// FP32 product with 128 x 128 output tiles: each thread owns an 8 x 8 block (rows ty*4+{0..3} and
// 64+ty*4+{0..3}, columns likewise) so that every 64 FMAs read four float4 from shared memory.
constexpr int RM2 = 128, CN2 = 128, JK2 = 16;
template <int KIND, int D>
__global__ void __launch_bounds__(256) k_kmv32w(const double* __restrict__ pts, int64_t n, double shift,
                                                double scale, const double* __restrict__ in, int64_t ld_in,
                                                const float* __restrict__ in32, double* __restrict__ out,
                                                int64_t ld_out, int64_t ncols) {
  __shared__ __align__(16) float Ks[JK2][RM2];
  __shared__ __align__(16) float Xs[JK2][CN2];
  __shared__ float Pi[RM2][D];
  __shared__ float Pj[JK2][D];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * RM2, c0 = (int64_t)blockIdx.y * CN2;
  for (int e = tid; e < RM2 * D; e += 256) {
    int i = e / D, k = e % D;
    Pi[i][k] = (i0 + i < n) ? (float)pts[(i0 + i) * D + k] : 0.f;
  }
  float acc[8][8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
  for (int64_t j0 = 0; j0 < n; j0 += JK2) {
    if (tid < JK2 * D) {
      int j = tid / D, k = tid % D;
      Pj[j][k] = (j0 + j < n) ? (float)pts[(j0 + j) * D + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < (RM2 * JK2) / 256; ++u) {
      int e = tid + 256 * u;
      int i = e & (RM2 - 1), jj = e / RM2;
      int64_t gi = i0 + i, gj = j0 + jj;
      float v = 0.f;
      if (gi < n && gj < n && gi != gj) {
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float dd = Pi[i][k] - Pj[jj][k];
          r2 = fmaf(dd, dd, r2);
        }
        v = kvalf<KIND>(r2);
      }
      Ks[jj][i] = v;
    }
#pragma unroll
    for (int u = 0; u < (JK2 * CN2) / 256; ++u) {
      int e = tid + 256 * u;
      int jj = e / CN2, c = e % CN2;
      int64_t gj = j0 + jj, gc = c0 + c;
      Xs[jj][c] = (gj < n && gc < ncols) ? in32[gj * ld_in + gc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < JK2; ++jj) {
      float4 a0 = *reinterpret_cast<const float4*>(&Ks[jj][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&Ks[jj][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Xs[jj][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Xs[jj][64 + tx * 4]);
      float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    int64_t gi = i0 + (u < 4 ? ty * 4 + u : 64 + ty * 4 + (u - 4));
    if (gi >= n) continue;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      int64_t gc = c0 + (v < 4 ? tx * 4 + v : 64 + tx * 4 + (v - 4));
      if (gc < ncols) out[gi * ld_out + gc] = shift * in[gi * ld_in + gc] + scale * (double)acc[u][v];
    }
  }
}

// FP64 product for a few columns (refinement residuals): 128 rows x 16 columns per CTA, each
// thread 8 rows of one column, so each kernel value (the expensive part in FP64) is evaluated
// once per CTA and used for 16 columns instead of being spread over a wide, mostly empty tile.
constexpr int RM3 = 128, CN3 = 16, JK3 = 32;
template <int KIND, int D>
__global__ void __launch_bounds__(256) k_kmv64n(const double* __restrict__ pts, int64_t n, double shift,
                                                double scale, const double* __restrict__ in, int64_t ld_in,
                                                double* __restrict__ out, int64_t ld_out, int64_t ncols) {
  __shared__ double Ks[JK3][RM3];
  __shared__ double Xs[JK3][CN3];
  __shared__ double Pi[RM3][D];
  __shared__ double Pj[JK3][D];
  const int tid = threadIdx.x, tc = tid & 15, tr = tid >> 4;  // column tc, rows tr + 16u
  const int64_t i0 = (int64_t)blockIdx.x * RM3, c0 = (int64_t)blockIdx.y * CN3;
  for (int e = tid; e < RM3 * D; e += 256) {
    int i = e / D, k = e % D;
    Pi[i][k] = (i0 + i < n) ? pts[(i0 + i) * D + k] : 0.0;
  }
  double acc[8] = {};
  for (int64_t j0 = 0; j0 < n; j0 += JK3) {
    if (tid < JK3 * D) {
      int j = tid / D, k = tid % D;
      Pj[j][k] = (j0 + j < n) ? pts[(j0 + j) * D + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int u = 0; u < (RM3 * JK3) / 256; ++u) {
      int e = tid + 256 * u;
      int i = e & (RM3 - 1), jj = e / RM3;
      int64_t gi = i0 + i, gj = j0 + jj;
      double v = 0.0;
      if (gi < n && gj < n && gi != gj) {
        double r2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          double dd = Pi[i][k] - Pj[jj][k];
          r2 = fma(dd, dd, r2);
        }
        v = kval<KIND>(r2);
      }
      Ks[jj][i] = v;
    }
    for (int e = tid; e < JK3 * CN3; e += 256) {
      int jj = e / CN3, c = e % CN3;
      int64_t gj = j0 + jj, gc = c0 + c;
      Xs[jj][c] = (gj < n && gc < ncols) ? in[gj * ld_in + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < JK3; ++jj) {
      double x = Xs[jj][tc];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = fma(Ks[jj][tr + 16 * u], x, acc[u]);
    }
    __syncthreads();
  }
  const int64_t gc = c0 + tc;
  if (gc >= ncols) return;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    int64_t gi = i0 + tr + 16 * u;
    if (gi < n) out[gi * ld_out + gc] = shift * in[gi * ld_in + gc] + scale * acc[u];
  }
}


}  // namespace

void launch_kernel_matvec(Launch L, int kind, const double* pts, int d, int64_t n, double shift, double scale,
                          const double* in, int64_t ld_in, double* out, int64_t ld_out, int64_t ncols) {
  launch_kernel_matvec_prec(L, kind, pts, d, n, shift, scale, in, ld_in, out, ld_out, ncols, 0, nullptr);
}

void launch_kernel_matvec_prec(Launch L, int kind, const double* pts, int d, int64_t n, double shift,
                               double scale, const double* in, int64_t ld_in, double* out, int64_t ld_out,
                               int64_t ncols, int fp32, const float* in32) {
  if (n <= 0 || ncols <= 0) return;
  if (fp32) {
    dim3 g2((unsigned)((n + RM2 - 1) / RM2), (unsigned)((ncols + CN2 - 1) / CN2));
    if (kind == RSRS_OP_LOG2D)
      k_kmv32w<RSRS_OP_LOG2D, 2><<<g2, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, in32, out, ld_out, ncols);
    else
      k_kmv32w<RSRS_OP_INVR3D, 3><<<g2, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, in32, out, ld_out,
                                                        ncols);
    if (L.counter) ++*L.counter;
    return;
  }
  if (ncols <= 32) {
    dim3 g3((unsigned)((n + RM3 - 1) / RM3), (unsigned)((ncols + CN3 - 1) / CN3));
    if (kind == RSRS_OP_LOG2D)
      k_kmv64n<RSRS_OP_LOG2D, 2><<<g3, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, out, ld_out, ncols);
    else
      k_kmv64n<RSRS_OP_INVR3D, 3><<<g3, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, out, ld_out, ncols);
    if (L.counter) ++*L.counter;
    return;
  }
  dim3 grid((unsigned)((n + RM - 1) / RM), (unsigned)((ncols + CN - 1) / CN));
  if (kind == RSRS_OP_LOG2D)
    k_kmv64<RSRS_OP_LOG2D, 2><<<grid, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, out, ld_out, ncols);
  else
    k_kmv64<RSRS_OP_INVR3D, 3><<<grid, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, out, ld_out, ncols);
  if (L.counter) ++*L.counter;
}

}  // namespace rsrs

namespace rsrs {
}  // namespace rsrs

namespace rsrs {
namespace {
__global__ void k_to_f32(const double* __restrict__ in, int64_t count, float* __restrict__ out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = (float)in[e];
}
// hi/lo TF32 split of in (n x s row-major, FP64), transposed to s x n (K-major for the tensor cores),
// through a 32 x 32 shared-memory tile so that both sides are coalesced.
__global__ void k_split_t(const double* __restrict__ in, int64_t n, int64_t s, float* __restrict__ hi,
                          float* __restrict__ lo, int64_t ldp) {
  __shared__ float t[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    int64_t j = j0 + r, c = c0 + tx;
    t[r][tx] = (j < n && c < s) ? (float)in[j * s + c] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int64_t c = c0 + r, j = j0 + tx;
    if (c < s && j < n) {
      float v = t[tx][r];
      float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
      hi[c * ldp + j] = h;
      lo[c * ldp + j] = v - h;
    }
  }
}
}  // namespace
void launch_to_f32(Launch L, const double* in, int64_t count, float* out) {
  if (count <= 0) return;
  k_to_f32<<<(unsigned)((count + 255) / 256), 256, 0, L.st>>>(in, count, out);
  if (L.counter) ++*L.counter;
}
void launch_split_transpose(Launch L, const double* in, int64_t n, int64_t s, float* hi, float* lo, int64_t ldp) {
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((s + 31) / 32));
  k_split_t<<<grid, 256, 0, L.st>>>(in, n, s, hi, lo, ldp);
  if (L.counter) ++*L.counter;
}
}  // namespace rsrs
