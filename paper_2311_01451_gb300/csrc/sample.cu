// Sampling matvec of eq. (rand_sample_setting) for the built-in kernel matrices,
// A = shift*I + scale*K with K_ij = log|x_i - x_j| (2D) or 1/|x_i - x_j| (3D),
// K_ii = 0, generated tile by tile on the fly (never stored).  The same kernel
// gives the FP64 residual product of iterative refinement.
//
// Tile: 64 rows x 128 columns of the output per CTA; each 32-deep slice of K is
// evaluated once into shared memory and reused across the 128 columns.  The
// identity term is added exactly in FP64.  The FP32 variant (mixed precision)
// evaluates K and accumulates in FP32, flushing the partial sums into FP64
// every 512 points so the rounding does not grow with N.
#include <cmath>

#include "common.cuh"

namespace rsrs {
namespace {

constexpr int RM = 64, CN = 128, JK = 32, JK64 = 16;

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

template <int KIND, int D>
__global__ void __launch_bounds__(256) k_kmv32(const double* __restrict__ pts, int64_t n, double shift,
                                               double scale, const double* __restrict__ in, int64_t ld_in,
                                               double* __restrict__ out, int64_t ld_out, int64_t ncols) {
  __shared__ float Ks[JK][RM];
  __shared__ float Xs[JK][CN];
  __shared__ float Pi[RM][D];
  __shared__ float Pj[JK][D];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * RM, c0 = (int64_t)blockIdx.y * CN;
  for (int e = tid; e < RM * D; e += 256) {
    int i = e / D, k = e % D;
    Pi[i][k] = (i0 + i < n) ? (float)pts[(i0 + i) * D + k] : 0.f;
  }
  double hi[4][8] = {};
  float acc[4][8] = {};
  int slices = 0;
  for (int64_t j0 = 0; j0 < n; j0 += JK) {
    if (tid < JK * D) {
      int j = tid / D, k = tid % D;
      Pj[j][k] = (j0 + j < n) ? (float)pts[(j0 + j) * D + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < (RM * JK) / 256; ++u) {
      int e = tid + 256 * u;
      int i = e & (RM - 1), jj = e / RM;
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
    for (int u = 0; u < (JK * CN) / 256; ++u) {
      int e = tid + 256 * u;
      int jj = e / CN, c = e % CN;
      int64_t gj = j0 + jj, gc = c0 + c;
      Xs[jj][c] = (gj < n && gc < ncols) ? (float)in[gj * ld_in + gc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < JK; ++jj) {
      float a[4], b[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Ks[jj][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 8; ++v) b[v] = Xs[jj][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
    if (++slices == 16) {
      slices = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          hi[u][v] += (double)acc[u][v];
          acc[u][v] = 0.f;
        }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t gi = i0 + ty + 16 * u;
    if (gi >= n) continue;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      int64_t gc = c0 + tx + 16 * v;
      if (gc < ncols)
        out[gi * ld_out + gc] = shift * in[gi * ld_in + gc] + scale * (hi[u][v] + (double)acc[u][v]);
    }
  }
}

}  // namespace

void launch_kernel_matvec(Launch L, int kind, const double* pts, int d, int64_t n, double shift, double scale,
                          const double* in, int64_t ld_in, double* out, int64_t ld_out, int64_t ncols) {
  launch_kernel_matvec_prec(L, kind, pts, d, n, shift, scale, in, ld_in, out, ld_out, ncols, 0);
}

void launch_kernel_matvec_prec(Launch L, int kind, const double* pts, int d, int64_t n, double shift,
                               double scale, const double* in, int64_t ld_in, double* out, int64_t ld_out,
                               int64_t ncols, int fp32) {
  if (n <= 0 || ncols <= 0) return;
  dim3 grid((unsigned)((n + RM - 1) / RM), (unsigned)((ncols + CN - 1) / CN));
  if (kind == RSRS_OP_LOG2D) {
    if (fp32)
      k_kmv32<RSRS_OP_LOG2D, 2><<<grid, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, out, ld_out, ncols);
    else
      k_kmv64<RSRS_OP_LOG2D, 2><<<grid, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, out, ld_out, ncols);
  } else {
    if (fp32)
      k_kmv32<RSRS_OP_INVR3D, 3><<<grid, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, out, ld_out, ncols);
    else
      k_kmv64<RSRS_OP_INVR3D, 3><<<grid, 256, 0, L.st>>>(pts, n, shift, scale, in, ld_in, out, ld_out, ncols);
  }
  if (L.counter) ++*L.counter;
}

}  // namespace rsrs
