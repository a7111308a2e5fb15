// Root block (Algorithm 1, root step): LU with partial pivoting of A~_{Bt Bt} and its inverse, for
// the roots of all problems of a build at once, in FP64.
//
// Right-looking blocked LU, 32-column panels: per panel one CTA per problem factors the panel
// (pivot search, interchange within the panel, column scaling, rank-1 updates), then many CTAs
// apply the panel's interchanges to the other columns and form U12 = L11^-1 A12, and many CTAs
// update the trailing block A22 -= L21 U12 in 64 x 64 tiles.  The interchange record is LAPACK's:
// piv[j] = the row exchanged with row j at step j.  The inverse A^-1 = U^-1 L^-1 P is then formed
// column block by column block (8 columns per CTA), so the root's block of the solve is a product.
#include <cmath>
#include <cstdint>

#include "common.cuh"

namespace rsrs {
namespace {

constexpr int NB = 32;       // panel width
constexpr int UT = 64;       // update tile
constexpr int INV_COLS = 8;  // inverse columns per CTA

__device__ inline void set_err_root(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// Panel factorization, one CTA per problem.  The panel (rows k0..n-1, nb columns) is staged in
// shared memory when it fits (stage = 1), else worked on in place in global memory.
__global__ void __launch_bounds__(256) k_root_panel(const RootLU* R, int64_t k0, int stage, int* err) {
  const RootLU r = R[blockIdx.x];
  const int64_t n = r.n;
  if (k0 >= n) return;
  const int64_t nb = imin64(NB, n - k0);
  extern __shared__ double pan[];  // (n - k0) x NB when staged
  double* A = r.A;
  // P(i, q) = element (k0 + i, k0 + q)
  double* P = stage ? pan : A + k0 * n + k0;
  const int64_t ldp = stage ? NB : n;
  const int64_t m = n - k0;
  if (stage) {
    for (int64_t e = threadIdx.x; e < m * NB; e += blockDim.x) {
      const int64_t i = e / NB, q = e % NB;
      pan[e] = q < nb ? A[(k0 + i) * n + k0 + q] : 0.0;
    }
    __syncthreads();
  }
  __shared__ double red_v[8];
  __shared__ int64_t red_i[8];
  __shared__ int64_t s_p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t jj = 0; jj < nb; ++jj) {
    double bv = -1.0;
    int64_t bp = -1;
    for (int64_t i = jj + threadIdx.x; i < m; i += blockDim.x) {
      const double v = fabs(P[i * ldp + jj]);
      if (v > bv) {  // ascending rows per thread: ties keep the lower row
        bv = v;
        bp = i;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int64_t op = __shfl_xor_sync(0xffffffffu, bp, o);
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
      int64_t p0 = jj;
      for (int w = 0; w < nw; ++w)
        if (red_i[w] >= 0 && (red_v[w] > v0 || (red_v[w] == v0 && red_i[w] < p0))) {
          v0 = red_v[w];
          p0 = red_i[w];
        }
      if (!(v0 > 0.0)) set_err_root(err, kDevSingular);
      else if (!isfinite(v0)) set_err_root(err, kDevNonfinite);
      s_p = p0;
      r.piv[k0 + jj] = (int32_t)(k0 + p0);
    }
    __syncthreads();
    const int64_t p = s_p;
    if (p != jj)  // interchange within the panel's columns
      for (int64_t c = threadIdx.x; c < nb; c += blockDim.x) {
        const double t = P[jj * ldp + c];
        P[jj * ldp + c] = P[p * ldp + c];
        P[p * ldp + c] = t;
      }
    __syncthreads();
    double dj = P[jj * ldp + jj];
    if (dj == 0.0) dj = 1.0;
    const double inv = 1.0 / dj;
    for (int64_t i = jj + 1 + threadIdx.x; i < m; i += blockDim.x) P[i * ldp + jj] *= inv;
    __syncthreads();
    // rank-1 update of the panel columns right of jj: lanes over columns, warps over rows
    if (jj + 1 < nb)
      for (int64_t i = jj + 1 + warp; i < m; i += nw) {
        const double lij = P[i * ldp + jj];
        for (int64_t c = jj + 1 + lane; c < nb; c += 32) P[i * ldp + c] -= lij * P[jj * ldp + c];
      }
    __syncthreads();
  }
  if (stage)
    for (int64_t e = threadIdx.x; e < m * NB; e += blockDim.x) {
      const int64_t i = e / NB, q = e % NB;
      if (q < nb) A[(k0 + i) * n + k0 + q] = pan[e];
    }
}

// Columns outside the panel: the panel's interchanges, then (right of the panel) U12 = L11^-1 A12.
__global__ void __launch_bounds__(UT) k_root_swap_trsm(const RootLU* R, int64_t k0) {
  const RootLU r = R[blockIdx.y];
  const int64_t n = r.n;
  if (k0 >= n) return;
  const int64_t nb = imin64(NB, n - k0);
  const int64_t c = (int64_t)blockIdx.x * UT + threadIdx.x;  // one column per thread
  if (c >= n || (c >= k0 && c < k0 + nb)) return;
  double* A = r.A;
  for (int64_t j = k0; j < k0 + nb; ++j) {
    const int64_t p = r.piv[j];
    if (p != j) {
      const double t = A[j * n + c];
      A[j * n + c] = A[p * n + c];
      A[p * n + c] = t;
    }
  }
  if (c < k0 + nb) return;
  for (int64_t j = k0; j < k0 + nb; ++j) {  // unit lower triangular solve down the column
    const double x = A[j * n + c];
    for (int64_t i = j + 1; i < k0 + nb; ++i) A[i * n + c] -= A[i * n + j] * x;
  }
}

// A22 -= L21 U12 over 64 x 64 tiles of the trailing block, K = nb.
__global__ void __launch_bounds__(256) k_root_update(const RootLU* R, int64_t k0) {
  const RootLU r = R[blockIdx.z];
  const int64_t n = r.n;
  const int64_t t0 = k0 + imin64(NB, n - k0);  // first trailing row / column
  if (k0 >= n || t0 >= n) return;
  const int64_t i0 = t0 + (int64_t)blockIdx.y * UT, j0 = t0 + (int64_t)blockIdx.x * UT;
  if (i0 >= n || j0 >= n) return;
  const int64_t nb = t0 - k0;
  double* A = r.A;
  __shared__ double Ls[UT][NB + 1];
  __shared__ double Us[NB][UT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int e = threadIdx.x; e < UT * NB; e += blockDim.x) {
    const int a = e / NB, q = e % NB;  // L21 row a, column q
    Ls[a][q] = (i0 + a < n && q < nb) ? A[(i0 + a) * n + k0 + q] : 0.0;
    const int qq = e / UT, b = e % UT;  // U12 row qq, column b
    Us[qq][b] = (qq < nb && j0 + b < n) ? A[(k0 + qq) * n + j0 + b] : 0.0;
  }
  __syncthreads();
  double acc[4][4] = {};
  for (int q = 0; q < NB; ++q) {
    double lv[4], uv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      lv[u] = Ls[ty + 16 * u][q];
      uv[u] = Us[q][tx + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(lv[u], uv[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + ty + 16 * u;
    if (i >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t j = j0 + tx + 16 * v;
      if (j < n) A[i * n + j] -= acc[u][v];
    }
  }
}

// INV_COLS columns of A^-1 = U^-1 L^-1 P per CTA, worked in place in the output.
__global__ void __launch_bounds__(256) k_root_inverse(const RootLU* R) {
  const RootLU r = R[blockIdx.y];
  const int64_t n = r.n;
  const int64_t c0 = (int64_t)blockIdx.x * INV_COLS;
  if (c0 >= n) return;
  const double* LU = r.A;
  double* X = r.inv;
  extern __shared__ int32_t perm[];  // n: row i of P I is e_perm[i]
  if (threadIdx.x == 0) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t j = 0; j < n; ++j) {
      const int32_t p = r.piv[j];
      const int32_t t = perm[j];
      perm[j] = perm[p];
      perm[p] = t;
    }
  }
  __syncthreads();
  const int64_t nc = imin64(INV_COLS, n - c0);
  for (int64_t e = threadIdx.x; e < n * INV_COLS; e += blockDim.x) {
    const int64_t i = e / INV_COLS, q = e % INV_COLS;
    if (q < nc) X[i * n + c0 + q] = (perm[i] == c0 + q) ? 1.0 : 0.0;
  }
  __syncthreads();
  // forward: unit lower
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t e = threadIdx.x; e < (n - j - 1) * INV_COLS; e += blockDim.x) {
      const int64_t i = j + 1 + e / INV_COLS, q = e % INV_COLS;
      if (q < nc) X[i * n + c0 + q] -= LU[i * n + j] * X[j * n + c0 + q];
    }
    __syncthreads();
  }
  // backward: upper
  for (int64_t j = n - 1; j >= 0; --j) {
    if (threadIdx.x < nc) {
      double d = LU[j * n + j];
      if (d == 0.0) d = 1.0;
      X[j * n + c0 + threadIdx.x] /= d;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < j * INV_COLS; e += blockDim.x) {
      const int64_t i = e / INV_COLS, q = e % INV_COLS;
      if (q < nc) X[i * n + c0 + q] -= LU[i * n + j] * X[j * n + c0 + q];
    }
    __syncthreads();
  }
}

}  // namespace

void launch_root_lu_inverse(Launch L, const RootLU* R_dev, int nprob, int64_t max_n, int* err) {
  if (nprob <= 0 || max_n <= 0) return;
  // stage the panel in shared memory when (max_n x NB) doubles fit
  const size_t pan_bytes = (size_t)max_n * NB * sizeof(double);
  const int stage = pan_bytes <= 200 * 1024 ? 1 : 0;
  if (stage && pan_bytes > 48 * 1024)
    cudaFuncSetAttribute(k_root_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pan_bytes);
  for (int64_t k0 = 0; k0 < max_n; k0 += NB) {
    k_root_panel<<<(unsigned)nprob, 256, stage ? pan_bytes : 0, L.st>>>(R_dev, k0, stage, err);
    dim3 gs((unsigned)cdiv(max_n, UT), (unsigned)nprob);
    k_root_swap_trsm<<<gs, UT, 0, L.st>>>(R_dev, k0);
    const int64_t rest = max_n - imin64(max_n, k0 + NB);
    if (rest > 0) {
      dim3 gu((unsigned)cdiv(rest, UT), (unsigned)cdiv(rest, UT), (unsigned)nprob);
      k_root_update<<<gu, 256, 0, L.st>>>(R_dev, k0);
    }
    if (L.counter) *L.counter += rest > 0 ? 3 : 2;
  }
  const size_t smem = (size_t)max_n * sizeof(int32_t);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_root_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 gi((unsigned)cdiv(max_n, INV_COLS), (unsigned)nprob);
  k_root_inverse<<<gi, 256, smem, L.st>>>(R_dev);
  if (L.counter) ++*L.counter;
}

}  // namespace rsrs
