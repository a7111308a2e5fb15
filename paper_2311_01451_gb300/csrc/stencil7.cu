// 7-point variable-coefficient operator on an m x m x m cell grid, as a matvec callback
// (rsrs_matvec_fn): cell-centred finite volumes with face coefficients beta = 2 b_i b_j / (b_i + b_j)
// (harmonic mean) between neighbouring cells and beta = 2 b_i on the boundary faces (Dirichlet wall
// half a cell away), no h^-2 scaling:
//   (A u)_i = sum over interior faces (i, j) of beta_ij (u_i - u_j) + sum over boundary faces of 2 b_i u_i.
// A is symmetric, so the adjoint is the same product.  Cells are ordered with x fastest, then y,
// then z (the order of the points the tree is built from).  The face coefficients are formed once in
// FP64 on the host; the product is HBM-bound (seven loads and one store per cell and column).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "common.cuh"

struct rsrs_stencil7 {
  int m = 0;
  double* face = nullptr;  // 4 x m^3: beta to the +x, +y, +z neighbour (0 at the far wall), boundary sum
};

namespace {

constexpr int kColChunk = 32;  // columns per CTA (grid.y), so that wide blocks fill the GPU

// face[0..2][e]: beta towards the +x / +y / +z neighbour of cell e (0 when there is none);
// face[3][e]: sum of 2 b_e over the cell's boundary faces.
__global__ void __launch_bounds__(256) k_stencil7(const double* __restrict__ face, int m, int ncols,
                                                  const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                                  int64_t ldy) {
  const int64_t n = (int64_t)m * m * m;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int x = (int)(e % m), y = (int)((e / m) % m), z = (int)(e / ((int64_t)m * m));
  const int64_t sy = m, sz = (int64_t)m * m;
  const double bxp = face[e], byp = face[n + e], bzp = face[2 * n + e], bnd = face[3 * n + e];
  const double bxm = x > 0 ? face[e - 1] : 0.0;
  const double bym = y > 0 ? face[n + e - sy] : 0.0;
  const double bzm = z > 0 ? face[2 * n + e - sz] : 0.0;
  const double diag = bxp + bxm + byp + bym + bzp + bzm + bnd;
  const int c1 = min(ncols, (int)(blockIdx.y + 1) * kColChunk);
  for (int c = blockIdx.y * kColChunk; c < c1; ++c) {
    const double* u = X + (int64_t)c * ldx;
    double acc = diag * u[e];
    if (x + 1 < m) acc -= bxp * u[e + 1];
    if (x > 0) acc -= bxm * u[e - 1];
    if (y + 1 < m) acc -= byp * u[e + sy];
    if (y > 0) acc -= bym * u[e - sy];
    if (z + 1 < m) acc -= bzp * u[e + sz];
    if (z > 0) acc -= bzm * u[e - sz];
    Y[(int64_t)c * ldy + e] = acc;
  }
}

}  // namespace

extern "C" {

rsrs_status rsrs_stencil7_create(const double* coef_host, int m, rsrs_stencil7** out) {
  if (!out) return RSRS_E_INVAL;
  *out = nullptr;
  if (!coef_host || m <= 0 || (int64_t)m * m * m > INT32_MAX) return RSRS_E_INVAL;
  const int64_t n = (int64_t)m * m * m;
  std::vector<double> face(4 * n, 0.0);
  for (int64_t e = 0; e < n; ++e) {
    const double b = coef_host[e];
    if (!(b > 0.0) || !std::isfinite(b)) return RSRS_E_INVAL;
  }
  for (int64_t e = 0; e < n; ++e) {
    const int x = (int)(e % m), y = (int)((e / m) % m), z = (int)(e / ((int64_t)m * m));
    const double bi = coef_host[e];
    const int64_t step[3] = {1, m, (int64_t)m * m};
    const int pos[3] = {x, y, z};
    double bnd = 0.0;
    for (int a = 0; a < 3; ++a) {
      if (pos[a] + 1 < m) {
        const double bj = coef_host[e + step[a]];
        face[a * n + e] = 2.0 * bi * bj / (bi + bj);
      } else {
        bnd += 2.0 * bi;
      }
      if (pos[a] == 0) bnd += 2.0 * bi;
    }
    face[3 * n + e] = bnd;
  }
  auto s = new rsrs_stencil7;
  s->m = m;
  if (cudaMalloc((void**)&s->face, face.size() * sizeof(double)) != cudaSuccess ||
      cudaMemcpy(s->face, face.data(), face.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(s->face);
    delete s;
    cudaGetLastError();
    return RSRS_E_NOMEM;
  }
  *out = s;
  return RSRS_OK;
}

int rsrs_stencil7_matvec(void* ctx, int adjoint, int64_t n, int32_t ncols, const double* X_dev, int64_t ldx,
                         double* Y_dev, int64_t ldy, void* stream) {
  (void)adjoint;  // symmetric
  const rsrs_stencil7* s = static_cast<const rsrs_stencil7*>(ctx);
  if (!s || n != (int64_t)s->m * s->m * s->m || ncols <= 0 || ldx < n || ldy < n) return 1;
  const dim3 grid((unsigned)((n + 255) / 256), (unsigned)((ncols + kColChunk - 1) / kColChunk));
  k_stencil7<<<grid, 256, 0, (cudaStream_t)stream>>>(s->face, s->m, ncols, X_dev, ldx, Y_dev, ldy);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

void rsrs_stencil7_free(rsrs_stencil7* s) {
  if (!s) return;
  cudaFree(s->face);
  delete s;
}

}  // extern "C"
