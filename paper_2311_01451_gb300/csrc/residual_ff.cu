// Refinement residual product out = shift*in + scale*K*in for the built-in kernels in float-float
// arithmetic on the FP32 pipe.
//
// A float-float value is an unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h)/2, 48
// significant bits.  The error-free transformations are the classical ones: Knuth's TwoSum,
// Dekker's FastTwoSum (|a| >= |b|), and TwoProduct through the fused multiply-add; the dot
// products accumulate with them in the manner of Ogita, Rump & Oishi (2005) and fold the running
// compensated pair into a float-float total every 256 terms, so that the second-order error term
// stays at the 2^-40 level of a 256-term block instead of growing with N.
//
// Kernel values: 2D log|x_i - x_j| = log(r^2)/2 and 3D 1/|x_i - x_j|; coordinates are held exactly
// as three floats, so r^2 keeps 48 bits relative to itself even for the closest pairs:
//   * log: r^2 = 2^e m, m in [1, 2); a 256-entry table of c = 1/fl(1/(1 + (t + 1/2)/256)) indexed
//     by the top 8 bits of m gives u = m fl(1/c) - 1 with |u| <= 2^-9 (Tang's table-driven
//     reduction, 1990), log m = log c + log1p(u) with log1p(u) = u - u^2/2 + u^3/3 (float-float)
//     + u^4 (-1/4 + u/5 - u^2/6 + u^3/7) (FP32, below 2^-27 |u|), and log(r^2) = e ln 2 + log m;
//     log c comes from the host's FP64 log, split into float-float;
//   * 1/r: y = rsqrtf(r^2) corrected by y (h/2 + 3h^2/8), the series of (1 - h)^-1/2 to second
//     order, with the residual h = 1 - r^2 y^2 formed in float-float.
// Relative accuracy of each kernel value is about 2^-46, of each output about 1e-14 of the sum of
// |K_ij x_j|, which is what FP64 refinement to 1e-12 / 1e-13 needs, at a fraction of the cost of
// FP64 arithmetic on this part (its FP32 pipe is 64 times wider than its FP64 pipe).
#include <cmath>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "ff.cuh"

namespace rsrs {
namespace {

constexpr int RT = 128;     // rows (threads) per CTA
constexpr int JT = 64;      // points per shared-memory tile
constexpr int FOLD = 4;     // tiles between folds of the compensated pair into the total

// part[ks][i][c]: float-float partial sum over the points of split ks.
template <int KIND, int D, int NC>
__global__ void __launch_bounds__(RT) k_kmv_ff(const float3* __restrict__ pff, int64_t n,
                                               const float2* __restrict__ xff, int64_t jspan,
                                               float2* __restrict__ part, const LogTable tab) {
  __shared__ LogTable T;
  __shared__ float3 ps[JT][D];
  __shared__ float2 xs[JT][NC];
  const int tid = threadIdx.x;
  for (int q = tid; q < kLogTab; q += RT) {
    T.ic[q] = tab.ic[q];
    T.lch[q] = tab.lch[q];
    T.lcl[q] = tab.lcl[q];
  }
  const int64_t i = (int64_t)blockIdx.x * RT + tid;
  const int ks = blockIdx.y;
  const int64_t j_begin = (int64_t)ks * jspan, j_end = imin64(j_begin + jspan, n);
  float3 pi[D];
#pragma unroll
  for (int k = 0; k < D; ++k) pi[k] = i < n ? pff[i * D + k] : make_float3(0.f, 0.f, 0.f);
  float S[NC], Cc[NC];
  ffv tot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    S[c] = Cc[c] = 0.f;
    tot[c] = {0.f, 0.f};
  }
  int since = 0;
  for (int64_t j0 = j_begin; j0 < j_end; j0 += JT) {
    __syncthreads();
    for (int q = tid; q < JT * D; q += RT) {
      const int64_t j = j0 + q / D;
      ps[q / D][q % D] = j < j_end ? pff[j * D + q % D] : make_float3(0.f, 0.f, 0.f);
    }
    for (int q = tid; q < JT * NC; q += RT) {
      const int64_t j = j0 + q / NC;
      xs[q / NC][q % NC] = j < j_end ? xff[j * NC + q % NC] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int jn = (int)imin64(JT, j_end - j0);
    for (int jj = 0; jj < jn; ++jj) {
      const int64_t j = j0 + jj;
      ffv r2 = {0.f, 0.f};
#pragma unroll
      for (int k = 0; k < D; ++k) r2 = ff_add_pos(r2, ff_sqr(coord_diff(pi[k], ps[jj][k])));
      ffv kv;
      if (KIND == RSRS_OP_LOG2D) {
        kv = ff_log(r2, T);
        kv.h *= 0.5f;
        kv.l *= 0.5f;
      } else {
        kv = ff_rsqrt(r2);
      }
      if (i >= n || j == i) kv = {0.f, 0.f};
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 x = xs[jj][c];
        float p, e, s, t;
        two_prod(kv.h, x.x, p, e);
        e = __fmaf_rn(kv.h, x.y, e);
        e = __fmaf_rn(kv.l, x.x, e);
        two_sum(S[c], p, s, t);
        S[c] = s;
        Cc[c] = __fadd_rn(Cc[c], __fadd_rn(t, e));
      }
    }
    if (++since == FOLD) {
      since = 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        ffv v;
        two_sum(S[c], Cc[c], v.h, v.l);
        tot[c] = ff_add(tot[c], v);
        S[c] = Cc[c] = 0.f;
      }
    }
  }
  if (i >= n) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    ffv v;
    two_sum(S[c], Cc[c], v.h, v.l);
    tot[c] = ff_add(tot[c], v);
    part[((int64_t)ks * n + i) * NC + c] = make_float2(tot[c].h, tot[c].l);
  }
}

// FP64 -> float-float, rows of nsrc values spread into rows of ndst (zero padded).
__global__ void k_to_ff(const double* __restrict__ in, int64_t rows, int nsrc, int64_t ld_in, int ndst,
                        float2* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * ndst) return;
  const int64_t r = e / ndst;
  const int c = (int)(e % ndst);
  float2 v = make_float2(0.f, 0.f);
  if (c < nsrc) {
    const double x = in[r * ld_in + c];
    v.x = (float)x;
    v.y = (float)(x - (double)v.x);
  }
  out[e] = v;
}

// FP64 -> three floats h + m + l equal to the value (53 <= 3 x 24 bits).
__global__ void k_to_f3(const double* __restrict__ in, int64_t count, float3* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const double x = in[e];
  const float h = (float)x;
  const double r = x - (double)h;
  const float m = (float)r;
  out[e] = make_float3(h, m, (float)(r - (double)m));
}

// out = shift * in + scale * (sum over splits of the float-float partials), in FP64.
__global__ void k_ff_finish(const float2* __restrict__ part, int ksplit, int64_t n, int nc, int ncols, double shift,
                            double scale, const double* __restrict__ in, int64_t ld_in, double* __restrict__ out,
                            int64_t ld_out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ncols) return;
  const int64_t i = e / ncols;
  const int c = (int)(e % ncols);
  ffv acc = {0.f, 0.f};
  for (int ks = 0; ks < ksplit; ++ks) {
    const float2 v = part[((int64_t)ks * n + i) * nc + c];
    acc = ff_add(acc, ffv{v.x, v.y});
  }
  out[i * ld_out + c] = shift * in[i * ld_in + c] + scale * ((double)acc.h + (double)acc.l);
}

template <int KIND, int D>
void launch_ff_nc(Launch L, int nc, const float3* pff, int64_t n, const float2* xff, int64_t jspan, int ksplit,
                  float2* part) {
  dim3 grid((unsigned)cdiv(n, RT), (unsigned)ksplit);
  const LogTable& t = log_table();
  switch (nc) {
    case 1: k_kmv_ff<KIND, D, 1><<<grid, RT, 0, L.st>>>(pff, n, xff, jspan, part, t); break;
    case 2: k_kmv_ff<KIND, D, 2><<<grid, RT, 0, L.st>>>(pff, n, xff, jspan, part, t); break;
    case 4: k_kmv_ff<KIND, D, 4><<<grid, RT, 0, L.st>>>(pff, n, xff, jspan, part, t); break;
    case 8: k_kmv_ff<KIND, D, 8><<<grid, RT, 0, L.st>>>(pff, n, xff, jspan, part, t); break;
    default: k_kmv_ff<KIND, D, 16><<<grid, RT, 0, L.st>>>(pff, n, xff, jspan, part, t); break;
  }
  if (L.counter) ++*L.counter;
}

int ff_group(int ncols) {
  int nc = 1;
  while (nc < ncols && nc < 16) nc *= 2;
  return nc;
}
int ff_splits(int64_t n, int split) {
  const int64_t blocks = cdiv(n, RT);
  int64_t ks = (split >= 1 && split <= 16) ? split : cdiv(4 * 152, blocks);
  ks = imax64(1, imin64(ks, cdiv(n, (int64_t)FOLD * JT)));
  return (int)ks;
}

}  // namespace

const LogTable& log_table() {
  static LogTable t;
  static std::once_flag once;
  std::call_once(once, [] {
    for (int q = 0; q < kLogTab; ++q) {
      const double c = 1.0 + (q + 0.5) / kLogTab;
      const float ic = (float)(1.0 / c);
      const double lc = -std::log((double)ic);
      t.ic[q] = ic;
      t.lch[q] = (float)lc;
      t.lcl[q] = (float)(lc - (double)t.lch[q]);
    }
  });
  return t;
}

int64_t ff_scratch_floats(int64_t n, int d, int ncols, int split) {
  const int nc = ff_group(ncols);
  return 4 * ((3 * n * d + 3) / 4) + 2 * (n * nc + (int64_t)ff_splits(n, split) * n * nc);
}

void launch_kernel_matvec_ff(Launch L, int kind, const double* pts, int d, int64_t n, double shift, double scale,
                             const double* in, int64_t ld_in, double* out, int64_t ld_out, int64_t ncols,
                             float* scratch, int split) {
  if (n <= 0 || ncols <= 0) return;
  const int ksplit = ff_splits(n, split);
  // a split covers whole folds of tiles
  const int64_t jspan = cdiv(cdiv(n, ksplit), (int64_t)FOLD * JT) * FOLD * JT;
  for (int64_t c0 = 0; c0 < ncols; c0 += 16) {
    const int nsrc = (int)imin64(16, ncols - c0);
    const int nc = ff_group(nsrc);
    float3* pff = reinterpret_cast<float3*>(scratch);
    float2* xff = reinterpret_cast<float2*>(scratch + 4 * ((3 * n * d + 3) / 4));
    float2* part = xff + n * nc;
    if (c0 == 0) {
      k_to_f3<<<(unsigned)cdiv(n * d, 256), 256, 0, L.st>>>(pts, n * d, pff);
      if (L.counter) ++*L.counter;
    }
    k_to_ff<<<(unsigned)cdiv(n * nc, 256), 256, 0, L.st>>>(in + c0, n, nsrc, ld_in, nc, xff);
    if (L.counter) ++*L.counter;
    if (kind == RSRS_OP_LOG2D) launch_ff_nc<RSRS_OP_LOG2D, 2>(L, nc, pff, n, xff, jspan, ksplit, part);
    else launch_ff_nc<RSRS_OP_INVR3D, 3>(L, nc, pff, n, xff, jspan, ksplit, part);
    const int64_t ksused = cdiv(n, jspan);
    k_ff_finish<<<(unsigned)cdiv(n * nsrc, 256), 256, 0, L.st>>>(part, (int)ksused, n, nc, nsrc, shift, scale,
                                                                  in + c0, ld_in, out + c0, ld_out);
    if (L.counter) ++*L.counter;
  }
}

}  // namespace rsrs
