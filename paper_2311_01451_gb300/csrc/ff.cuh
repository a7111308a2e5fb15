// Float-float arithmetic on the FP32 pipe: an unevaluated sum h + l of two FP32 numbers with
// |l| <= ulp(h)/2 (48 significant bits).  Error-free transformations: Knuth's TwoSum, Dekker's
// FastTwoSum (|a| >= |b|) and TwoProduct through the fused multiply-add.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace rsrs {

struct ffv {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// a + b with both pairs' rounding errors kept (Bailey's accurate addition).
__device__ __forceinline__ ffv ff_add(ffv a, ffv b) {
  float s, e, t, f;
  two_sum(a.h, b.h, s, e);
  two_sum(a.l, b.l, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return {s, e};
}

// ---- kernel values in float-float (the refinement residual products) ----------------------------
// Sum of two non-negative values (no cancellation): one TwoSum suffices.
__device__ __forceinline__ ffv ff_add_pos(ffv a, ffv b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  fast_two_sum(s, e, s, e);
  return {s, e};
}
// a - b for coordinates held exactly as three floats (h + m + l = the FP64 value): the two
// leading differences are split exactly by TwoSum and summed in float-float, so the result is
// accurate to 2^-48 of |a - b| however close the points are.
__device__ __forceinline__ ffv coord_diff(float3 a, float3 b) {
  float s, e, t, f;
  two_sum(a.x, -b.x, s, e);
  two_sum(a.y, -b.y, t, f);
  ffv d = ff_add(ffv{s, e}, ffv{t, f});
  d.l = __fadd_rn(d.l, __fsub_rn(a.z, b.z));
  fast_two_sum(d.h, d.l, d.h, d.l);
  return d;
}
__device__ __forceinline__ ffv ff_sqr(ffv a) {
  float p, e;
  two_prod(a.h, a.h, p, e);
  e = __fmaf_rn(__fmul_rn(2.f, a.h), a.l, e);
  fast_two_sum(p, e, p, e);
  return {p, e};
}

constexpr int kLogTab = 256;
struct LogTable {
  float ic[kLogTab];   // fl(1 / (1 + (t + 1/2) / 256))
  float lch[kLogTab];  // -log(ic[t]) = log(1 / ic[t]), high part
  float lcl[kLogTab];  // low part
};
// ln 2 to 48 bits
constexpr float kLn2H = 0.693147182464599609375f;
constexpr float kLn2L = -1.904654323148236e-09f;

__device__ __forceinline__ ffv ff_log(ffv x, const LogTable& T) {
  const int bits = __float_as_int(x.h);
  const int e = ((bits >> 23) & 0xFF) - 127;
  const float mh = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);
  const float ml = __fmul_rn(x.l, __int_as_float((127 - e) << 23));  // x.l * 2^-e, exact
  const int t = (bits >> 15) & 0xFF;
  const float ic = T.ic[t];
  // u = m ic - 1
  float p, pe;
  two_prod(mh, ic, p, pe);
  pe = __fmaf_rn(ml, ic, pe);
  float uh, ul;
  two_sum(__fsub_rn(p, 1.f), pe, uh, ul);  // p - 1 is exact (p within 2^-8 of 1)
  // q = u^2, c = u^3 / 3
  float qh, ql;
  two_prod(uh, uh, qh, ql);
  ql = __fmaf_rn(__fmul_rn(2.f, uh), ul, ql);
  float ch, cl;
  two_prod(qh, uh, ch, cl);
  cl = __fmaf_rn(qh, ul, cl);
  cl = __fmaf_rn(ql, uh, cl);
  const float c3h = __fmul_rn(ch, 1.f / 3.f);
  const float c3l = __fmul_rn(__fadd_rn(__fmaf_rn(-3.f, c3h, ch), cl), 1.f / 3.f);
  const float poly = __fmaf_rn(uh, __fmaf_rn(uh, __fmaf_rn(uh, 1.f / 7.f, -1.f / 6.f), 1.f / 5.f), -0.25f);
  const float tail = __fmul_rn(__fmul_rn(qh, qh), poly);
  ffv a;
  fast_two_sum(c3h, __fadd_rn(c3l, tail), a.h, a.l);
  a = ff_add(a, ffv{-0.5f * qh, -0.5f * ql});
  a = ff_add(a, ffv{uh, ul});
  a = ff_add(a, ffv{T.lch[t], T.lcl[t]});
  ffv el;
  two_prod((float)e, kLn2H, el.h, el.l);
  el.l = __fmaf_rn((float)e, kLn2L, el.l);
  return ff_add(el, a);
}

__device__ __forceinline__ ffv ff_rsqrt(ffv x) {
  const float y = rsqrtf(x.h);
  float y2h, y2l;
  two_prod(y, y, y2h, y2l);
  float p, pe;
  two_prod(x.h, y2h, p, pe);
  pe = __fmaf_rn(x.h, y2l, pe);
  pe = __fmaf_rn(x.l, y2h, pe);
  const float h = __fsub_rn(__fsub_rn(1.f, p), pe);  // 1 - p is exact (p within 2^-21 of 1)
  // (1 - h)^-1/2 = 1 + h/2 + 3h^2/8 + O(h^3), |h| <= 2^-21
  const float corr = __fmul_rn(y, __fmaf_rn(__fmul_rn(0.375f, h), h, __fmul_rn(0.5f, h)));
  ffv r;
  fast_two_sum(y, corr, r.h, r.l);
  return r;
}

// The log table of ff_log (host side, built once from the host's FP64 log).
const LogTable& log_table();

// FP64 -> three floats h + m + l equal to the value (53 <= 3 x 24 bits).
__device__ __forceinline__ float3 f64_to_f3(double x) {
  const float h = (float)x;
  const double r = x - (double)h;
  const float m = (float)r;
  return make_float3(h, m, (float)(r - (double)m));
}

}  // namespace rsrs
