// Float-float arithmetic: a value is hi + lo with two FP32 numbers,
// |lo| <= ulp(hi)/2, about 48 significant bits.  Error-free transformations
// after Dekker (1971) and Knuth (TAOCP vol. 2): TwoSum, FastTwoSum and
// TwoProduct (with an FMA); square root and division by one Karp-Markstein
// correction of the correctly rounded FP32 result (Karp & Markstein, ACM
// TOMS 1997).  The intrinsics __fadd_rn / __fmul_rn keep the compiler from
// contracting the operations these transformations rely on.
//
// Used where an FP64-accurate result is needed but B300's FP64 pipe (2 lanes
// per clock per SM against 128 for FP32) would be the bottleneck.
#pragma once
#include <cuda_runtime.h>

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// a + b, error <= ~2^-47 (|a| + |b|)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  const ff s = ff_two_sum(a.hi, b);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// a * b, error <= ~2^-47 |a b|
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const ff p = ff_two_prod(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return ff_fast_two_sum(p.hi, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const ff p = ff_two_prod(a.hi, b);
  return ff_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// a * 2^k scalings are exact: use ff_mul_f with 0.5f, 2.0f

// sqrt(a), a > 0: y = sqrt_rn(hi), then y + (a - y^2)/(2y)
__device__ __forceinline__ ff ff_sqrt(ff a) {
  const float y = __fsqrt_rn(a.hi);
  const ff y2 = ff_two_prod(y, y);
  const float r = __fadd_rn(__fadd_rn(__fsub_rn(a.hi, y2.hi), -y2.lo), a.lo);  // a - y^2 (exact head)
  return ff_fast_two_sum(y, __fmul_rn(r, __fdiv_rn(0.5f, y)));
}

// a / b: q = hi(a)/hi(b), then q + (a - q b)/hi(b)
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q = __fdiv_rn(a.hi, b.hi);
  const ff qb = ff_mul_f(b, q);
  const ff r = ff_sub(a, qb);
  return ff_fast_two_sum(q, __fdiv_rn(r.hi, b.hi));
}

__device__ __forceinline__ ff ff_rcp(ff b) { return ff_div(ff{1.0f, 0.0f}, b); }

// e^{i phi} in float-float for |phi| < FF_PHI_MAX, by the accurate-table
// method as in phase.cuh: phi = j h + t, h = 2 pi / 256 = FF_H1 + FF_H2 + FF_H3
// (FF_H1 has 8 significant bits, so j FF_H1 is exact for |j| < 2^16; the three
// parts leave 1.3e-21 of h, from a 60-digit value of pi), |t| <= h/2 = 0.0123;
// sin t = t + t(-t^2/6 + t^4/120 - t^6/5040), cos t = 1 - t^2/2 + t^4/24 - t^6/720
// (the next terms are below 1e-20); the t^4 and t^6 terms are below 2e-10 and
// need only FP32.  tab[j] = (cos hi, cos lo, sin hi, sin lo)(j h).
constexpr float FF_INV_H = 40.743664f;         // 256 / (2 pi)
constexpr float FF_H1 = 0x1.92p-6f;
constexpr float FF_H2 = 0x1.fb5444p-18f;
constexpr float FF_H3 = 0x1.68c234p-45f;
constexpr float FF_PHI_MAX = 1000.0f;
constexpr float FF_C3_HI = -0.16666667f;       // -1/6 = hi + lo
constexpr float FF_C3_LO = 4.967054e-09f;

__device__ __forceinline__ void ff_phase_table_fill(float4* tab) {
  for (int j = threadIdx.x; j < 256; j += blockDim.x) {
    double sv, cv;
    sincospi(j / 128.0, &sv, &cv);
    const ff c = ff_from_double(cv), s = ff_from_double(sv);
    tab[j] = make_float4(c.hi, c.lo, s.hi, s.lo);
  }
}

__device__ __forceinline__ void ff_sincos(ff phi, const float4* __restrict__ tab, ff* sn, ff* cs) {
  if (!(fabsf(phi.hi) < FF_PHI_MAX)) {
    double s, c;
    sincos(ff_to_double(phi), &s, &c);
    *sn = ff_from_double(s);
    *cs = ff_from_double(c);
    return;
  }
  const float jf = rintf(__fmul_rn(phi.hi, FF_INV_H));
  const int j = ((int)jf) & 255;
  ff t = ff_two_sum(__fmaf_rn(-jf, FF_H1, phi.hi), phi.lo);  // the head difference is exact
  t = ff_sub(t, ff_two_prod(jf, FF_H2));
  t = ff_add_f(t, __fmul_rn(-jf, FF_H3));
  const ff t2 = ff_mul(t, t);
  const float q = t2.hi;
  const float vs = __fmul_rn(__fmul_rn(q, q), __fmaf_rn(-q, 1.0f / 5040.0f, 1.0f / 120.0f));
  const ff w = ff_add_f(ff_mul(t2, ff{FF_C3_HI, FF_C3_LO}), vs);
  const ff st = ff_add(t, ff_mul(t, w));
  const float vc = __fmul_rn(__fmul_rn(q, q), __fmaf_rn(-q, 1.0f / 720.0f, 1.0f / 24.0f));
  const ff u = ff_add_f(ff_mul_f(t2, -0.5f), vc);
  const ff ct = ff_add(ff{1.0f, 0.0f}, u);
  const float4 e = tab[j];
  const ff cj{e.x, e.y}, sj{e.z, e.w};
  *sn = ff_add(ff_mul(sj, ct), ff_mul(cj, st));
  *cs = ff_sub(ff_mul(cj, ct), ff_mul(sj, st));
}
