// e^{i phi} in FP64 by the accurate-table method (Gal 1986; Tang, ACM TOMS
// 1989/1990): phi = j h + t with h = 2 pi / PH_N and |t| <= h/2, then
//   sin(jh + t) = s_j cos t + c_j sin t,  cos(jh + t) = c_j cos t - s_j sin t.
// j = rint(phi / h) by adding 1.5 * 2^52 (its low mantissa bits hold j, also
// for negative phi); t = phi - j C1 - j C2 with C1 = h rounded to 36 bits
// (j C1 exact for |j| < 2^17) and C2 = the next 53 bits of h (both from a
// 60-digit value of pi); |t| <= 0.0123, so the Taylor polynomials of degree 5
// (sin) and 6 (cos) are exact to 1e-17.  |phi| >= PH_MAX takes the library
// sincos.  Maximum error 2e-16 (checked against 40-digit values).
#pragma once
#include <cuda_runtime.h>

constexpr int PH_N = 256;
constexpr double PH_INV_H = 40.74366543152521;   // PH_N / (2 pi)
constexpr double PH_C1 = 0x1.921fb54440000p-6;   // 2 pi / PH_N, 36 bits
constexpr double PH_C2 = 0x1.68c234c4c6629p-45;  // 2 pi / PH_N - PH_C1
constexpr double PH_MAX = 3000.0;                // |j| < 2^17
constexpr double PH_ROUND = 6755399441055744.0;  // 1.5 * 2^52

// table (cos, sin)(2 pi j / PH_N), j < PH_N, in shared memory; the caller
// synchronises before the first use
__device__ __forceinline__ void phase_table_fill(double2* tab) {
  for (int j = threadIdx.x; j < PH_N; j += blockDim.x) {
    double sv, cv;
    sincospi(2.0 * j / PH_N, &sv, &cv);
    tab[j] = make_double2(cv, sv);
  }
}

__device__ __forceinline__ void sincos_table(double phi, const double2* __restrict__ tab, double* sn,
                                             double* cs) {
  if (!(fabs(phi) < PH_MAX)) {
    sincos(phi, sn, cs);
    return;
  }
  const double big = fma(phi, PH_INV_H, PH_ROUND);
  const int j = __double2loint(big) & (PH_N - 1);
  const double jd = big - PH_ROUND;
  double t = fma(-jd, PH_C1, phi);
  t = fma(-jd, PH_C2, t);
  const double t2 = t * t;
  const double st = fma(fma(0x1.1111111111111p-7, t2, -0x1.5555555555555p-3) * t2, t, t);  // t - t^3/6 + t^5/120
  const double ct = fma(fma(fma(-0x1.6c16c16c16c17p-10, t2, 0x1.5555555555555p-5), t2, -0.5), t2, 1.0);
  const double2 e = tab[j];  // (cos, sin)(j h)
  *sn = fma(e.y, ct, e.x * st);
  *cs = fma(e.x, ct, -(e.y * st));
}
