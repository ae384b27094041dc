// Self-block assembly (Sec. 3.1-3.4): one row of the combined-layer self block per CTA,
//   A_b[t, (i,l,j)] = 1/2 delta + int_{panel i} P_l(s) [F^D_j(s) + |J_ilj| F^S_j(s)] ds,
//   F^D_j = int [(|J| n_r) K^r + (|J| n_z) K^z] L_j dtheta,  F^S_j = -i eta int G L_j dtheta,
// for every panel i within one of the target's panel (Eq. sx); farther panels
// take the plain smooth rule.  The double layer integrates the exact
// area-weighted normal |J| n_r = a0 + a1 cos theta, |J| n_z = b0 + b1 cos theta
// + b2 sin theta (arc-axis bodies: r l'(1 - kappa r cos theta) and -r r'; the
// paper's horizontal-ring shapes: r z' and -r (r' + x_c' cos + y_c' sin))
// against an interpolant of mu; the single layer keeps the interpolant of
// mu |J| (the paper's); on bodies of revolution the two coincide.
//
// Azimuthal integrals come from the modal Green's functions (Eq. modalgreen)
// of the source ring at s:
//   static part  g^_m = Q_{m-1/2}(chi)/(2 pi sqrt(r r~)) (Eq. modal0), Q by the
//                recursion of Eq. leg_recur (forward near chi = 1, Miller's
//                backward recursion on ratios otherwise), Q' by Eq. dleg_recur;
//   k != 0       G^_m = (1/2pi) sum_n f1^_n g^_{m-n} + i f2^_m (Eqs. conv, I1),
//                and the same split for the source derivatives; the smooth
//                factors cos(k rho), sinc(k rho) and
//                (k rho cos k rho - sin k rho)/(k rho)^3 are transformed by a
//                cosine DFT (all kernels are even in phi = theta - alpha).
// The theta-coefficients of both integrands (k^_|m| e^{-i m alpha}, cos(theta)
// averaging neighbouring modes) are accumulated over the outer nodes of a
// panel, weighted by w P_l(s); the inverse DFT against L_j (Sec. 3.1) runs
// once per panel instead of once per outer node.
//
// The outer s-integral replaces the paper's generalised Gaussian tables (not
// available) with a composite rule: dyadic sub-panels toward the
// (near-)singular point with max(2 order + 4, 36) Gauss-Legendre nodes on the
// outermost (where P_l varies fastest next to the panel end), max(order + 4, 20)
// on the next and 12 on the inner ones, and a graded innermost panel (u^6
// substitution, 20 nodes) for the logarithm.  Ring-target geometry uses
// difference formulas in h = s - s_t so that r - r~ and c keep full relative
// precision as h -> 0 (the double-layer pieces each grow like 1/|h| and cancel).
#include <algorithm>
#include <cmath>

#include "ffloat.cuh"
#include "phase.cuh"
#include "qams_internal.h"

namespace {

constexpr int NT = 128;      // threads per CTA
constexpr int BATCH = 32;    // most outer nodes whose recursions run together (lanes of warp 0)
constexpr int MAXP = 96;     // highest static mode N + n1 + 1
constexpr int MAXM2 = 72;    // M/2 + 1 samples of the smooth factors
constexpr int MAXN1 = 64;    // highest smooth-factor mode + 2 (k r_max up to ~35)
constexpr int MAXN = 32;     // N = n_theta / 2
constexpr int MAXORD = 19;
constexpr int MILLER_MAX = 768;  // start indices of Miller's recurrence (tabulated coefficients)
constexpr int MAXE = (MAXORD * 2 * MAXN + NT - 1) / NT;  // panel entries per thread

// The outer nodes of a row come in at most four pieces (the self panel split
// at s_t, one piece per neighbour), each K dyadic levels toward its singular
// end plus a graded innermost panel; nodes are generated from these
// descriptors when a batch needs them.
struct alignas(16) RowShared {
  double rowc[8];               // row constants: cos, sin(theta_t); sin, cos(s_t); u_t, rho(u_t); r_t
  double pc_h0[4], pc_L[4];     // piece start (offset from s_t) and signed length
  int pc_K[4], pc_panel[4], pc_self[4], pc_end[4];  // levels, panel, u^6-graded innermost, cumulative node count
  int npc, nq;
  // per-batch node data (filled by warp 0; Q and dQ/dchi live in dynamic shared memory)
  double bs[BATCH][18];         // scalars
  double bw[BATCH];             // outer weights
  int bp[BATCH];                // panels
  int bflush[BATCH];            // 1 on the last outer node of a panel
  // per-node work arrays
  double sg0[MAXP + 1], sdq[MAXP + 1];  // static g^ and Q'(chi) scale (modes 0..P)
  float2 fs[3][MAXM2];          // samples of cos(k rho), sinc(k rho), q3(k rho) (float-float)
  double fc[3][MAXN1 + 1];      // their cosine coefficients
  double pr[MAXN1 + 1], pz[MAXN1 + 1], f2[MAXN1 + 1];
  double cA[MAXN + 2], cBr[MAXN + 2], cBz[MAXN + 2], cC[MAXN + 3];  // the phi-convolutions (stage D)
  float4 gff[3][MAXN + 2];  // G^, d_r G^, d_z G^ (phi coefficients, m <= N+1): re hi, re lo, im hi, im lo
  float4 eff[MAXN + 2];     // (cos hi, cos lo, sin hi, sin lo)(m alpha)
  double ecs[8 + (MAXN + 9) / 8], esn[8 + (MAXN + 9) / 8];  // cos/sin(j alpha), j < 8, then of 8 l alpha
  double dre[2 * MAXN], dim_[2 * MAXN];        // theta-coefficients of the double-layer integrand
  double tre[2 * MAXN], tim[2 * MAXN];         // theta-coefficients of the single-layer integrand
  double pl[MAXORD];
  // row constants
  double s2tab[MAXM2];     // sin^2(pi q / M)
  float2 ctab[2 * MAXM2];  // cos(2 pi j / M), j < M (float-float)
  double cth[2 * MAXN], sth[2 * MAXN];
  double inv_odd[MAXP + 1];  // 1/(2n - 1)
  // float-float copies for the accumulation and the panel's inverse DFT
  float4 dff[2 * MAXN], tff[2 * MAXN];  // theta-coefficients (re hi, re lo, im hi, im lo)
  float4 csff[2 * MAXN];                // (cos hi, cos lo, sin hi, sin lo)(2 pi j / 2N)
  float2 plff[MAXORD];                  // outer weight x P_l
  float2 fcff[2][MAXN1 + 1];            // cos^ and sinc^ coefficients (convolution inputs)
  float2 sg0ff[MAXP + 1], srff[MAXP + 1], szff[MAXP + 1];  // g^, dchi_r Q' scale, dchi_z Q' scale
};

struct AsmBody {
  int n_panels, order, n_theta, n_modes;
  int kind, n_terms;  // profile kind; kind 1: terms per series
  int ser, brk;       // table offsets: kind-1 series [4][n_terms][3], panel breaks [n_panels+1]
  double base, L, kappa;
  double a[8], b[8];
  long long offset;  // first node of the body
  long long crow;    // first row of the body among the assembled rows
  long long blk;     // first entry of the body's self block
  int n1, M;       // smooth-factor bandwidth and cosine-DFT size
  int rule;        // offset of the order's rule tables
};

__device__ __forceinline__ double rho_prof(const AsmBody& B, double u) {
  double s = 1.0;
  for (int m = 1; m <= B.n_modes; ++m) {
    double sn, cs;
    sincospi(2.0 * m * u, &sn, &cs);
    s += B.a[m - 1] * cs + B.b[m - 1] * sn;
  }
  return B.base * s;
}

// complete elliptic integrals K, E of modulus mu (mu_c = sqrt(1 - mu^2)) by the AGM
__device__ void agm_KE(double mu, double mu_c, double* K, double* E) {
  double a = 1.0, b = mu_c, c = mu;
  double s = 0.5 * c * c, p = 0.5;
  for (int it = 0; it < 40; ++it) {
    const double an = 0.5 * (a + b);
    const double bn = sqrt(a * b);
    c = 0.25 * c * c / an;
    a = an;
    b = bn;
    p *= 2.0;
    s += p * c * c;
    if (c < 1e-18 * a) break;
  }
  *K = M_PI / (2.0 * a);
  *E = *K * (1.0 - s);
}

// cos x, sin(x)/x and (x cos x - sin x)/x^3 from one sincos (accurate-table method of
// phase.cuh with the table `ptab` in global memory; Taylor series near 0)
__device__ __forceinline__ void smooth_factors(double x, const double2* __restrict__ ptab, double* c, double* sinc,
                                               double* q3) {
  double sn, cs;
  sincos_table(x, ptab, &sn, &cs);
  *c = cs;
  const double ax = fabs(x);
  if (ax < 0.5) {
    const double x2 = x * x;
    *sinc = ax < 0.1 ? 1.0 - x2 / 6.0 + x2 * x2 / 120.0 - x2 * x2 * x2 / 5040.0 + x2 * x2 * x2 * x2 / 362880.0
                     : sn / x;
    double term = 1.0, sum = 0.0, fact = 6.0, sign = -1.0;
    for (int n = 1; n <= 12; ++n) {
      if (n > 1) fact *= (2.0 * n) * (2.0 * n + 1.0);
      sum += sign * (2.0 * n) / fact * term;
      term *= x2;
      sign = -sign;
    }
    *q3 = sum;
    return;
  }
  const double inv = 1.0 / x;
  *sinc = sn * inv;
  *q3 = (x * cs - sn) * inv * inv * inv;
}


// Lane work: geometry of the ring at s_t + h seen from (s_t, theta_t) and the
// static modal sequence.  Scalars: 0 r, 1 rt, 2 c, 3 dr, 4 alpha, 5 scale,
// 6 dchi_r, 7 dchi_z, 8 s, 9..13 the area-weighted normal
//   |J| n_r = a0 + a1 cos theta,  |J| n_3 = b0 + b1 cos theta + b2 sin theta
// (9 a0, 10 a1, 11 b0, 12 b1, 13 b2), 14 far flag, 15 cos(alpha), 16 sin(alpha).
// Rings with eta N >= FAR_ETA_N (eta = acosh chi) are far enough from the
// target that the kernels are resolved by the 2N azimuthal nodes to 1e-14
// (checked against the modal evaluation): their Lagrange weights are the
// trapezoidal values (pi/N) K(theta_j), and the modal machinery (recursion,
// transforms, convolution) is skipped -- the paper's modal technique is for
// rings close to the target.
constexpr double FAR_ETA_N = 48.0;
constexpr double INV_2PI = 0.15915494309189533577;
constexpr double INV_4PI = 0.079577471545947667884;

// kind-1 series at s: f, f' and the drop f(s_t) - f(s) by sum-to-product,
//   cos w s_t - cos w s = 2 sin(w m) sin(w h/2),  sin w s_t - sin w s = -2 cos(w m) sin(w h/2),
// m = s_t + h/2, so the drop keeps relative precision as h -> 0.
__device__ __forceinline__ void series_at(const double* T, int nt, double s, double mid, double h, double* f,
                                          double* df, double* drop) {
  double v = 0.0, dv = 0.0, dp = 0.0;
  for (int j = 0; j < nt; ++j) {
    const double om = T[3 * j], A = T[3 * j + 1], Bs = T[3 * j + 2];
    double sn, cs, sm, cm;
    sincos(om * s, &sn, &cs);
    sincos(om * mid, &sm, &cm);
    v += A * cs + Bs * sn;
    dv += om * (Bs * cs - A * sn);
    dp += 2.0 * sin(0.5 * om * h) * (A * sm - Bs * cm);
  }
  *f = v;
  *df = dv;
  *drop = dp;
}

__device__ void ring_node(const AsmBody& B, const double* __restrict__ tab, double s_t, double th_t, double h,
                          int P, int Nhalf, const double* __restrict__ inv_odd, double* q, double* dq, double* sc,
                          const double* off, const double* rowc) {
  const double s = s_t + h;
  const double sh = sin(0.5 * h);
  const double mid = s_t + 0.5 * h;
  double r, rt, c, dr, alpha, a0, a1, b0, b1, b2, ca, sa;
  const double ct = rowc[0], st = rowc[1];
  if (B.kind == 1) {
    const int nt = B.n_terms;
    const double* T = tab + B.ser;
    double f[4], df[4], drop[4];
    for (int qq = 0; qq < 4; ++qq) series_at(T + 3 * nt * qq, nt, s, mid, h, &f[qq], &df[qq], &drop[qq]);
    const double r_t = rowc[6];
    r = f[3];
    c = drop[2];
    const double dx = drop[0], dy = drop[1];
    const double a = r_t * ct + dx;
    const double b = r_t * st + dy;
    rt = hypot(a, b);
    const double drt = (2.0 * r_t * (ct * dx + st * dy) + dx * dx + dy * dy) / (rt + r_t);  // r~ - r_t
    dr = -drop[3] - drt;
    double ao = a, bo = b;
    if (off) {
      // off-surface target y_t + v (v = nu n^ in the body frame, which is every ring's frame here)
      ao = a + off[0];
      bo = b + off[1];
      const double rto = hypot(ao, bo);
      dr -= (2.0 * (a * off[0] + b * off[1]) + off[0] * off[0] + off[1] * off[1]) / (rto + rt);
      rt = rto;
      c += off[2];
    }
    alpha = atan2(bo, ao);
    ca = ao / rt;
    sa = bo / rt;
    a0 = r * df[2];
    a1 = 0.0;
    b0 = -r * df[3];
    b1 = -r * df[0];
    b2 = -r * df[1];
  } else {
    const double u_t = rowc[4], rho_t = rowc[5], r_t = rowc[6];
    double sin_s, cos_s, sin_mid, cos_mid;
    sincos(s, &sin_s, &cos_s);
    sincos(mid, &sin_mid, &cos_mid);
    const double u = 0.5 * (1.0 + sin_s);
    const double du = cos_mid * sh;  // u - u_t
    // profile at u and its u-derivative, and rho(u) - rho(u_t) by sum-to-product,
    //   cos 2pi m u - cos 2pi m u_t = -2 sin(pi m (u + u_t)) sin(pi m du),
    //   sin 2pi m u - sin 2pi m u_t =  2 cos(pi m (u + u_t)) sin(pi m du),
    // with the multiples of each angle by the angle-addition recurrence (m <= 8)
    double s1, c1, sA, cA, sD, cD;
    sincospi(2.0 * u, &s1, &c1);
    sincospi(u + u_t, &sA, &cA);
    sincospi(du, &sD, &cD);
    double cm = c1, sm = s1, cAm = cA, sAm = sA, cDm = cD, sDm = sD;
    double prof = 1.0, dprof = 0.0, drho = 0.0;
    for (int m = 1; m <= B.n_modes; ++m) {
      const double am = B.a[m - 1], bm = B.b[m - 1];
      prof += am * cm + bm * sm;
      dprof += 2.0 * M_PI * m * (bm * cm - am * sm);
      drho += 2.0 * sDm * (bm * cAm - am * sAm);
      double t = cm * c1 - sm * s1;
      sm = sm * c1 + cm * s1;
      cm = t;
      t = cAm * cA - sAm * sA;
      sAm = sAm * cA + cAm * sA;
      cAm = t;
      t = cDm * cD - sDm * sD;
      sDm = sDm * cD + cDm * sD;
      cDm = t;
    }
    drho *= B.base;
    const double rho_s = B.base * prof;
    r = rho_s * cos_s;
    const double dr_t = drho * cos_s + rho_t * (-2.0 * sin_mid * sh);
    const double Delta = -B.L * cos_mid * sh;
    const double kd = B.kappa * Delta;
    double sh2, ch2;
    sincos(0.5 * kd, &sh2, &ch2);
    const double skd = 2.0 * sh2 * ch2, ckd = 1.0 - 2.0 * sh2 * sh2;
    const double sinc_h = fabs(kd) > 1e-8 ? sh2 / (0.5 * kd) : 1.0;
    const double sinc_f = fabs(kd) > 1e-8 ? skd / kd : 1.0;
    const double omc = 0.5 * B.kappa * Delta * Delta * sinc_h * sinc_h;
    const double a = omc + r_t * ct * ckd;
    const double b = r_t * st;
    c = Delta * sinc_f - r_t * ct * skd;
    rt = hypot(a, b);
    const double d2 = -(r_t * ct * skd) * (r_t * ct * skd) + 2.0 * r_t * ct * ckd * omc + omc * omc;
    dr = dr_t - d2 / (rt + r_t);
    double ao = a, bo = b;
    if (off) {
      // off-surface target y_t + v, v = (v1, v2, v3) in the target's frame (e1, e2, e3)(s_t);
      // moving along the axis by Delta turns e1, e3 by kappa Delta about e2:
      //   e1(s_t) = cos e1(s) - sin e3(s),  e3(s_t) = sin e1(s) + cos e3(s)
      const double va = off[0] * ckd + off[2] * skd, vb = off[1], vc = -off[0] * skd + off[2] * ckd;
      ao = a + va;
      bo = b + vb;
      const double rto = hypot(ao, bo);
      dr -= (2.0 * (a * va + b * vb) + va * va + vb * vb) / (rto + rt);
      rt = rto;
      c += vc;
    }
    alpha = atan2(bo, ao);
    ca = ao / rt;
    sa = bo / rt;
    const double dl = 0.5 * B.L * cos_s;                                       // l'(s)
    const double rp = B.base * dprof * 0.5 * cos_s * cos_s - rho_s * sin_s;    // r'(s)
    a0 = r * dl;
    a1 = -B.kappa * r * r * dl;
    b0 = -r * rp;
    b1 = 0.0;
    b2 = 0.0;
  }

  double delta = (dr * dr + c * c) / (2.0 * r * rt);
  if (delta < 1e-300) delta = 1e-300;
  const double chi = 1.0 + delta;
  const double eta = log1p(delta + sqrt(delta * (2.0 + delta)));
  // ring scalars (also the far path's inputs)
  sc[0] = r;
  sc[1] = rt;
  sc[2] = c;
  sc[3] = dr;
  sc[4] = alpha;
  sc[5] = 1.0 / (2.0 * M_PI * sqrt(r * rt));
  sc[6] = (dr * (r + rt) - c * c) / (2.0 * rt * r * r);
  sc[7] = -c / (r * rt);
  sc[8] = s;
  sc[9] = a0;
  sc[10] = a1;
  sc[11] = b0;
  sc[12] = b1;
  sc[13] = b2;
  sc[14] = (eta * Nhalf >= FAR_ETA_N) ? 1.0 : 0.0;
  sc[15] = rt > 0.0 ? ca : 1.0;  // cos(alpha)
  sc[16] = rt > 0.0 ? sa : 0.0;  // sin(alpha)
  if (sc[14] != 0.0) return;
  const double mu = sqrt(2.0 / (2.0 + delta));
  const double mu_c = sqrt(delta / (2.0 + delta));
  double K, E;
  agm_KE(mu, mu_c, &K, &E);
  q[0] = mu * K;
  if (eta * P <= 3.0) {
    if (P >= 1) q[1] = chi * mu * K - sqrt(2.0 * (chi + 1.0)) * E;
    // (2n-1) q_n = 4 (n-1) chi q_{n-1} - (2n-3) q_{n-2}; counters carried in FP64, 1/(2n-1) from a table
    double fn1 = 1.0, f2n3 = 1.0;
    for (int n = 2; n <= P; ++n) {
      q[n] = (4.0 * fn1 * chi * q[n - 1] - f2n3 * q[n - 2]) * inv_odd[n];
      fn1 += 1.0;
      f2n3 += 2.0;
    }
  } else {
    // Miller's algorithm: the backward recurrence
    //   q_{n-2} = alpha_n chi q_{n-1} - beta_n q_n,  alpha_n = 4(n-1)/(2n-3), beta_n = (2n-1)/(2n-3)
    // (coefficients tabulated at the head of `tab`: no division in the loop) from
    // q_{n_start} = 0, q_{n_start-1} = 1, rescaled by 2^-600 whenever it passes 2^600, then
    // normalised by q_0 = mu K.  The error at index n <= P decays like e^{-2 (n_start - n) eta}
    // (minimal against dominant solution), so n_start = P + 10 + 20/eta leaves e^{-40}
    // (eta P > 3 here, so n_start < P + 11 + 20 P/3 < MILLER_MAX).
    int n_start = P + 10 + (int)ceil(20.0 / eta);
    if (n_start > MILLER_MAX - 1) n_start = MILLER_MAX - 1;
    double qn = 0.0, qn1 = 1.0;  // q_n, q_{n-1}
    for (int n = n_start; n >= 2; --n) {
      const double qm = tab[2 * n] * chi * qn1 - tab[2 * n + 1] * qn;  // q_{n-2}
      qn = qn1;
      qn1 = qm;
      if (n - 2 <= P) q[n - 2] = qm;
      if ((__double2hiint(qm) & 0x7fffffff) > 0x65700000) {  // |q| > 2^600
        qn *= 0x1p-600;
        qn1 *= 0x1p-600;
        for (int m = max(n - 2, 0); m <= P; ++m) q[m] *= 0x1p-600;
      }
    }
    const double s0 = q[0] != 0.0 ? mu * K / q[0] : 0.0;
    for (int n = 1; n <= P; ++n) q[n] *= s0;
    q[0] = mu * K;
  }
  const double half_inv = 0.5 / (delta * (2.0 + delta));  // 1 / (2 (chi^2 - 1))
  for (int m = 0; m <= P; ++m) {
    const double prev = m == 0 ? q[1] : q[m - 1];
    dq[m] = (2.0 * m - 1.0) * half_inv * (chi * q[m] - prev);
  }
}

// plain smooth combined-layer kernel (far panels of the same body)
__device__ void smooth_kernel(const qd4& x, const qd4& y, const qd4& n, double k, double eta,
                              const double2* __restrict__ ptab, double* kre, double* kim) {
  const double dx = y.x - x.x, dy = y.y - x.y, dz = y.z - x.z;
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double rinv = rsqrt(r2);
  double sn, cs;
  sincos_table(k * r2 * rinv, ptab, &sn, &cs);
  const double nyx = n.x * dx + n.y * dy + n.z * dz;
  const double are = -nyx * rinv * rinv, aim = k * nyx * rinv - eta;
  const double f = rinv * 0.079577471545947667884;
  *kre = (cs * are - sn * aim) * f;
  *kim = (sn * are + cs * aim) * f;
}

// complex float-float helpers
struct ffc {
  ff re, im;
};
__device__ __forceinline__ ffc ffc_load(float4 v) { return {ff{v.x, v.y}, ff{v.z, v.w}}; }
__device__ __forceinline__ ffc ffc_mul(ffc a, ffc b) {
  return {ff_sub(ff_mul(a.re, b.re), ff_mul(a.im, b.im)), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
// e^{-i m alpha} from (cos, sin)(|m| alpha): cos - i sin for m >= 0, cos + i sin otherwise
__device__ __forceinline__ ffc ephase(float4 cs, bool nonneg) {
  const ff c{cs.x, cs.y}, sn{cs.z, cs.w};
  return {c, nonneg ? ff_neg(sn) : sn};
}

// Nodes of the two outermost dyadic levels of a piece: they carry the Lagrange
// factor P_l across half (and a quarter) of the piece, so they grow with the order,
// with a floor for long low-order panels where the kernel itself varies on that scale.
__host__ __device__ __forceinline__ int level0_nodes(int order) { return 2 * order + 4 > 36 ? 2 * order + 4 : 36; }
__host__ __device__ __forceinline__ int level1_nodes(int order) { return order + 4 > 20 ? order + 4 : 20; }

// Rule tables of one order (see qams_assemble_launch for the layout).
struct Rules {
  const double *d0_x, *d0_w, *dy_x, *dy_w, *g12_x, *g12_w, *in_x, *in_w, *ad_x, *ad_w;
};

// Outer node `idx` of the row: offset h = s - s_t, weight, panel and whether it
// ends its panel.  Same arithmetic, node for node, as writing the pieces out.
__device__ void outer_node(const RowShared& S, const Rules& R, int order, int idx, double* h, double* w, int* panel,
                           int* flush) {
  int pc = 0;
  while (pc + 1 < S.npc && idx >= S.pc_end[pc]) ++pc;
  *panel = S.pc_panel[pc];
  *flush = (idx == S.pc_end[pc] - 1) && (pc + 1 == S.npc || S.pc_panel[pc + 1] != S.pc_panel[pc]);
  int j = idx - (pc > 0 ? S.pc_end[pc - 1] : 0);
  const double h0 = S.pc_h0[pc], L = S.pc_L[pc], aL = fabs(L);
  const int K = S.pc_K[pc];
  const int n0 = level0_nodes(order), n1l = level1_nodes(order);
  double top = 1.0;
  for (int kk = 0; kk < K; ++kk) {
    const int nk = kk == 0 ? n0 : (kk == 1 ? n1l : 12);
    const double bot = 0.5 * top;
    if (j < nk) {
      const double* kx = kk == 0 ? R.d0_x : (kk == 1 ? R.dy_x : R.g12_x);
      const double* kw = kk == 0 ? R.d0_w : (kk == 1 ? R.dy_w : R.g12_w);
      const double v = bot + (top - bot) * kx[j];
      *h = h0 + L * v;
      *w = (top - bot) * kw[j] * aL;
      return;
    }
    j -= nk;
    top = bot;
  }
  const bool self = S.pc_self[pc] != 0;
  const double uu = (self ? R.in_x : R.ad_x)[j];
  const double iw = (self ? R.in_w : R.ad_w)[j];
  const int pp = self ? 6 : 2;
  const double up = pp == 6 ? uu * uu * uu * uu * uu * uu : uu * uu;
  *h = h0 + L * top * up;
  *w = top * iw * pp * (up / uu) * aL;
}

__global__ void __launch_bounds__(NT, 3) selfblock_kernel(const AsmBody* __restrict__ bodies, int nb,
                                                       const double* __restrict__ rules,
                                                       const qd4* __restrict__ x64, const qd4* __restrict__ n64,
                                                       const double* __restrict__ jac, double k, double eta,
                                                       long long row0, double2* __restrict__ blocks,
                                                       unsigned long long* __restrict__ counts, int pstride,
                                                       int batch,
                                                       const NearTarget* __restrict__ near) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RowShared& S = *reinterpret_cast<RowShared*>(smem_raw);
  // Q_{m-1/2} and dQ/dchi of the batch, [batch][pstride] each (pstride >= P + 1, even),
  // then the modal-domain accumulators of the current panel, [order][2N] complex each
  // for the double layer and the single layer (RowShared's size is a multiple of 16,
  // so every array stays 16-byte aligned)
  double* bq = reinterpret_cast<double*>(smem_raw + sizeof(RowShared));
  double* bdq = bq + batch * pstride;
  float4* accD = reinterpret_cast<float4*>(bdq + batch * pstride);

  // rows of the assembled bodies (one per class of congruent bodies), back to back;
  // or, with `near`, one off-surface target per CTA (the near-field rows)
  const long long gc = row0 + blockIdx.x;
  const bool nearm = near != nullptr;
  int lo = 0, hi = nb - 1;
  if (nearm) {
    lo = near[gc].cls;
  } else {
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bodies[mid].crow <= gc) lo = mid; else hi = mid - 1;
    }
  }
  const AsmBody B = bodies[lo];
  const int tid = threadIdx.x;
  const int nth = B.n_theta, N = nth / 2, order = B.order;
  const int per_panel = order * nth;
  float4* accS = accD + per_panel;
  const int nbn = B.n_panels * per_panel;
  const int t = nearm ? -1 : (int)(gc - B.crow);  // target node within the body
  const int p = nearm ? near[gc].panel : t / per_panel;
  const int lt = nearm ? 0 : (t % per_panel) / nth;
  const int jt = nearm ? 0 : t % nth;
  const double* toff = nearm ? near[gc].v : nullptr;
  const double* gl_x = rules + B.rule;              // [order] on [-1,1]
  const double* dy_x = gl_x + 2 * order;            // [level1_nodes] on [0,1]
  const double* dy_w = dy_x + level1_nodes(order);
  const double* d0_x = dy_w + level1_nodes(order);  // [level0_nodes] on [0,1], outermost level
  const double* d0_w = d0_x + level0_nodes(order);
  const double* in_x = d0_w + level0_nodes(order);  // [20]
  const double* in_w = in_x + 20;
  const double* ad_x = in_w + 20;                   // [16]
  const double* ad_w = ad_x + 16;
  const double* g12_x = ad_w + 16;                  // [12], inner dyadic levels
  const double* g12_w = g12_x + 12;
  const Rules RL{d0_x, d0_w, dy_x, dy_w, g12_x, g12_w, in_x, in_w, ad_x, ad_w};
  const double* bw = g12_w + 12;                    // [order] barycentric weights of the GL nodes
  const double2* ptab = reinterpret_cast<const double2*>(rules + 2 * MILLER_MAX);  // (cos, sin)(2 pi j/PH_N)
  const double* brk = rules + B.brk;                // panel breakpoints [n_panels + 1]
  const double s_t = nearm ? near[gc].s : 0.5 * (brk[p] + brk[p + 1]) + 0.5 * (brk[p + 1] - brk[p]) * gl_x[lt];
  const double th_t = nearm ? near[gc].th : 2.0 * M_PI * jt / nth;
  const double inv_nth = 1.0 / nth;
  const bool kz = (k == 0.0);
  const int n1 = kz ? 0 : B.n1;
  const int M = B.M, M2 = M / 2;
  const double twopi_M = 2.0 * M_PI / M;
  const int P = N + n1 + 2;
  double2* row = nearm ? blocks + near[gc].row : blocks + B.blk + (long long)t * nbn;

  for (int e = tid; e < 2 * per_panel; e += NT) accD[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  int n_far = 0;  // thread 0: far outer nodes of this row
  // far-ring contributions in sample space, entries e = tid + q NT of the current panel
  double far_re[MAXE], far_im[MAXE];
#pragma unroll
  for (int qq = 0; qq < MAXE; ++qq) far_re[qq] = far_im[qq] = 0.0;
  // outer-node pieces (thread 0; panels in increasing order, the self panel's two pieces adjacent)
  if (tid == 0) {
    int nq = 0, npc = 0;
    const double dpole = fmin(s_t + M_PI / 2, M_PI / 2 - s_t);
    for (int i = max(0, p - 1); i <= min(B.n_panels - 1, p + 1); ++i) {
      const double plo = brk[i], phi_ = brk[i + 1];
      double s0[2], e0[2];
      int npieces;
      if (i == p) { s0[0] = s_t; e0[0] = plo; s0[1] = s_t; e0[1] = phi_; npieces = 2; }
      else if (i < p) { s0[0] = phi_; e0[0] = plo; npieces = 1; }
      else { s0[0] = plo; e0[0] = phi_; npieces = 1; }
      for (int pc = 0; pc < npieces; ++pc) {
        const double L = e0[pc] - s0[pc], aL = fabs(L);
        const double h0 = s0[pc] - s_t;
        // dyadic levels toward the (near-)singular end: on the self panel until the
        // innermost piece is within half the distance to the nearer pole; on a
        // neighbour until it is within ~3 times the target's distance to the shared
        // edge (6 levels on equal panels)
        int K;
        if (i == p) K = max(5, (int)ceil(log2(aL / (0.5 * dpole))));
        else K = max(6, (int)ceil(log2(aL / (3.2 * fabs(h0)))));
        K = min(K, 14);
        // off-surface target at distance ds (in s) from s_t: the integrand is smooth on
        // the scale ds, so the self panel's levels continue until the innermost piece is
        // about ds long, which then takes the mildly graded (u^2) rule
        const bool graded6 = (i == p) && !nearm;
        if (nearm && i == p) K = min(44, max(K, (int)ceil(log2(aL / fmax(near[gc].ds, 1e-13))) + 1));
        nq += level0_nodes(order) + level1_nodes(order) + 12 * (K - 2) + (graded6 ? 20 : 16);
        S.pc_h0[npc] = h0;
        S.pc_L[npc] = L;
        S.pc_K[npc] = K;
        S.pc_panel[npc] = i;
        S.pc_self[npc] = graded6;
        S.pc_end[npc] = nq;
        ++npc;
      }
    }
    S.npc = npc;
    S.nq = nq;
    // row constants of the ring-target geometry
    double sth, cth;
    sincos(th_t, &sth, &cth);
    S.rowc[0] = cth;
    S.rowc[1] = sth;
    if (B.kind == 1) {
      const int nt = B.n_terms;
      const double* T = rules + B.ser;
      double r_t = 0.0;
      for (int j = 0; j < nt; ++j) {
        const double* tt = T + 3 * (3 * nt + j);
        double sn, cs;
        sincos(tt[0] * s_t, &sn, &cs);
        r_t += tt[1] * cs + tt[2] * sn;
      }
      S.rowc[6] = r_t;
    } else {
      double sst, cst;
      sincos(s_t, &sst, &cst);
      const double u_t = 0.5 * (1.0 + sst);
      const double rho_t = rho_prof(B, u_t);
      S.rowc[2] = sst;
      S.rowc[3] = cst;
      S.rowc[4] = u_t;
      S.rowc[5] = rho_t;
      S.rowc[6] = rho_t * cst;
    }
  }
  // row tables
  for (int q = tid; q <= M2; q += NT) {
    const double sv = sinpi((double)q / M);
    S.s2tab[q] = sv * sv;
  }
  for (int j = tid; j < M; j += NT) {
    const ff cj = ff_from_double(cospi(2.0 * j / M));
    S.ctab[j] = make_float2(cj.hi, cj.lo);
  }
  for (int j = tid; j < nth; j += NT) {
    sincospi(2.0 * j / nth, &S.sth[j], &S.cth[j]);
    const ff cj = ff_from_double(S.cth[j]), sj = ff_from_double(S.sth[j]);
    S.csff[j] = make_float4(cj.hi, cj.lo, sj.hi, sj.lo);
  }
  for (int n = tid; n <= MAXP; n += NT) S.inv_odd[n] = 1.0 / (2.0 * n - 1.0);
  __syncthreads();
  const int nq = S.nq;

  for (int b0 = 0; b0 < nq; b0 += batch) {
    const int nbatch = min(batch, nq - b0);
    if (tid < nbatch) {
      double hq, wq;
      int pq, fq;
      outer_node(S, RL, order, b0 + tid, &hq, &wq, &pq, &fq);
      S.bw[tid] = wq;
      S.bp[tid] = pq;
      S.bflush[tid] = fq;
      ring_node(B, rules, s_t, th_t, hq, P, N, S.inv_odd, bq + tid * pstride, bdq + tid * pstride, S.bs[tid],
                toff, S.rowc);
    }
    __syncthreads();
    for (int bi = 0; bi < nbatch; ++bi) {
      const double* sc = S.bs[bi];
      const double r = sc[0], rt = sc[1], c = sc[2], dr = sc[3], alpha = sc[4], scale = sc[5];
      const double dchi_r = sc[6], dchi_z = sc[7], s = sc[8];
      const double* q = bq + bi * pstride;
      const double* dq = bdq + bi * pstride;
      const bool farn = sc[14] != 0.0;
      if (tid == 0) n_far += farn ? 1 : 0;
      const int ip = S.bp[bi];
      if (tid < order) {
        const double xs = (s - brk[ip]) / (brk[ip + 1] - brk[ip]) * 2.0 - 1.0;  // panel coordinate
        // outer weight times P_l(x), P_l(x) = w_l prod_{m != l} (x - x_m), w_l = 1 / prod_{m != l} (x_l - x_m)
        double v = bw[tid] * S.bw[bi];
        for (int mm = 0; mm < order; ++mm)
          if (mm != tid) v *= xs - gl_x[mm];
        S.pl[tid] = v;
        const ff vf = ff_from_double(v);
        S.plff[tid] = make_float2(vf.hi, vf.lo);
      }
      if (farn) {
        // far ring: integrands sampled at the azimuthal nodes, times the
        // trapezoidal weight pi/N (held in dre/dim_ = double layer, tre/tim = single layer)
        const double na0 = sc[9], na1 = sc[10], nb0 = sc[11], nb1 = sc[12], nb2 = sc[13];
        const double cal = sc[15], sal = sc[16];
        const double wt = 2.0 * M_PI * inv_nth;
        for (int j = tid; j < nth; j += NT) {
          // sin^2(phi/2) = (1 - cos(theta_j - alpha))/2: on a far ring (dr^2 + c^2 >= 2.7 r r~)
          // the rounding of the difference is far below rho^2
          const double s2 = 0.5 * (1.0 - (S.cth[j] * cal + S.sth[j] * sal));
          const double rho2 = dr * dr + c * c + 4.0 * r * rt * s2;
          const double inv = rsqrt(rho2), rho = rho2 * inv;
          const double radial = dr + 2.0 * rt * s2;  // r - r~ cos(phi)
          double sn, cs;
          sincos_table(k * rho, ptab, &sn, &cs);
          const double f = 0.079577471545947667884 * inv;
          const double gr = cs * f, gi = sn * f;                               // G
          const double dpr = (-cs - k * rho * sn) * f * inv * inv, dpi = (k * rho * cs - sn) * f * inv * inv;  // G'/rho
          const double nr = na0 + na1 * S.cth[j];                              // |J| n_r
          const double nz = nb0 + nb1 * S.cth[j] + nb2 * S.sth[j];             // |J| n_3
          // |J| n_r K^r + |J| n_3 K^z with K^r = (G'/rho)(r - r~ cos phi), K^z = -(G'/rho) c
          const double dre_ = nr * dpr * radial - nz * dpr * c;
          const double dim = nr * dpi * radial - nz * dpi * c;
          S.dre[j] = wt * dre_;
          S.dim_[j] = wt * dim;
          S.tre[j] = wt * eta * gi;
          S.tim[j] = -wt * eta * gr;
        }
        __syncthreads();
        const int base = ip * per_panel;
#pragma unroll
        for (int qq = 0; qq < MAXE; ++qq) {
          const int e = tid + qq * NT;
          if (e < per_panel) {
            const int l = e / nth, j = e % nth;
            const double J = jac[B.offset + base + e];
            const double f = S.pl[l];
            far_re[qq] += f * (S.dre[j] + J * S.tre[j]);
            far_im[qq] += f * (S.dim_[j] + J * S.tim[j]);
          }
        }
        __syncthreads();
      } else {
      // B: scaled static modal sequences, samples of the smooth factors, cos/sin(m alpha)
      // static coefficients: g^_m = Q scale, d_r g^_m = dchi_r Q' scale - g^_m/(2r),
      // d_z g^_m = dchi_z Q' scale -- all from g^ and Q' scale
      for (int m = tid; m <= P; m += NT) {
        const double g0 = q[m] * scale, gd = dq[m] * scale;
        S.sg0[m] = g0;
        S.sdq[m] = gd;
        // Q' scale grows like r / h^2 near the singular point (beyond FP32's range on
        // refined panels); the products with dchi_r, dchi_z grow only like 1/(r h)
        const ff a = ff_from_double(g0), b = ff_from_double(dchi_r * gd), cz = ff_from_double(dchi_z * gd);
        S.sg0ff[m] = make_float2(a.hi, a.lo);
        S.srff[m] = make_float2(b.hi, b.lo);
        S.szff[m] = make_float2(cz.hi, cz.lo);
      }
      if (!kz) {
        for (int e = tid; e <= M2; e += NT) {
          const double rho = sqrt(dr * dr + c * c + 4.0 * r * rt * S.s2tab[e]);
          double f0, f1, f2v;
          smooth_factors(k * rho, ptab, &f0, &f1, &f2v);
          const ff a = ff_from_double(f0), b = ff_from_double(f1), cc = ff_from_double(f2v);
          S.fs[0][e] = make_float2(a.hi, a.lo);
          S.fs[1][e] = make_float2(b.hi, b.lo);
          S.fs[2][e] = make_float2(cc.hi, cc.lo);
        }
      }
      // e^{i m alpha} = e^{i 8 l alpha} e^{i j alpha}, m = 8 l + j: 13 sincos, combined in D2
      if (tid < 8 + (N + 2 + 7) / 8) {
        const int j = tid < 8 ? tid : 8 * (tid - 8);
        sincos(j * alpha, &S.esn[tid], &S.ecs[tid]);
      }
      __syncthreads();
      if (!kz) {
        // C1: cosine coefficients f^_n = (2pi/M)[f_0 + (-1)^n f_{M/2} + 2 sum f_q cos(2 pi n q/M)]
        // (float-float: a sum of M/2 FP64-accurate samples times table cosines)
        for (int e = tid; e < 3 * (n1 + 2); e += NT) {
          const int fn = e / (n1 + 2), n = e % (n1 + 2);
          const float2* f = S.fs[fn];
          ff sum{0.f, 0.f};
          int idx = 0;
          for (int qq = 1; qq < M2; ++qq) {
            idx += n;
            if (idx >= M) idx -= M;
            sum = ff_add(sum, ff_mul(ff{f[qq].x, f[qq].y}, ff{S.ctab[idx].x, S.ctab[idx].y}));
          }
          const ff fend{(n & 1) ? -f[M2].x : f[M2].x, (n & 1) ? -f[M2].y : f[M2].y};
          const ff tot = ff_add(ff_add(ff{f[0].x, f[0].y}, fend), ff_mul_f(sum, 2.0f));
          const double fcv = twopi_M * ff_to_double(tot);
          S.fc[fn][n] = fcv;
          if (fn < 2) {
            const ff a = ff_from_double(fcv);
            S.fcff[fn][n] = make_float2(a.hi, a.lo);
          }
        }
        __syncthreads();
        // C2: spectra of the smooth imaginary parts (multiplying by cos(phi) averages neighbours)
        const double k3 = k * k * k * INV_4PI, k1 = k * INV_4PI;
        for (int n = tid; n <= n1; n += NT) {
          const double Qm = S.fc[2][n == 0 ? 1 : n - 1], Qp = S.fc[2][n + 1];
          S.f2[n] = k1 * S.fc[1][n];
          S.pr[n] = k3 * ((dr + rt) * S.fc[2][n] - 0.5 * rt * (Qm + Qp));
          S.pz[n] = -k3 * c * S.fc[2][n];
        }
        // D: the four convolutions the real parts need (all sequences even in n),
        //   A_m = sum_n cos^_n g^_{m-n},  B^r_m, B^z_m = sum_n cos^_n (dchi_{r,z} Q' scale)_{m-n},
        //   C_m = sum_n sinc^_n g^_{m-n}   (m = 0..N+1; C also at N+2),
        // because d_r g^ = dchi_r Q' scale - g^/(2r) and d_z g^ = dchi_z Q' scale, and the
        // sinc-weighted terms are C_m and its cos(phi)-shift (C_{m-1} + C_{m+1})/2.
        // (in float-float: these are sums of FP64-computed products, ~48 bits suffice)
        const int L0 = N + 2;
        for (int e = tid; e < 4 * L0 + 1; e += NT) {
          const int part = min(e / L0, 3);  // 0 A, 1 B^r, 2 B^z, 3 C
          const float2* f = part < 3 ? S.fcff[0] : S.fcff[1];
          const float2* g = part == 1 ? S.srff : (part == 2 ? S.szff : S.sg0ff);
          const int m = e - part * L0;
          ff sum = ff_mul(ff{f[0].x, f[0].y}, ff{g[m].x, g[m].y});
          for (int n = 1; n <= n1; ++n) {
            const float2 ga = g[abs(m - n)], gb = g[m + n];
            sum = ff_add(sum, ff_mul(ff{f[n].x, f[n].y}, ff_add(ff{ga.x, ga.y}, ff{gb.x, gb.y})));
          }
          (part == 0 ? S.cA : (part == 1 ? S.cBr : (part == 2 ? S.cBz : S.cC)))[m] = ff_to_double(sum);
        }
        __syncthreads();
      }
      // D2: modal coefficients of G, d_r G, d_z G for m = 0..N+1, and cos/sin(m alpha)
      for (int m = tid; m <= N + 1; m += NT) {
        const int l = 8 + (m >> 3), j = m & 7;
        const ff cm = ff_from_double(S.ecs[l] * S.ecs[j] - S.esn[l] * S.esn[j]);
        const ff sm = ff_from_double(S.esn[l] * S.ecs[j] + S.ecs[l] * S.esn[j]);
        S.eff[m] = make_float4(cm.hi, cm.lo, sm.hi, sm.lo);
      }
      {
        const double inv2r = 0.5 / r, k2 = k * k;
        for (int e = tid; e < 3 * (N + 2); e += NT) {
          const int comp = e / (N + 2), m = e % (N + 2);
          double re, im = 0.0;
          if (kz) {
            re = comp == 0 ? S.sg0[m] : (comp == 1 ? dchi_r * S.sdq[m] - S.sg0[m] * inv2r : dchi_z * S.sdq[m]);
          } else if (comp == 0) {
            re = S.cA[m] * INV_2PI;
            im = m <= n1 ? S.f2[m] : 0.0;
          } else if (comp == 1) {
            const double cbar = 0.5 * (S.cC[m == 0 ? 1 : m - 1] + S.cC[m + 1]);
            re = (S.cBr[m] - S.cA[m] * inv2r - k2 * ((dr + rt) * S.cC[m] - rt * cbar)) * INV_2PI;
            im = m <= n1 ? S.pr[m] : 0.0;
          } else {
            re = (S.cBz[m] + k2 * c * S.cC[m]) * INV_2PI;
            im = m <= n1 ? S.pz[m] : 0.0;
          }
          const ff a = ff_from_double(re), b = ff_from_double(im);
          S.gff[comp][m] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
      }
      __syncthreads();
      // E: theta-coefficients, index m = -N+1..N stored at m mod 2N (the entry at N is the
      // symmetric Nyquist average), of
      //   double layer  (a0 + a1 cos theta) K^r + (b0 + b1 cos theta + b2 sin theta) K^z,
      //   single layer  -i eta G,
      // with K(theta - alpha) -> k^_|m| e^{-i m alpha}; cos(theta) averages m -+ 1 and
      // sin(theta) gives (k_{m-1} - k_{m+1})/(2i).
      // (in float-float: complex products of FP64-computed coefficients)
      const ff na0 = ff_from_double(sc[9]), na1 = ff_from_double(sc[10]), nb0 = ff_from_double(sc[11]);
      const ff nb1h = ff_from_double(0.5 * sc[12]), nb2h = ff_from_double(0.5 * sc[13]);
      const ff etaf = ff_from_double(eta);
      const bool zshift = (sc[12] != 0.0) || (sc[13] != 0.0);
      for (int mm = tid; mm < nth; mm += NT) {
        const int m0 = mm <= N ? mm : mm - nth;
        const int nsum = (m0 == N) ? 2 : 1;
        const float fac = (nsum == 2) ? 0.5f : 1.0f;
        ffc dsum{{0.f, 0.f}, {0.f, 0.f}}, g0sum{{0.f, 0.f}, {0.f, 0.f}};
        for (int sgn = 0; sgn < nsum; ++sgn) {
          const int m = (sgn == 0) ? m0 : -N;
          const int a0 = abs(m), am1 = abs(m - 1), ap1 = abs(m + 1);
          // e^{-i mv alpha} = cos(|mv| alpha) -/+ i sin(|mv| alpha)
          const ffc c0 = ephase(S.eff[a0], m >= 0), cm = ephase(S.eff[am1], m - 1 >= 0),
                    cp = ephase(S.eff[ap1], m + 1 >= 0);
          const ffc kr = ffc_mul(ffc_load(S.gff[1][a0]), c0);
          const ffc kz = ffc_mul(ffc_load(S.gff[2][a0]), c0);
          const ffc g0 = ffc_mul(ffc_load(S.gff[0][a0]), c0);
          const ffc km = ffc_mul(ffc_load(S.gff[1][am1]), cm);
          const ffc kp = ffc_mul(ffc_load(S.gff[1][ap1]), cp);
          const ffc kc{ff_mul_f(ff_add(km.re, kp.re), 0.5f), ff_mul_f(ff_add(km.im, kp.im), 0.5f)};  // (K^r cos)^_m
          ffc z{ff_add(ff_add(ff_mul(na0, kr.re), ff_mul(na1, kc.re)), ff_mul(nb0, kz.re)),
                ff_add(ff_add(ff_mul(na0, kr.im), ff_mul(na1, kc.im)), ff_mul(nb0, kz.im))};
          if (zshift) {
            const ffc zm = ffc_mul(ffc_load(S.gff[2][am1]), cm);
            const ffc zp = ffc_mul(ffc_load(S.gff[2][ap1]), cp);
            // cos: (z_{m-1} + z_{m+1})/2;  sin: -i (z_{m-1} - z_{m+1})/2
            z.re = ff_add(z.re, ff_add(ff_mul(nb1h, ff_add(zm.re, zp.re)), ff_mul(nb2h, ff_sub(zm.im, zp.im))));
            z.im = ff_add(z.im, ff_sub(ff_mul(nb1h, ff_add(zm.im, zp.im)), ff_mul(nb2h, ff_sub(zm.re, zp.re))));
          }
          dsum.re = ff_add(dsum.re, ff_mul_f(z.re, fac));
          dsum.im = ff_add(dsum.im, ff_mul_f(z.im, fac));
          g0sum.re = ff_add(g0sum.re, ff_mul_f(g0.re, fac));
          g0sum.im = ff_add(g0sum.im, ff_mul_f(g0.im, fac));
        }
        // single layer -i eta G
        const ff tre = ff_mul(etaf, g0sum.im), tim = ff_neg(ff_mul(etaf, g0sum.re));
        S.dff[mm] = make_float4(dsum.re.hi, dsum.re.lo, dsum.im.hi, dsum.im.lo);
        S.tff[mm] = make_float4(tre.hi, tre.lo, tim.hi, tim.lo);
      }
      __syncthreads();
      // F: accumulate w P_l(s) x (theta-coefficients) for the node's panel, in
      // float-float (~48 bits; the FP32 pipe instead of the 64x slower FP64 one)
      for (int e = tid; e < per_panel; e += NT) {
        const int l = e / nth, mm = e % nth;
        const ff f{S.plff[l].x, S.plff[l].y};
        const float4 dv = S.dff[mm], tv = S.tff[mm];
        const float4 ad = accD[e], as = accS[e];
        const ff d0 = ff_add(ff{ad.x, ad.y}, ff_mul(f, ff{dv.x, dv.y}));
        const ff d1 = ff_add(ff{ad.z, ad.w}, ff_mul(f, ff{dv.z, dv.w}));
        const ff s0 = ff_add(ff{as.x, as.y}, ff_mul(f, ff{tv.x, tv.y}));
        const ff s1 = ff_add(ff{as.z, as.w}, ff_mul(f, ff{tv.z, tv.w}));
        accD[e] = make_float4(d0.hi, d0.lo, d1.hi, d1.lo);
        accS[e] = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
      }
      __syncthreads();
      }  // modal path
      // panel finished: inverse DFT of the accumulated coefficients into the row,
      //   A[t,(ip,l,j)] = (1/2N) sum_m [D_lm + |J_lj| S_lm] e^{i m theta_j}
      if (S.bflush[bi]) {
        const int base = ip * per_panel;
        for (int e = tid; e < per_panel; e += NT) {
          const int l = e / nth, j = e % nth;
          const ff J = ff_from_double(jac[B.offset + base + e]);
          ff sr{0.f, 0.f}, si{0.f, 0.f};
          int idx = 0;
          for (int mm = 0; mm < nth; ++mm) {
            // e^{i m theta_j} with m = mm or mm - 2N (the same value): table[(mm j) mod 2N]
            const float4 cs = S.csff[idx];
            const float4 ad = accD[l * nth + mm], as = accS[l * nth + mm];
            const ff cr{cs.x, cs.y}, ci{cs.z, cs.w};
            const ff ar = ff_add(ff{ad.x, ad.y}, ff_mul(J, ff{as.x, as.y}));
            const ff ai = ff_add(ff{ad.z, ad.w}, ff_mul(J, ff{as.z, as.w}));
            sr = ff_add(sr, ff_sub(ff_mul(ar, cr), ff_mul(ai, ci)));
            si = ff_add(si, ff_add(ff_mul(ar, ci), ff_mul(ai, cr)));
            idx += j;
            if (idx >= nth) idx -= nth;
          }
          double2 v = make_double2(ff_to_double(sr) * inv_nth, ff_to_double(si) * inv_nth);
          if (base + e == t) v.x += 0.5;  // (never for an off-surface target: t < 0)
          row[base + e] = v;
        }
        // add the far-ring part (same entries per thread: e = tid + q NT)
#pragma unroll
        for (int qq = 0; qq < MAXE; ++qq) {
          const int e = tid + qq * NT;
          if (e < per_panel) {
            row[base + e].x += far_re[qq];
            row[base + e].y += far_im[qq];
          }
          far_re[qq] = far_im[qq] = 0.0;
        }
        __syncthreads();
        for (int e = tid; e < 2 * per_panel; e += NT) accD[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
      }
    }
  }
  // outer nodes of this row by kind (modal, far) for the work accounting
  if (tid == 0 && counts) {
    atomicAdd(&counts[0], (unsigned long long)(nq - n_far));
    atomicAdd(&counts[1], (unsigned long long)n_far);
  }
  if (nearm) {
    // near-field row: product integration minus the smooth rule on the near panels
    // (the caller adds the smooth rule over all nodes), zero beyond them
    qd4 xt;
    xt.x = near[gc].x[0];
    xt.y = near[gc].x[1];
    xt.z = near[gc].x[2];
    xt.w = 0.0;
    const long long node0 = near[gc].node0;
    for (int e = tid; e < nbn; e += NT) {
      const int i = e / per_panel;
      if (abs(i - p) > 1) {
        row[e] = make_double2(0.0, 0.0);
        continue;
      }
      double kre, kim;
      const qd4 ys = x64[node0 + e];
      smooth_kernel(xt, ys, n64[node0 + e], k, eta, ptab, &kre, &kim);
      row[e].x -= kre * ys.w;
      row[e].y -= kim * ys.w;
    }
    return;
  }
  // panels beyond the neighbours: the plain smooth rule
  const long long g = B.offset + t;  // global target node
  const qd4 xt = x64[g];
  for (int e = tid; e < nbn; e += NT) {
    const int i = e / per_panel;
    if (abs(i - p) <= 1) continue;
    const long long src = B.offset + e;
    double kre, kim;
    smooth_kernel(xt, x64[src], n64[src], k, eta, ptab, &kre, &kim);
    const double w = x64[src].w;
    row[e] = make_double2(kre * w, kim * w);
  }
}

}  // namespace

static_assert(sizeof(RowShared) % 16 == 0, "double2 accumulators follow RowShared");

// Dynamic shared memory of one CTA: RowShared, Q and dQ of a batch, two panel
// accumulators of float-float complex entries.
size_t qams_selfblock_smem(int max_per_panel, int pstride, int batch) {
  return sizeof(RowShared) + 2 * sizeof(double) * batch * (size_t)pstride + 2 * sizeof(float4) * (size_t)max_per_panel;
}

// Outer nodes per batch: all 32 lanes of warp 0 when three CTAs still fit on an SM
// (228 KB of shared memory, 1 KB reserved per CTA), else 16.
int qams_selfblock_batch(int max_per_panel, int pstride) {
  return 3 * (qams_selfblock_smem(max_per_panel, pstride, 32) + 1024) <= 228 * 1024 ? 32 : 16;
}

namespace {

// Kernel tables of the context's classes of congruent bodies (one AsmBody per
// class, from its first body) and the rule tables per distinct order.  r_extra
// widens the smooth-factor bandwidth for targets up to r_extra off the surface.
int build_tables(qams_ctx* c, double r_extra, std::vector<AsmBody>& ab, std::vector<double>& rules, long long* blk_out,
                 long long* rows_out, int* max_nb_out, int* pstride_out) {
  const int nb = (int)c->class_rep.size();
  std::vector<int> rule_off(64, -1);
  ab.assign(nb, AsmBody{});
  rules.clear();
  // Miller coefficients alpha_n = 4(n-1)/(2n-3), beta_n = (2n-1)/(2n-3), n < MILLER_MAX
  for (int n = 0; n < MILLER_MAX; ++n) {
    rules.push_back(n >= 2 ? 4.0 * (n - 1) / (2.0 * n - 3.0) : 0.0);
    rules.push_back(n >= 2 ? (2.0 * n - 1.0) / (2.0 * n - 3.0) : 0.0);
  }
  // table of the accurate-table sincos (phase.cuh), 16-byte aligned (offset 2 MILLER_MAX doubles)
  for (int j = 0; j < PH_N; ++j) {
    rules.push_back(std::cos(2.0 * M_PI * j / PH_N));
    rules.push_back(std::sin(2.0 * M_PI * j / PH_N));
  }
  long long blk = 0, rows = 0;
  int max_nb = 0, pstride = 0;
  for (int b = 0; b < nb; ++b) {
    const BodyHost& bh = c->bodies[c->class_rep[b]];
    const qams_body_desc& d = bh.d;
    if (d.order > MAXORD || d.n_theta / 2 > MAXN) return QAMS_EINVAL;
    if (rule_off[d.order] < 0) {
      rule_off[d.order] = (int)rules.size();
      std::vector<double> x, w;
      qams_gauss_legendre(d.order, x, w);
      rules.insert(rules.end(), x.begin(), x.end());
      rules.insert(rules.end(), w.begin(), w.end());
      qams_gauss_legendre(level1_nodes(d.order), x, w);
      for (auto& v : x) v = 0.5 * (v + 1.0);
      for (auto& v : w) v *= 0.5;
      rules.insert(rules.end(), x.begin(), x.end());
      rules.insert(rules.end(), w.begin(), w.end());
      qams_gauss_legendre(level0_nodes(d.order), x, w);
      for (auto& v : x) v = 0.5 * (v + 1.0);
      for (auto& v : w) v *= 0.5;
      rules.insert(rules.end(), x.begin(), x.end());
      rules.insert(rules.end(), w.begin(), w.end());
      qams_gauss_legendre(20, x, w);
      for (auto& v : x) v = 0.5 * (v + 1.0);
      for (auto& v : w) v *= 0.5;
      rules.insert(rules.end(), x.begin(), x.end());
      rules.insert(rules.end(), w.begin(), w.end());
      qams_gauss_legendre(16, x, w);
      for (auto& v : x) v = 0.5 * (v + 1.0);
      for (auto& v : w) v *= 0.5;
      rules.insert(rules.end(), x.begin(), x.end());
      rules.insert(rules.end(), w.begin(), w.end());
      qams_gauss_legendre(12, x, w);
      for (auto& v : x) v = 0.5 * (v + 1.0);
      for (auto& v : w) v *= 0.5;
      rules.insert(rules.end(), x.begin(), x.end());
      rules.insert(rules.end(), w.begin(), w.end());
      qams_gauss_legendre(d.order, x, w);
      for (int l = 0; l < d.order; ++l) {
        double prod = 1.0;
        for (int m = 0; m < d.order; ++m)
          if (m != l) prod *= x[l] - x[m];
        rules.push_back(1.0 / prod);
      }
    }
    AsmBody& A = ab[b];
    A.kind = d.profile_kind;
    A.n_terms = d.profile_kind == 1 ? d.n_terms : 0;
    A.ser = (int)rules.size();
    rules.insert(rules.end(), bh.series.begin(), bh.series.end());
    A.brk = (int)rules.size();
    rules.insert(rules.end(), bh.breaks.begin(), bh.breaks.end());
    A.n_panels = d.n_panels;
    A.order = d.order;
    A.n_theta = d.n_theta;
    A.n_modes = (int)bh.a.size();
    A.base = d.base_radius;
    A.L = d.axis_length;
    A.kappa = d.curvature;
    for (int m = 0; m < 8; ++m) {
      A.a[m] = m < A.n_modes ? bh.a[m] : 0.0;
      A.b[m] = m < A.n_modes ? bh.b[m] : 0.0;
    }
    A.offset = bh.offset;
    A.crow = rows;
    rows += bh.n;
    A.blk = blk;
    blk += (long long)bh.n * bh.n;
    const double rmax = bh.rmax + r_extra;
    A.n1 = (int)std::ceil(1.3 * c->k * rmax + 16.0);
    A.M = 2 * (A.n1 + 8);
    if (A.n1 + 2 > MAXN1 || A.M / 2 + 1 > MAXM2 || d.n_theta / 2 + A.n1 + 2 > MAXP || A.M > 2 * MAXM2)
      return QAMS_EINVAL;
    A.rule = rule_off[d.order];
    max_nb = std::max(max_nb, d.order * d.n_theta);
    pstride = std::max(pstride, (d.n_theta / 2 + A.n1 + 2 + 1 + 1) & ~1);  // P + 1, rounded up to even
  }
  *blk_out = blk;
  *rows_out = rows;
  *max_nb_out = max_nb;
  *pstride_out = pstride;
  return QAMS_OK;
}

}  // namespace

int qams_assemble_launch(qams_ctx* c, cudaStream_t st) {
  // one block per class of congruent bodies, from its first body's rows
  const int nb = (int)c->class_rep.size();
  std::vector<AsmBody> ab;
  std::vector<double> rules;
  long long blk = 0, rows = 0;
  int max_nb = 0, pstride = 0;
  int rc = build_tables(c, 0.0, ab, rules, &blk, &rows, &max_nb, &pstride);
  if (rc) return rc;
  qams_dev_free(c, &c->blocks64);
  if ((rc = qams_dev_alloc(c, &c->blocks64, sizeof(double2) * (size_t)blk))) return rc;
  c->block_entries = blk;
  DeviceBuf d_bodies, d_rules, d_counts;
  if ((rc = qams_dev_alloc(c, &d_bodies, sizeof(AsmBody) * nb))) return rc;
  if ((rc = qams_dev_alloc(c, &d_rules, sizeof(double) * rules.size()))) return rc;
  QAMS_CUDA(cudaMemcpy(d_bodies.p, ab.data(), sizeof(AsmBody) * nb, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(d_rules.p, rules.data(), sizeof(double) * rules.size(), cudaMemcpyHostToDevice));
  if ((rc = qams_dev_alloc(c, &d_counts, 2 * sizeof(unsigned long long)))) return rc;
  QAMS_CUDA(cudaMemsetAsync(d_counts.p, 0, 2 * sizeof(unsigned long long), st));
  const int batch = qams_selfblock_batch(max_nb, pstride);
  const size_t smem = qams_selfblock_smem(max_nb, pstride, batch);
  // The attribute is process-wide: requests served concurrently must not lower it under
  // one another, so it is always set to the kernel's largest possible launch size.
  static_assert(sizeof(RowShared) + 2 * sizeof(double) * BATCH * (MAXP + 2) +
                        2 * sizeof(float4) * MAXORD * 2 * MAXN <= 227 * 1024,
                "largest self-block launch exceeds the shared memory of a CTA");
  const int smem_max = (int)qams_selfblock_smem(MAXORD * 2 * MAXN, MAXP + 2, BATCH);
  QAMS_CUDA(cudaFuncSetAttribute(selfblock_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  QAMS_CUDA(cudaFuncSetAttribute(selfblock_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  const long long chunk = 1 << 20;
  for (long long r0 = 0; r0 < rows; r0 += chunk) {
    const long long n = std::min(chunk, rows - r0);
    cudaEvent_t pe = qams_prof_begin(c, QAMS_PROF_ASSEMBLY, st);
    selfblock_kernel<<<(unsigned)n, NT, smem, st>>>((const AsmBody*)d_bodies.p, nb, (const double*)d_rules.p,
                                                    (const qd4*)c->x64.p, (const qd4*)c->n64.p,
                                                    (const double*)c->jac64.p, c->k, c->eta, r0,
                                                    (double2*)c->blocks64.p, (unsigned long long*)d_counts.p,
                                                    pstride, batch, nullptr); qams_count_launch();
    qams_prof_end(c, QAMS_PROF_ASSEMBLY, st, pe);
    QAMS_CUDA(cudaGetLastError());
  }
  QAMS_CUDA(cudaStreamSynchronize(st));
  unsigned long long hc[2] = {0, 0};
  QAMS_CUDA(cudaMemcpy(hc, d_counts.p, sizeof(hc), cudaMemcpyDeviceToHost));
  c->asm_counts[0] = (long long)hc[0];
  c->asm_counts[1] = (long long)hc[1];
  qams_dev_free(c, &d_bodies);
  qams_dev_free(c, &d_rules);
  qams_dev_free(c, &d_counts);
  return QAMS_OK;
}

// Near-field rows (see selfblock_kernel with `near`): one row of n_b entries per
// target, at targets[i].row of `rows`, for n targets already on the device.
int qams_near_rows_launch(qams_ctx* c, const NearTarget* targets, long long n, double r_extra, double2* rows,
                          cudaStream_t st) {
  if (n <= 0) return QAMS_OK;
  const int nb = (int)c->class_rep.size();
  std::vector<AsmBody> ab;
  std::vector<double> rules;
  long long blk = 0, nrows = 0;
  int max_nb = 0, pstride = 0;
  int rc = build_tables(c, r_extra, ab, rules, &blk, &nrows, &max_nb, &pstride);
  if (rc) return rc;
  DeviceBuf d_bodies, d_rules;
  if ((rc = qams_dev_alloc(c, &d_bodies, sizeof(AsmBody) * nb))) return rc;
  if ((rc = qams_dev_alloc(c, &d_rules, sizeof(double) * rules.size()))) {
    qams_dev_free(c, &d_bodies);
    return rc;
  }
  QAMS_CUDA(cudaMemcpy(d_bodies.p, ab.data(), sizeof(AsmBody) * nb, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(d_rules.p, rules.data(), sizeof(double) * rules.size(), cudaMemcpyHostToDevice));
  const int batch = qams_selfblock_batch(max_nb, pstride);
  const size_t smem = qams_selfblock_smem(max_nb, pstride, batch);
  const int smem_max = (int)qams_selfblock_smem(MAXORD * 2 * MAXN, MAXP + 2, BATCH);
  QAMS_CUDA(cudaFuncSetAttribute(selfblock_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  QAMS_CUDA(cudaFuncSetAttribute(selfblock_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  const long long chunk = 1 << 20;
  for (long long r0 = 0; r0 < n; r0 += chunk) {
    const long long m = std::min(chunk, n - r0);
    selfblock_kernel<<<(unsigned)m, NT, smem, st>>>((const AsmBody*)d_bodies.p, nb, (const double*)d_rules.p,
                                                    (const qd4*)c->x64.p, (const qd4*)c->n64.p,
                                                    (const double*)c->jac64.p, c->k, c->eta, r0, rows, nullptr,
                                                    pstride, batch, targets);
    qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
  }
  QAMS_CUDA(cudaStreamSynchronize(st));
  qams_dev_free(c, &d_bodies);
  qams_dev_free(c, &d_rules);
  return QAMS_OK;
}
