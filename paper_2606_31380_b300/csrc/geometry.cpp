// Host-side geometry and Nystrom nodes (Eq. para_quasi, Sec. 3.1, Eq. sx).
//
// Kind 0, s in [-pi/2, pi/2]:
//   u = (1 + sin s)/2, rho(u) = base (1 + sum a_m cos 2 pi m u + b_m sin 2 pi m u)
//   r(s) = rho(u) cos s, l(s) = L (u - 1/2)
//   axis: planar arc of curvature kappa, frame e1 = (cos kl, 0, -sin kl),
//         e2 = (0, 1, 0), e3 = (sin kl, 0, cos kl) (rotation minimising)
//   y(s, theta) = gamma(l) + r (cos theta e1 + sin theta e2)
//   d_s = l'(1 - kappa r cos theta) e3 + r' e_r,  d_theta = r e_theta
// Kind 1 (the paper's shapes, Eqs. quasiwave and geometries):
//   y(s, theta) = (x_c + r cos theta, y_c + r sin theta, z), each a sum of
//   A cos(omega s) + B sin(omega s); frame e1, e2, e3 = x, y, z;
//   d_s = z' e3 + (r' + x_c' cos theta + y_c' sin theta) e_r + (...) e_theta
// Both: with A the e3 part and B the e_r part of d_s,
//   n = (A e_r - B e3)/sqrt(A^2 + B^2),  |J| = r sqrt(A^2 + B^2),
//   w = |J| (2 pi / n_theta) omega_l.
#include <cmath>
#include <cstring>

#include "qams_internal.h"

void qams_gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    // i-th root from the top, then stored ascending
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

namespace {

// f = sum A cos(omega s) + B sin(omega s) and f' for one of the four kind-1 functions
void series_eval(const double* T, int nt, double s, double* f, double* df) {
  double v = 0.0, dv = 0.0;
  for (int j = 0; j < nt; ++j) {
    const double om = T[3 * j], A = T[3 * j + 1], B = T[3 * j + 2];
    const double c = std::cos(om * s), sn = std::sin(om * s);
    v += A * c + B * sn;
    dv += om * (B * c - A * sn);
  }
  *f = v;
  *df = dv;
}

struct Shape {
  const BodyCopy& bc;
  double rho(double u) const {
    double s = 1.0;
    for (size_t m = 1; m <= bc.a.size(); ++m) s += bc.a[m - 1] * std::cos(2 * M_PI * m * u);
    for (size_t m = 1; m <= bc.b.size(); ++m) s += bc.b[m - 1] * std::sin(2 * M_PI * m * u);
    return bc.d.base_radius * s;
  }
  double drho(double u) const {
    double s = 0.0;
    for (size_t m = 1; m <= bc.a.size(); ++m) s -= bc.a[m - 1] * 2 * M_PI * m * std::sin(2 * M_PI * m * u);
    for (size_t m = 1; m <= bc.b.size(); ++m) s += bc.b[m - 1] * 2 * M_PI * m * std::cos(2 * M_PI * m * u);
    return bc.d.base_radius * s;
  }
  // local point, normal and |J| at (s, theta)
  void eval(double s, double th, double p[3], double nrm[3], double* jac) const {
    const double ct = std::cos(th), st = std::sin(th);
    if (bc.d.profile_kind == 1) {
      const int nt = bc.d.n_terms;
      double f[4], df[4];
      for (int q = 0; q < 4; ++q) series_eval(bc.series.data() + 3 * nt * q, nt, s, &f[q], &df[q]);
      const double A = df[2], B = df[3] + df[0] * ct + df[1] * st;
      const double hh = std::sqrt(A * A + B * B);
      p[0] = f[0] + f[3] * ct;
      p[1] = f[1] + f[3] * st;
      p[2] = f[2];
      nrm[0] = A * ct / hh;
      nrm[1] = A * st / hh;
      nrm[2] = -B / hh;
      *jac = f[3] * hh;
      return;
    }
    const double kappa = bc.d.curvature, L = bc.d.axis_length;
    double u = 0.5 * (1.0 + std::sin(s));
    double du = 0.5 * std::cos(s);
    double r = rho(u) * std::cos(s);
    double dr = drho(u) * du * std::cos(s) - rho(u) * std::sin(s);
    double l = 0.5 * L * std::sin(s);
    double dl = 0.5 * L * std::cos(s);
    double kl = kappa * l;
    double h = 0.5 * kl;
    double sh = std::fabs(h) > 1e-8 ? std::sin(h) / h : 1.0;
    double sf = std::fabs(kl) > 1e-8 ? std::sin(kl) / kl : 1.0;
    double g[3] = {0.5 * kappa * l * l * sh * sh, 0.0, l * sf};
    double e1[3] = {std::cos(kl), 0.0, -std::sin(kl)};
    double e3[3] = {std::sin(kl), 0.0, std::cos(kl)};
    double er[3] = {ct * e1[0], st, ct * e1[2]};
    double A = dl * (1.0 - kappa * r * ct);
    double B = dr;
    double hh = std::sqrt(A * A + B * B);
    for (int i = 0; i < 3; ++i) {
      p[i] = g[i] + r * er[i];
      nrm[i] = (A * er[i] - B * e3[i]) / hh;
    }
    *jac = r * hh;
  }
};

}  // namespace

int qams_copy_body(const qams_body_desc& d, BodyCopy* out) {
  if (d.n_panels < 1 || d.order < 1 || d.n_theta < 2 || (d.n_theta & 1) ||
      (d.profile_kind != 0 && d.profile_kind != 1))
    return QAMS_EINVAL;
  BodyCopy& bc = *out;
  bc.d = d;
  bc.d.mode_cos = bc.d.mode_sin = bc.d.series = bc.d.panel_breaks = nullptr;
  bc.a.clear();
  bc.b.clear();
  bc.series.clear();
  if (d.profile_kind == 0) {
    if (d.n_modes < 0 || d.n_modes > 8 || !(d.base_radius > 0) || !(d.axis_length > 0) || !(d.curvature >= 0))
      return QAMS_EINVAL;
    bc.a.assign(d.n_modes, 0.0);
    bc.b.assign(d.n_modes, 0.0);
    double amp = 0.0;
    for (int m = 0; m < d.n_modes; ++m) {
      if (d.mode_cos) bc.a[m] = d.mode_cos[m];
      if (d.mode_sin) bc.b[m] = d.mode_sin[m];
      if (!std::isfinite(bc.a[m]) || !std::isfinite(bc.b[m])) return QAMS_EINVAL;
      amp += std::fabs(bc.a[m]) + std::fabs(bc.b[m]);
    }
    if (amp >= 1.0 || d.curvature * d.base_radius * (1.0 + amp) >= 1.0) return QAMS_EINVAL;
    bc.rmax = d.base_radius * (1.0 + amp);
    bc.radius = 0.5 * d.axis_length + bc.rmax;
  } else {
    const int nt = d.n_terms;
    if (nt < 1 || nt > 8 || !d.series) return QAMS_EINVAL;
    bc.series.assign(d.series, d.series + 12 * nt);
    double bound[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q)
      for (int j = 0; j < nt; ++j) {
        const double* t = &bc.series[3 * (nt * q + j)];
        if (!std::isfinite(t[0]) || !std::isfinite(t[1]) || !std::isfinite(t[2])) return QAMS_EINVAL;
        bound[q] += std::fabs(t[1]) + std::fabs(t[2]);
      }
    // r > 0 and z' > 0 inside, r = 0 at both ends (checked on a fine grid)
    const double* Tz = bc.series.data() + 6 * nt;
    const double* Tr = bc.series.data() + 9 * nt;
    double f, df;
    for (int i = 1; i < 2048; ++i) {
      const double s = -M_PI / 2 + M_PI * i / 2048.0;
      series_eval(Tr, nt, s, &f, &df);
      if (!(f > 0)) return QAMS_EINVAL;
      series_eval(Tz, nt, s, &f, &df);
      if (!(df > 0)) return QAMS_EINVAL;
    }
    for (double s : {-M_PI / 2, M_PI / 2}) {
      series_eval(Tr, nt, s, &f, &df);
      if (std::fabs(f) > 1e-12 * bound[3]) return QAMS_EINVAL;
    }
    bc.rmax = bound[3];
    bc.radius = std::sqrt(bound[0] * bound[0] + bound[1] * bound[1] + bound[2] * bound[2]) + bound[3];
  }
  bc.breaks.assign(d.n_panels + 1, 0.0);
  if (d.panel_breaks) {
    for (int i = 0; i <= d.n_panels; ++i) {
      bc.breaks[i] = d.panel_breaks[i];
      if (!std::isfinite(bc.breaks[i]) || (i > 0 && !(bc.breaks[i] > bc.breaks[i - 1]))) return QAMS_EINVAL;
    }
    if (std::fabs(bc.breaks[0] + M_PI / 2) > 1e-14 || std::fabs(bc.breaks[d.n_panels] - M_PI / 2) > 1e-14)
      return QAMS_EINVAL;
  } else {
    for (int i = 0; i <= d.n_panels; ++i) bc.breaks[i] = -M_PI / 2 + M_PI * i / d.n_panels;
  }
  bc.breaks[0] = -M_PI / 2;
  bc.breaks[d.n_panels] = M_PI / 2;
  return QAMS_OK;
}

qams_body_desc qams_desc_view(const BodyCopy& bc) {
  qams_body_desc d = bc.d;
  d.n_modes = (int)bc.a.size();
  d.mode_cos = bc.a.empty() ? nullptr : bc.a.data();
  d.mode_sin = bc.b.empty() ? nullptr : bc.b.data();
  d.series = bc.series.empty() ? nullptr : bc.series.data();
  d.panel_breaks = bc.breaks.data();
  return d;
}

// Nodes of one body (order panel -> Gauss-Legendre node -> azimuth): world
// position, world normal, weight w = |J| (2 pi / n_theta) omega and |J|.
static void body_nodes_into(const BodyCopy& bc, double* x, double* n, double* w, double* jac_out) {
  const qams_body_desc& d = bc.d;
  Shape sh{bc};
  std::vector<double> gx, gw;
  qams_gauss_legendre(d.order, gx, gw);
  long long idx = 0;
  const double dth = 2.0 * M_PI / d.n_theta;
  for (int i = 0; i < d.n_panels; ++i) {
    const double lo = bc.breaks[i], hi = bc.breaks[i + 1];
    for (int l = 0; l < d.order; ++l) {
      const double s = 0.5 * (lo + hi) + 0.5 * (hi - lo) * gx[l];
      const double om = 0.5 * (hi - lo) * gw[l];
      for (int j = 0; j < d.n_theta; ++j, ++idx) {
        double p[3], nl[3], jac;
        sh.eval(s, j * dth, p, nl, &jac);
        for (int r = 0; r < 3; ++r) {
          double xr = d.center[r], nr = 0.0;
          for (int q = 0; q < 3; ++q) {
            xr += d.rotation[3 * r + q] * p[q];
            nr += d.rotation[3 * r + q] * nl[q];
          }
          if (x) x[3 * idx + r] = xr;
          if (n) n[3 * idx + r] = nr;
        }
        if (w) w[idx] = jac * dth * om;
        if (jac_out) jac_out[idx] = jac;
      }
    }
  }
}

int qams_build_nodes(qams_ctx* c) {
  long long N = 0;
  for (auto& bh : c->bodies) {
    bh.offset = N;
    bh.n = bh.d.n_panels * bh.d.order * bh.d.n_theta;
    N += bh.n;
  }
  c->N = N;
  c->hx.assign(3 * N, 0.0);
  c->hn.assign(3 * N, 0.0);
  c->hw.assign(N, 0.0);
  c->hj.assign(N, 0.0);
  for (auto& bh : c->bodies)
    body_nodes_into(bh, c->hx.data() + 3 * bh.offset, c->hn.data() + 3 * bh.offset, c->hw.data() + bh.offset,
                    c->hj.data() + bh.offset);
  return QAMS_OK;
}

extern "C" int qams_body_nodes(const qams_body_desc* desc, double* x_host, double* n_host, double* w_host) {
  if (!desc) return QAMS_EINVAL;
  BodyCopy bc;
  const int rc = qams_copy_body(*desc, &bc);
  if (rc) return rc;
  body_nodes_into(bc, x_host, n_host, w_host, nullptr);
  return QAMS_OK;
}

void qams_nearest_point(const BodyHost& b, const double* hx_body, const double x[3], double* s_out,
                        double* th_out, int* panel_out, double* dist_out, double* ds_out, double v_out[3]) {
  const qams_body_desc& d = b.d;
  Shape sh{b};
  // body-local target
  double xl[3];
  for (int q = 0; q < 3; ++q) {
    xl[q] = 0.0;
    for (int r = 0; r < 3; ++r) xl[q] += d.rotation[3 * r + q] * (x[r] - d.center[r]);
  }
  // start at the nearest node
  long long best = 0;
  double bd = 1e300;
  for (long long t = 0; t < b.n; ++t) {
    const double dx = hx_body[3 * t] - x[0], dy = hx_body[3 * t + 1] - x[1], dz = hx_body[3 * t + 2] - x[2];
    const double dd = dx * dx + dy * dy + dz * dz;
    if (dd < bd) {
      bd = dd;
      best = t;
    }
  }
  std::vector<double> gx, gw;
  qams_gauss_legendre(d.order, gx, gw);
  const int per_panel = d.order * d.n_theta;
  const int p0 = (int)(best / per_panel), l0 = (int)((best % per_panel) / d.n_theta), j0 = (int)(best % d.n_theta);
  double s = 0.5 * (b.breaks[p0] + b.breaks[p0 + 1]) + 0.5 * (b.breaks[p0 + 1] - b.breaks[p0]) * gx[l0];
  double th = 2.0 * M_PI * j0 / d.n_theta;
  const double smax = 0.5 * M_PI - 1e-7;
  // Levenberg-Marquardt on f = |x - y(s, th)|^2 with difference Jacobians: a step is
  // taken only if it lowers f (so the result is never farther than the nearest node,
  // also where the surface curves on the scale of the distance, e.g. near a pole);
  // the Jacobian's error only slows the iteration, the fixed point is set by f
  auto dist2 = [&](double ss, double tt) {
    double p[3], nn[3], jac;
    sh.eval(ss, tt, p, nn, &jac);
    double f = 0.0;
    for (int q = 0; q < 3; ++q) f += (xl[q] - p[q]) * (xl[q] - p[q]);
    return f;
  };
  double f = dist2(s, th), lam = 1e-3;
  for (int it = 0; it < 100; ++it) {
    double p[3], nn[3], jac, pa[3], pb[3], dummy;
    const double hs = 1e-6, ht = 1e-6;
    sh.eval(s, th, p, nn, &jac);
    const double sa = std::min(smax, s + hs), sb = std::max(-smax, s - hs);
    sh.eval(sa, th, pa, nn, &dummy);
    sh.eval(sb, th, pb, nn, &dummy);
    double Js[3], Jt[3];
    for (int q = 0; q < 3; ++q) Js[q] = (pa[q] - pb[q]) / (sa - sb);
    sh.eval(s, th + ht, pa, nn, &dummy);
    sh.eval(s, th - ht, pb, nn, &dummy);
    for (int q = 0; q < 3; ++q) Jt[q] = (pa[q] - pb[q]) / (2.0 * ht);
    double a11 = 0, a12 = 0, a22 = 0, g1 = 0, g2 = 0;
    for (int q = 0; q < 3; ++q) {
      const double r = xl[q] - p[q];
      a11 += Js[q] * Js[q];
      a12 += Js[q] * Jt[q];
      a22 += Jt[q] * Jt[q];
      g1 += Js[q] * r;
      g2 += Jt[q] * r;
    }
    bool moved = false;
    for (int tries = 0; tries < 30 && !moved; ++tries) {
      const double b11 = a11 * (1.0 + lam) + 1e-300, b22 = a22 * (1.0 + lam) + 1e-300;
      const double det = b11 * b22 - a12 * a12;
      if (!(det > 0.0)) {
        lam *= 10.0;
        continue;
      }
      const double ds = (b22 * g1 - a12 * g2) / det, dt = (b11 * g2 - a12 * g1) / det;
      const double s2 = std::max(-smax, std::min(smax, s + ds)), t2 = th + dt;
      const double f2 = dist2(s2, t2);
      if (f2 < f) {
        const bool small = std::fabs(s2 - s) < 1e-14 && std::fabs(t2 - th) < 1e-14;
        s = s2;
        th = t2;
        f = f2;
        lam = std::max(lam * 0.1, 1e-12);
        moved = true;
        if (small) it = 100;
      } else {
        lam *= 10.0;
      }
    }
    if (!moved) break;
  }
  th = std::fmod(th, 2.0 * M_PI);
  if (th < 0) th += 2.0 * M_PI;
  double p[3], nn[3], jac;
  sh.eval(s, th, p, nn, &jac);
  double v[3];
  for (int q = 0; q < 3; ++q) v[q] = xl[q] - p[q];
  *dist_out = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  {
    // |d_s y| by a central difference: the distance in units of s
    double pa[3], pb[3], dummy;
    const double hs = 1e-6, sa = std::min(smax, s + hs), sb = std::max(-smax, s - hs);
    sh.eval(sa, th, pa, nn, &dummy);
    sh.eval(sb, th, pb, nn, &dummy);
    double sp = 0.0;
    for (int q = 0; q < 3; ++q) sp += (pa[q] - pb[q]) * (pa[q] - pb[q]);
    sp = std::sqrt(sp) / (sa - sb);
    *ds_out = sp > 0.0 ? *dist_out / sp : *dist_out;
  }
  if (d.profile_kind == 1) {
    for (int q = 0; q < 3; ++q) v_out[q] = v[q];
  } else {
    // components in (e1, e2, e3)(s) of the arc axis
    const double kl = d.curvature * 0.5 * d.axis_length * std::sin(s);
    const double ck = std::cos(kl), sk = std::sin(kl);
    v_out[0] = ck * v[0] - sk * v[2];
    v_out[1] = v[1];
    v_out[2] = sk * v[0] + ck * v[2];
  }
  int pan = 0;
  while (pan + 1 < d.n_panels && s >= b.breaks[pan + 1]) ++pan;
  *s_out = s;
  *th_out = th;
  *panel_out = pan;
}

extern "C" int qams_nearest_surface_point(const qams_body_desc* desc, const double* x, double* s_out,
                                          double* theta_out, double* dist_out) {
  if (!desc || !x || !s_out || !theta_out || !dist_out) return QAMS_EINVAL;
  BodyHost b;
  const int rc = qams_copy_body(*desc, &b);
  if (rc) return rc;
  b.n = b.d.n_panels * b.d.order * b.d.n_theta;
  std::vector<double> hx(3 * (size_t)b.n);
  body_nodes_into(b, hx.data(), nullptr, nullptr, nullptr);
  int panel;
  double ds, v[3];
  qams_nearest_point(b, hx.data(), x, s_out, theta_out, &panel, dist_out, &ds, v);
  return QAMS_OK;
}

std::string qams_shape_key(const BodyCopy& bc) {
  const qams_body_desc& d = bc.d;
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  const int ints[5] = {d.profile_kind, d.n_panels, d.order, d.n_theta, d.profile_kind == 1 ? d.n_terms : 0};
  put(ints, sizeof(ints));
  if (d.profile_kind == 0) {
    const double v[3] = {d.base_radius, d.axis_length, d.curvature};
    put(v, sizeof(v));
    const int nm = (int)bc.a.size();
    put(&nm, sizeof(nm));
    put(bc.a.data(), sizeof(double) * bc.a.size());
    put(bc.b.data(), sizeof(double) * bc.b.size());
  } else {
    put(bc.series.data(), sizeof(double) * bc.series.size());
  }
  put(bc.breaks.data(), sizeof(double) * bc.breaks.size());
  return k;
}
