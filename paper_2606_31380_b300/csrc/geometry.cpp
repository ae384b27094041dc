// Host-side geometry and Nystrom nodes (Eq. para_quasi, Sec. 3.1, Eq. sx).
//
// Reference shape of one body, s in [-pi/2, pi/2]:
//   u = (1 + sin s)/2, rho(u) = base (1 + sum a_m cos 2 pi m u + b_m sin 2 pi m u)
//   r(s) = rho(u) cos s, l(s) = L (u - 1/2)
//   axis: planar arc of curvature kappa, frame e1 = (cos kl, 0, -sin kl),
//         e2 = (0, 1, 0), e3 = (sin kl, 0, cos kl) (rotation minimising)
//   y(s, theta) = gamma(l) + r (cos theta e1 + sin theta e2)
//   d_s = l'(1 - kappa r cos theta) e3 + r' e_r,  d_theta = r e_theta
//   n = (A e_r - B e3)/sqrt(A^2 + B^2), A = l'(1 - kappa r cos theta), B = r'
//   |J| = r sqrt(A^2 + B^2), w = |J| (2 pi / n_theta) omega_l.
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

struct Shape {
  double base, L, kappa;
  const double* a;
  const double* b;
  int na, nb;
  double rho(double u) const {
    double s = 1.0;
    for (int m = 1; m <= na; ++m) s += a[m - 1] * std::cos(2 * M_PI * m * u);
    for (int m = 1; m <= nb; ++m) s += b[m - 1] * std::sin(2 * M_PI * m * u);
    return base * s;
  }
  double drho(double u) const {
    double s = 0.0;
    for (int m = 1; m <= na; ++m) s -= a[m - 1] * 2 * M_PI * m * std::sin(2 * M_PI * m * u);
    for (int m = 1; m <= nb; ++m) s += b[m - 1] * 2 * M_PI * m * std::cos(2 * M_PI * m * u);
    return base * s;
  }
  // local point, normal and |J| at (s, theta)
  void eval(double s, double th, double p[3], double nrm[3], double* jac) const {
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
    double ct = std::cos(th), st = std::sin(th);
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
  for (auto& bh : c->bodies) {
    const qams_body_desc& d = bh.d;
    Shape sh{d.base_radius, d.axis_length, d.curvature, bh.a.data(), bh.b.data(),
             (int)bh.a.size(), (int)bh.b.size()};
    std::vector<double> gx, gw;
    qams_gauss_legendre(d.order, gx, gw);
    long long idx = bh.offset;
    double dth = 2.0 * M_PI / d.n_theta;
    for (int i = 0; i < d.n_panels; ++i) {
      double lo = -M_PI / 2 + M_PI * i / d.n_panels;
      double hi = -M_PI / 2 + M_PI * (i + 1) / d.n_panels;
      for (int l = 0; l < d.order; ++l) {
        double s = 0.5 * (lo + hi) + 0.5 * (hi - lo) * gx[l];
        double om = 0.5 * (hi - lo) * gw[l];
        for (int j = 0; j < d.n_theta; ++j, ++idx) {
          double p[3], nl[3], jac;
          sh.eval(s, j * dth, p, nl, &jac);
          for (int r = 0; r < 3; ++r) {
            double xr = d.center[r], nr = 0.0;
            for (int q = 0; q < 3; ++q) {
              xr += d.rotation[3 * r + q] * p[q];
              nr += d.rotation[3 * r + q] * nl[q];
            }
            c->hx[3 * idx + r] = xr;
            c->hn[3 * idx + r] = nr;
          }
          c->hw[idx] = jac * dth * om;
          c->hj[idx] = jac;
        }
      }
    }
  }
  return QAMS_OK;
}
