// Restarted GMRES on the device (Sec. 6 solver description; the paper gives
// no restart length, tolerance or orthogonalisation, readings below).
//
//  * R right-hand sides iterate together: one Krylov basis per column of the
//    [N][R] block, dot products and norms per column, a small Hessenberg
//    least-squares problem per column on the host (Givens rotations).
//  * Arnoldi: classical Gram-Schmidt applied twice, always in FP64 (basis
//    stored as complex128).
//  * QAMS_PREC_FP64: the operator is the FP64 apply; stop at
//    ||b - A x|| <= tol ||b|| per column.
//  * QAMS_PREC_FP32: iterative refinement.  The correction equation
//    A d = r is solved by the same GMRES with the FP32 apply (the FP64 basis
//    vector is rounded to complex64 on the way in and the result widened on
//    the way out) to a relative reduction inner_tol (or less, when less is
//    enough to reach tol); the inner solve stops on its Arnoldi residual
//    estimate.  After the first correction the residual r = b - A x is
//    formed with the FP64-accurate apply (float-float pair sum by default),
//    and the FP32 operator's error is measured on the same x:
//        eta = ||(A - A_32) x|| / ||x||   (per column).
//    A later correction d is small, and its residual is updated as
//        r <- r - A_32 d,   error <= eta ||d||   (to first order),
//    whenever eta ||d|| <= tol ||b|| / 2; convergence then needs
//    ||r|| + eta ||d|| <= tol ||b||.  Otherwise r is recomputed with the
//    FP64-accurate apply.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "qams_internal.h"

namespace {

using cd = std::complex<double>;
constexpr int DOT_BLOCKS = 296;  // 2 x 148 SMs
constexpr int MAXR = 16;

// partial[i][blk][r] = sum_{t in blk} conj(V_i[t][r]) w[t][r], i < ni (grid.y = i)
__global__ void multidot_kernel(const double2* __restrict__ V, long long vstride, const double2* __restrict__ w,
                                long long N, int R, double2* __restrict__ partial) {
  __shared__ double2 red[256];
  const int i = blockIdx.y;
  const double2* v = V + vstride * i;
  double2 acc[MAXR];
  for (int r = 0; r < R; ++r) acc[r] = make_double2(0.0, 0.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    for (int r = 0; r < R; ++r) {
      const double2 a = v[t * R + r], b = w[t * R + r];
      acc[r].x += a.x * b.x + a.y * b.y;
      acc[r].y += a.x * b.y - a.y * b.x;
    }
  }
  for (int r = 0; r < R; ++r) {
    red[threadIdx.x] = acc[r];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        red[threadIdx.x].x += red[threadIdx.x + s].x;
        red[threadIdx.x].y += red[threadIdx.x + s].y;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[((long long)i * gridDim.x + blockIdx.x) * R + r] = red[0];
    __syncthreads();
  }
}

// out[i][r] = sum_blk partial[i][blk][r]  (fixed order)
__global__ void reduce_partial_kernel(const double2* __restrict__ partial, int nblk, int ni, int R,
                                      double2* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ni * R) return;
  const int i = idx / R, r = idx % R;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) {
    const double2 v = partial[((long long)i * nblk + b) * R + r];
    s.x += v.x;
    s.y += v.y;
  }
  out[idx] = s;
}

// w[t][r] -= sum_{i<ni} V_i[t][r] h[i][r]   (sign = -1), or x += V y (sign = +1)
__global__ void basis_combine_kernel(const double2* __restrict__ V, long long vstride, int ni,
                                     const double2* __restrict__ h, double2* __restrict__ w, long long N, int R,
                                     double sign) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N * R) return;
  const int r = (int)(idx % R);
  double2 acc = w[idx];
  for (int i = 0; i < ni; ++i) {
    const double2 v = V[vstride * i + idx], c = h[i * R + r];
    acc.x += sign * (v.x * c.x - v.y * c.y);
    acc.y += sign * (v.x * c.y + v.y * c.x);
  }
  w[idx] = acc;
}

// dst[t][r] = src[t][r] * s[r]
__global__ void scale_cols_kernel(const double2* __restrict__ src, const double2* __restrict__ s,
                                  double2* __restrict__ dst, long long N, int R) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N * R) return;
  const double2 a = src[idx], c = s[idx % R];
  dst[idx] = make_double2(a.x * c.x - a.y * c.y, a.x * c.y + a.y * c.x);
}

__global__ void narrow_kernel(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void widen_kernel(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2(a[i].x, a[i].y);
}

// r = b - y
__global__ void residual_kernel(const double2* b, const double2* y,
                                double2* r, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) r[i] = make_double2(b[i].x - y[i].x, b[i].y - y[i].y);
}

__global__ void add_kernel(double2* __restrict__ x, const double2* __restrict__ d, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    x[i].x += d[i].x;
    x[i].y += d[i].y;
  }
}

// s[r] = 1 / sqrt(max(0, nsq[r].x)) (0 for a zero or NaN norm; the host reads the
// norms back and rejects a non-finite one)
__global__ void inv_norm_kernel(const double2* __restrict__ nsq, double2* __restrict__ s, int R) {
  const int r = threadIdx.x;
  if (r >= R) return;
  const double v = nsq[r].x;
  const double hn = isnan(v) ? v : sqrt(fmax(0.0, v));
  s[r] = make_double2(hn > 0.0 ? 1.0 / hn : 0.0, 0.0);
}

inline unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

struct Solver {
  qams_ctx* c;
  int R, m;
  long long N;
  cudaStream_t st;
  DeviceBuf V, w, partial, hbuf, hstep, t32a, t32b, t32c, t64;
  std::vector<double2> hhost;
  bool prec = false;  // right block-Jacobi preconditioning: the operator is A P^{-1}

  int init() {
    int rc;
    if ((rc = qams_dev_alloc(c, &V, sizeof(double2) * (size_t)N * R * (m + 1)))) return rc;
    if ((rc = qams_dev_alloc(c, &w, sizeof(double2) * (size_t)N * R))) return rc;
    if ((rc = qams_dev_alloc(c, &partial, sizeof(double2) * (size_t)DOT_BLOCKS * (m + 1) * R))) return rc;
    if ((rc = qams_dev_alloc(c, &hbuf, sizeof(double2) * (size_t)(m + 1) * R))) return rc;
    if ((rc = qams_dev_alloc(c, &hstep, sizeof(double2) * (size_t)(2 * (m + 1) + 2) * R))) return rc;
    if ((rc = qams_dev_alloc(c, &t32a, sizeof(float2) * (size_t)N * R))) return rc;
    if ((rc = qams_dev_alloc(c, &t32b, sizeof(float2) * (size_t)N * R))) return rc;
    if ((rc = qams_dev_alloc(c, &t32c, sizeof(float2) * (size_t)N * R))) return rc;
    if ((rc = qams_dev_alloc(c, &t64, sizeof(double2) * (size_t)N * R))) return rc;
    hhost.resize((size_t)(2 * (m + 1) + 2) * R);
    return QAMS_OK;
  }
  void release() {
    for (DeviceBuf* b : {&V, &w, &partial, &hbuf, &hstep, &t32a, &t32b, &t32c, &t64}) qams_dev_free(c, b);
  }
  double2* Vi(int i) { return (double2*)V.p + (size_t)i * N * R; }

  // y = A x (or A P^{-1} x when preconditioned) with the requested operator
  // precision; FP64 in and out
  int applies = 0;
  int op(const double2* x, double2* y, int precision) {
    ++applies;
    int rc;
    if (precision == QAMS_PREC_FP64) {
      const double2* xin = x;
      if (prec) {
        if ((rc = qams_block_apply_ptr(c, c->pinv64.p, R, x, t64.p, QAMS_PREC_FP64, false, st))) return rc;
        xin = (const double2*)t64.p;
      }
      return qams_apply_launch(c, R, xin, y, QAMS_PREC_FP64, st);
    }
    const long long n = N * R;
    narrow_kernel<<<nblk(n), 256, 0, st>>>(x, (float2*)t32a.p, n); qams_count_launch();
    const void* xin = t32a.p;
    if (prec) {
      if ((rc = qams_block_apply_ptr(c, c->pinv32.p, R, t32a.p, t32c.p, QAMS_PREC_FP32, false, st))) return rc;
      xin = t32c.p;
    }
    rc = qams_apply_launch(c, R, xin, t32b.p, QAMS_PREC_FP32, st);
    if (rc) return rc;
    widen_kernel<<<nblk(n), 256, 0, st>>>((const float2*)t32b.p, y, n); qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
    return QAMS_OK;
  }

  // y = A_32 x for FP64 x and y (no preconditioner): the FP32 operator on
  // the rounded vector, widened
  int apply32(const double2* x, double2* y) {
    ++applies;
    const long long n = N * R;
    narrow_kernel<<<nblk(n), 256, 0, st>>>(x, (float2*)t32a.p, n); qams_count_launch();
    int rc = qams_apply_launch(c, R, t32a.p, t32b.p, QAMS_PREC_FP32, st);
    if (rc) return rc;
    widen_kernel<<<nblk(n), 256, 0, st>>>((const float2*)t32b.p, y, n); qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
    return QAMS_OK;
  }

  // x <- P^{-1} x (back from the preconditioned variable), FP64
  int unprecondition(double2* x) {
    if (!prec) return QAMS_OK;
    int rc = qams_block_apply_ptr(c, c->pinv64.p, R, x, t64.p, QAMS_PREC_FP64, false, st);
    if (rc) return rc;
    QAMS_CUDA(cudaMemcpyAsync(x, t64.p, sizeof(double2) * (size_t)N * R, cudaMemcpyDeviceToDevice, st));
    return QAMS_OK;
  }

  // hhost[i][r] = <V_i, v> for i < ni
  int dots(const double2* Vbase, int ni, const double2* v) {
    multidot_kernel<<<dim3(DOT_BLOCKS, ni), 256, 0, st>>>(Vbase, N * R, v, N, R, (double2*)partial.p); qams_count_launch();
    reduce_partial_kernel<<<(ni * R + 127) / 128, 128, 0, st>>>((const double2*)partial.p, DOT_BLOCKS, ni, R,
                                                               (double2*)hbuf.p); qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
    QAMS_CUDA(cudaMemcpyAsync(hhost.data(), hbuf.p, sizeof(double2) * ni * R, cudaMemcpyDeviceToHost, st));
    QAMS_CUDA(cudaStreamSynchronize(st));
    return QAMS_OK;
  }
  // out_dev[i][r] = <V_i, v> for i < ni, left on the device
  int dots_dev(const double2* Vbase, int ni, const double2* v, double2* out_dev) {
    multidot_kernel<<<dim3(DOT_BLOCKS, ni), 256, 0, st>>>(Vbase, N * R, v, N, R, (double2*)partial.p); qams_count_launch();
    reduce_partial_kernel<<<(ni * R + 127) / 128, 128, 0, st>>>((const double2*)partial.p, DOT_BLOCKS, ni, R,
                                                               out_dev); qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
    return QAMS_OK;
  }
  int norms(const double2* v, std::vector<double>& out) {
    int rc = dots(v, 1, v);
    if (rc) return rc;
    out.resize(R);
    // a NaN must stay NaN (std::max(0, NaN) would return 0 and hide it)
    for (int r = 0; r < R; ++r) {
      const double v = hhost[r].x;
      out[r] = std::isnan(v) ? v : std::sqrt(std::max(0.0, v));
    }
    return QAMS_OK;
  }

  // GMRES for A x = b from x = 0 (x overwritten); per-column stop at
  // ||r|| <= tol * ||b||.  Returns iterations through *iters.
  //  inner = true: a correction solve inside refinement; when the Arnoldi
  //  estimate meets tol the cycle's true residual is not recomputed (the
  //  refinement forms its own residual next).
  int gmres(const double2* b, double2* x, int precision, double tol, int maxit, int* iters, double* relres,
            bool inner = false) {
    const long long n = N * R;
    QAMS_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n, st));
    std::vector<double> bn, beta;
    int rc = norms(b, bn);
    if (rc) return rc;
    for (double v : bn)
      if (!std::isfinite(v)) return QAMS_ENUMERIC;
    // r0 = b (x0 = 0)
    QAMS_CUDA(cudaMemcpyAsync(w.p, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
    beta = bn;
    int it = 0;
    std::vector<double> res(R);
    for (int r = 0; r < R; ++r) res[r] = bn[r] > 0 ? 1.0 : 0.0;
    while (true) {
      bool done = true;
      for (int r = 0; r < R; ++r) done = done && (bn[r] == 0 || beta[r] <= tol * bn[r]);
      if (done || it >= maxit) break;
      if (c->cancel && __atomic_load_n(c->cancel, __ATOMIC_RELAXED)) return QAMS_ECANCELLED;
      // V0 = r / beta
      std::vector<double2> sc(R);
      for (int r = 0; r < R; ++r) sc[r] = make_double2(beta[r] > 0 ? 1.0 / beta[r] : 0.0, 0.0);
      QAMS_CUDA(cudaMemcpyAsync(hbuf.p, sc.data(), sizeof(double2) * R, cudaMemcpyHostToDevice, st));
      scale_cols_kernel<<<nblk(n), 256, 0, st>>>((const double2*)w.p, (const double2*)hbuf.p, Vi(0), N, R); qams_count_launch();
      std::vector<cd> H((size_t)(m + 1) * m * R, 0.0), g((size_t)(m + 1) * R, 0.0), cs((size_t)m * R),
          sn((size_t)m * R);
      for (int r = 0; r < R; ++r) g[r] = beta[r];
      int j = 0;
      bool conv = false;
      for (; j < m && it < maxit; ++j) {
        if ((rc = op(Vi(j), (double2*)w.p, precision))) return rc;
        // classical Gram-Schmidt twice, the norm and the new basis vector on the device;
        // one read-back per step: [pass 0 (j+1) R][pass 1 (j+1) R][|w|^2 R]
        double2* h0 = (double2*)hstep.p;
        double2* h1 = h0 + (size_t)(j + 1) * R;
        double2* nsq = h1 + (size_t)(j + 1) * R;
        double2* scl = nsq + R;
        for (int pass = 0; pass < 2; ++pass) {
          double2* hp = pass == 0 ? h0 : h1;
          if ((rc = dots_dev(Vi(0), j + 1, (const double2*)w.p, hp))) return rc;
          basis_combine_kernel<<<nblk(n), 256, 0, st>>>(Vi(0), N * R, j + 1, hp, (double2*)w.p, N, R, -1.0); qams_count_launch();
        }
        if ((rc = dots_dev((const double2*)w.p, 1, (const double2*)w.p, nsq))) return rc;
        inv_norm_kernel<<<1, 32, 0, st>>>(nsq, scl, R); qams_count_launch();
        scale_cols_kernel<<<nblk(n), 256, 0, st>>>((const double2*)w.p, scl, Vi(j + 1), N, R); qams_count_launch();
        QAMS_CUDA(cudaGetLastError());
        const size_t nback = (size_t)(2 * (j + 1) + 1) * R;
        QAMS_CUDA(cudaMemcpyAsync(hhost.data(), h0, sizeof(double2) * nback, cudaMemcpyDeviceToHost, st));
        QAMS_CUDA(cudaStreamSynchronize(st));
        for (int pass = 0; pass < 2; ++pass)
          for (int i = 0; i <= j; ++i)
            for (int r = 0; r < R; ++r) {
              const double2 v = hhost[(size_t)(pass * (j + 1) + i) * R + r];
              H[((size_t)i * m + j) * R + r] += cd(v.x, v.y);
            }
        for (int r = 0; r < R; ++r) {
          const double v = hhost[(size_t)2 * (j + 1) * R + r].x;
          const double hn = std::isnan(v) ? v : std::sqrt(std::max(0.0, v));
          if (!std::isfinite(hn)) return QAMS_ENUMERIC;
          H[((size_t)(j + 1) * m + j) * R + r] = hn;
        }
        // Givens rotations per column: G_i = [[c*, s*], [-s, c]]
        bool all = true;
        for (int r = 0; r < R; ++r) {
          auto Hc = [&](int i, int jj) -> cd& { return H[((size_t)i * m + jj) * R + r]; };
          for (int i = 0; i < j; ++i) {
            const cd a = Hc(i, j), bb = Hc(i + 1, j);
            const cd c0 = cs[(size_t)i * R + r], s0 = sn[(size_t)i * R + r];
            Hc(i, j) = std::conj(c0) * a + std::conj(s0) * bb;
            Hc(i + 1, j) = -s0 * a + c0 * bb;
          }
          const cd a = Hc(j, j), bb = Hc(j + 1, j);
          const double den = std::sqrt(std::norm(a) + std::norm(bb));
          const cd c0 = den > 0 ? a / den : cd(1.0), s0 = den > 0 ? bb / den : cd(0.0);
          cs[(size_t)j * R + r] = c0;
          sn[(size_t)j * R + r] = s0;
          Hc(j, j) = den;
          Hc(j + 1, j) = 0.0;
          const cd gj = g[(size_t)j * R + r];
          g[(size_t)(j + 1) * R + r] = -s0 * gj;
          g[(size_t)j * R + r] = std::conj(c0) * gj;
          res[r] = bn[r] > 0 ? std::abs(g[(size_t)(j + 1) * R + r]) / bn[r] : 0.0;
          all = all && res[r] <= tol;
        }
        ++it;
        if (all) {
          ++j;
          conv = true;
          break;
        }
      }
      // x += V y, H y = g (upper triangular, per column)
      std::vector<double2> y((size_t)j * R);
      for (int r = 0; r < R; ++r) {
        std::vector<cd> yy(j);
        for (int i = j - 1; i >= 0; --i) {
          cd s = g[(size_t)i * R + r];
          for (int l = i + 1; l < j; ++l) s -= H[((size_t)i * m + l) * R + r] * yy[l];
          const cd d = H[((size_t)i * m + i) * R + r];
          yy[i] = std::abs(d) > 0 ? s / d : cd(0.0);
        }
        for (int i = 0; i < j; ++i) y[(size_t)i * R + r] = make_double2(yy[i].real(), yy[i].imag());
      }
      if (j > 0) {
        QAMS_CUDA(cudaMemcpyAsync(hbuf.p, y.data(), sizeof(double2) * j * R, cudaMemcpyHostToDevice, st));
        basis_combine_kernel<<<nblk(n), 256, 0, st>>>(Vi(0), N * R, j, (const double2*)hbuf.p, x, N, R, 1.0); qams_count_launch();
      }
      if (inner && conv) break;  // res[] holds the Arnoldi estimates
      // true residual for the restart
      if ((rc = op(x, (double2*)w.p, precision))) return rc;
      residual_kernel<<<nblk(n), 256, 0, st>>>(b, (const double2*)w.p, (double2*)w.p, n); qams_count_launch();
      QAMS_CUDA(cudaGetLastError());
      if ((rc = norms((const double2*)w.p, beta))) return rc;
      for (int r = 0; r < R; ++r) {
        if (!std::isfinite(beta[r])) return QAMS_ENUMERIC;
        res[r] = bn[r] > 0 ? beta[r] / bn[r] : 0.0;
      }
    }
    *iters = it;
    double mx = 0;
    for (int r = 0; r < R; ++r) mx = std::max(mx, res[r]);
    *relres = mx;
    return mx <= tol ? QAMS_OK : QAMS_ENOCONV;
  }
};

}  // namespace

extern "C" int qams_solve(qams_ctx* c, int R, const void* rhs, void* mu, const qams_solve_opts* opts,
                          qams_solve_stats* stats, void* stream) {
  if (!c || R < 1 || R > MAXR || !rhs || !mu || !c->assembled) return QAMS_EINVAL;
  qams_solve_opts o;
  qams_solve_opts_default(&o);
  if (opts) o = *opts;
  if (o.precision != QAMS_PREC_FP64 && o.precision != QAMS_PREC_FP32) return QAMS_EINVAL;
  if (o.precision == QAMS_PREC_FP32 && o.residual != QAMS_PREC_FP64 && o.residual != QAMS_PREC_FF) return QAMS_EINVAL;
  if (o.restart < 1 || o.restart > 200 || o.max_iters < 1 || !(o.tol > 0)) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  QAMS_CUDA(cudaEventCreate(&e0));
  QAMS_CUDA(cudaEventCreate(&e1));
  QAMS_CUDA(cudaEventRecord(e0, st));
  Solver S{c, R, o.restart, c->N, st};
  int rc = QAMS_OK;
  if (o.precondition && !c->have_precond) {
    rc = qams_precond_launch(c, st);
    if (rc) return rc;
    c->have_precond = true;
  }
  S.prec = o.precondition != 0;
  rc = S.init();
  qams_solve_stats s{};
  const long long n = c->N * R;
  if (!rc) {
    if (o.precision == QAMS_PREC_FP64) {
      rc = S.gmres((const double2*)rhs, (double2*)mu, QAMS_PREC_FP64, o.tol, o.max_iters, &s.iterations,
                   &s.rel_residual);
      if (!rc || rc == QAMS_ENOCONV) {
        const int rc2 = S.unprecondition((double2*)mu);
        if (rc2) rc = rc2;
      }
      s.refinements = 0;
    } else {
      // iterative refinement: x = 0, r = b; repeat d = GMRES_32(r), x += d and
      // a new r (FP64-accurate apply, or the residual update, see the header)
      DeviceBuf xr, rr, dd, yy;
      rc = qams_dev_alloc(c, &xr, sizeof(double2) * n);
      if (!rc) rc = qams_dev_alloc(c, &rr, sizeof(double2) * n);
      if (!rc) rc = qams_dev_alloc(c, &dd, sizeof(double2) * n);
      if (!rc) rc = qams_dev_alloc(c, &yy, sizeof(double2) * n);
      if (!rc) {
        cudaMemsetAsync(xr.p, 0, sizeof(double2) * n, st);
        cudaMemcpyAsync(rr.p, rhs, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st);
        std::vector<double> bn, rn, dn, xn, en;
        std::vector<double> eta_op;  // measured FP32 operator error per column (empty: not yet)
        rc = S.norms((const double2*)rhs, bn);
        int total = 0;
        double rel = 1.0;
        int fp64_applies = 0;
        for (int k = 0; !rc && k < o.max_refine; ++k) {
          int its = 0;
          double inner_rel = 0;
          // a reduction of tol/rel is enough for this correction (0.3: margin)
          const double want = k == 0 ? o.inner_tol : std::max(o.inner_tol, std::min(0.1, 0.3 * o.tol / rel));
          int irc = S.gmres((const double2*)rr.p, (double2*)dd.p, QAMS_PREC_FP32, want,
                            std::max(1, o.max_iters - total), &its, &inner_rel, true);
          total += its;
          if (irc && irc != QAMS_ENOCONV) { rc = irc; break; }
          if ((rc = S.unprecondition((double2*)dd.p))) break;
          add_kernel<<<nblk(n), 256, 0, st>>>((double2*)xr.p, (const double2*)dd.p, n); qams_count_launch();
          bool update = false;
          if (!eta_op.empty()) {
            if ((rc = S.norms((const double2*)dd.p, dn))) break;
            update = true;
            for (int r = 0; r < R; ++r) update = update && eta_op[r] * dn[r] <= 0.5 * o.tol * bn[r];
          }
          if (update) {
            // r <- r - A_32 d
            if ((rc = S.apply32((const double2*)dd.p, (double2*)yy.p))) break;
            residual_kernel<<<nblk(n), 256, 0, st>>>((const double2*)rr.p, (const double2*)yy.p, (double2*)rr.p, n); qams_count_launch();
            if ((rc = S.norms((const double2*)rr.p, rn))) break;
            rel = 0;
            for (int r = 0; r < R; ++r) {
              if (!std::isfinite(rn[r])) { rc = QAMS_ENUMERIC; break; }
              rel = std::max(rel, bn[r] > 0 ? (rn[r] + eta_op[r] * dn[r]) / bn[r] : 0.0);
            }
          } else {
            rc = qams_apply_launch(c, R, xr.p, yy.p, o.residual, st);
            ++fp64_applies;
            if (rc) break;
            residual_kernel<<<nblk(n), 256, 0, st>>>((const double2*)rhs, (const double2*)yy.p, (double2*)rr.p, n); qams_count_launch();
            if ((rc = S.norms((const double2*)rr.p, rn))) break;
            rel = 0;
            for (int r = 0; r < R; ++r) {
              if (!std::isfinite(rn[r])) { rc = QAMS_ENUMERIC; break; }
              rel = std::max(rel, bn[r] > 0 ? rn[r] / bn[r] : 0.0);
            }
            if (!rc && eta_op.empty() && rel > o.tol) {
              // eta = ||A x - A_32 x|| / ||x||, dd reused for A_32 x
              if ((rc = S.apply32((const double2*)xr.p, (double2*)dd.p))) break;
              residual_kernel<<<nblk(n), 256, 0, st>>>((const double2*)yy.p, (const double2*)dd.p, (double2*)dd.p, n); qams_count_launch();
              if ((rc = S.norms((const double2*)dd.p, en))) break;
              if ((rc = S.norms((const double2*)xr.p, xn))) break;
              eta_op.assign(R, 0.0);
              for (int r = 0; r < R; ++r) eta_op[r] = xn[r] > 0 ? en[r] / xn[r] : 0.0;
            }
          }
          s.refinements = k + 1;
          if (rc || rel <= o.tol || total >= o.max_iters) break;
        }
        s.iterations = total;
        s.rel_residual = rel;
        s.applies_fp64 = fp64_applies;
        if (!rc && rel > o.tol) rc = QAMS_ENOCONV;
        if (!rc || rc == QAMS_ENOCONV)
          cudaMemcpyAsync(mu, xr.p, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st);
      }
      qams_dev_free(c, &yy);
      qams_dev_free(c, &xr);
      qams_dev_free(c, &rr);
      qams_dev_free(c, &dd);
    }
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  s.solve_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (o.precision == QAMS_PREC_FP64) s.applies_fp64 = S.applies; else s.applies_fp32 = S.applies;
  S.release();
  if (stats) *stats = s;
  return rc;
}

extern "C" void qams_solve_opts_default(qams_solve_opts* o) {
  if (!o) return;
  o->precision = QAMS_PREC_FP32;
  o->restart = 50;
  o->max_iters = 1000;
  o->tol = 1e-11;
  o->inner_tol = 1e-5;
  o->max_refine = 12;
  o->residual = QAMS_PREC_FF;
  o->precondition = 1;
}
