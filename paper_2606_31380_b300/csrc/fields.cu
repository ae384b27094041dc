// Right-hand sides and far field (Sec. 6): plane-wave incidence and the
// far-field pattern of the combined-layer density.
#include <cmath>

#include "phase.cuh"
#include "qams_internal.h"

namespace {

constexpr int MAXR = 16;

// rhs[t][r] = -exp(ik d_r . x_t)
__global__ void incident_kernel(const qd4* __restrict__ x, long long N, int R, const double* __restrict__ dirs,
                                double k, double2* __restrict__ rhs) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N * R) return;
  const long long t = idx / R;
  const int r = (int)(idx % R);
  const qd4 p = x[t];
  const double ph = k * (dirs[3 * r] * p.x + dirs[3 * r + 1] * p.y + dirs[3 * r + 2] * p.z);
  double s, c;
  sincos(ph, &s, &c);
  rhs[idx] = make_double2(-c, -s);
}

// One CTA per direction; R right-hand sides at a time (R <= MAXR).
__global__ void farfield_kernel(const qd4* __restrict__ x, const qd4* __restrict__ n, long long N,
                                const double2* __restrict__ mu, int R, int r0, int rc,
                                const double* __restrict__ dirs, double k, double eta,
                                double2* __restrict__ uinf) {
  __shared__ double2 red[256];
  __shared__ double2 ph[PH_N];
  phase_table_fill(ph);
  __syncthreads();
  const int m = blockIdx.x;
  const double hx = dirs[3 * m], hy = dirs[3 * m + 1], hz = dirs[3 * m + 2];
  double2 acc[MAXR];
  for (int r = 0; r < rc; ++r) acc[r] = make_double2(0.0, 0.0);
  for (long long s = threadIdx.x; s < N; s += blockDim.x) {
    const qd4 p = x[s];
    const qd4 q = n[s];
    double sn, cs;
    sincos_table(-k * (hx * p.x + hy * p.y + hz * p.z), ph, &sn, &cs);
    // (-ik xhat.n - i eta) e^{-ik xhat.y} w
    const double fi = -(k * (hx * q.x + hy * q.y + hz * q.z) + eta) * p.w;
    const double fre = -sn * fi, fim = cs * fi;
    for (int r = 0; r < rc; ++r) {
      const double2 v = mu[s * R + r0 + r];
      acc[r].x += fre * v.x - fim * v.y;
      acc[r].y += fre * v.y + fim * v.x;
    }
  }
  for (int r = 0; r < rc; ++r) {
    red[threadIdx.x] = acc[r];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        red[threadIdx.x].x += red[threadIdx.x + w].x;
        red[threadIdx.x].y += red[threadIdx.x + w].y;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double f = 0.079577471545947667884;
      uinf[(long long)m * R + r0 + r] = make_double2(red[0].x * f, red[0].y * f);
    }
    __syncthreads();
  }
}

// Scattered field at off-surface points (Sec. 6, the point-source check):
//   u(x_p) = sum_y [(ik/rho - 1/rho^2) n(y).(y - x_p) - i eta] e^{ik rho}/(4 pi rho) w mu(y),
// rho = |x_p - y|, by the smooth rule on the surface nodes.  One CTA per
// point, R right-hand sides at a time (R <= MAXR).
__global__ void field_kernel(const qd4* __restrict__ x, const qd4* __restrict__ n, long long N,
                             const double2* __restrict__ mu, int R, int r0, int rc,
                             const double* __restrict__ pts, double k, double eta,
                             double2* __restrict__ u) {
  __shared__ double2 red[256];
  const int m = blockIdx.x;
  const double px = pts[3 * m], py = pts[3 * m + 1], pz = pts[3 * m + 2];
  double2 acc[MAXR];
  for (int r = 0; r < rc; ++r) acc[r] = make_double2(0.0, 0.0);
  for (long long s = threadIdx.x; s < N; s += blockDim.x) {
    const qd4 p = x[s];
    const qd4 q = n[s];
    const double dx = p.x - px, dy = p.y - py, dz = p.z - pz;  // y - x_p
    const double rho2 = dx * dx + dy * dy + dz * dz;
    const double inv = rsqrt(rho2);
    const double rho = rho2 * inv;
    const double nd = (q.x * dx + q.y * dy + q.z * dz) * inv;  // n.(y - x)/rho
    double sn, cs;
    sincos(k * rho, &sn, &cs);
    // f = (ik - 1/rho) nd - i eta;  K w = f (cos + i sin) w / (4 pi rho)
    const double fre = -nd * inv, fim = k * nd - eta;
    const double g = 0.079577471545947667884 * inv * p.w;
    const double kre = (fre * cs - fim * sn) * g, kim = (fre * sn + fim * cs) * g;
    for (int r = 0; r < rc; ++r) {
      const double2 v = mu[s * R + r0 + r];
      acc[r].x += kre * v.x - kim * v.y;
      acc[r].y += kre * v.y + kim * v.x;
    }
  }
  for (int r = 0; r < rc; ++r) {
    red[threadIdx.x] = acc[r];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        red[threadIdx.x].x += red[threadIdx.x + w].x;
        red[threadIdx.x].y += red[threadIdx.x + w].y;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) u[(long long)m * R + r0 + r] = red[0];
    __syncthreads();
  }
}

}  // namespace

int qams_incident_launch(qams_ctx* c, int R, const double* dirs_host, void* rhs, cudaStream_t st) {
  DeviceBuf d;
  int rc = qams_dev_alloc(c, &d, sizeof(double) * 3 * R);
  if (rc) return rc;
  QAMS_CUDA(cudaMemcpyAsync(d.p, dirs_host, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, st));
  const long long n = c->N * R;
  incident_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const qd4*)c->x64.p, c->N, R,
                                                               (const double*)d.p, c->k, (double2*)rhs); qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  QAMS_CUDA(cudaStreamSynchronize(st));
  qams_dev_free(c, &d);
  return QAMS_OK;
}

int qams_farfield_launch(qams_ctx* c, int R, const void* mu, int M, const double* dirs_host, void* uinf,
                         cudaStream_t st) {
  DeviceBuf d;
  int rc = qams_dev_alloc(c, &d, sizeof(double) * 3 * M);
  if (rc) return rc;
  QAMS_CUDA(cudaMemcpyAsync(d.p, dirs_host, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, st));
  for (int r0 = 0; r0 < R; r0 += MAXR) {
    const int cnt = std::min(MAXR, R - r0);
    farfield_kernel<<<M, 256, 0, st>>>((const qd4*)c->x64.p, (const qd4*)c->n64.p, c->N,
                                       (const double2*)mu, R, r0, cnt, (const double*)d.p, c->k, c->eta,
                                       (double2*)uinf); qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
  }
  QAMS_CUDA(cudaStreamSynchronize(st));
  qams_dev_free(c, &d);
  return QAMS_OK;
}

int qams_field_launch(qams_ctx* c, int R, const void* mu, int M, const double* pts_host, void* u,
                      cudaStream_t st) {
  DeviceBuf d;
  int rc = qams_dev_alloc(c, &d, sizeof(double) * 3 * M);
  if (rc) return rc;
  QAMS_CUDA(cudaMemcpyAsync(d.p, pts_host, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, st));
  for (int r0 = 0; r0 < R; r0 += MAXR) {
    const int cnt = std::min(MAXR, R - r0);
    field_kernel<<<M, 256, 0, st>>>((const qd4*)c->x64.p, (const qd4*)c->n64.p, c->N, (const double2*)mu, R,
                                    r0, cnt, (const double*)d.p, c->k, c->eta, (double2*)u); qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
  }
  QAMS_CUDA(cudaStreamSynchronize(st));
  qams_dev_free(c, &d);
  return QAMS_OK;
}
