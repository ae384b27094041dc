// Right-hand sides and far field (Sec. 6): plane-wave incidence and the
// far-field pattern of the combined-layer density.
#include <cmath>

#include "ffloat.cuh"
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

// Scattered field at off-surface points (Sec. 6, the point-source check):
//   u(x_p) = sum_y [(ik/rho - 1/rho^2) n(y).(y - x_p) - i eta] e^{ik rho}/(4 pi rho) w mu(y),
// rho = |x_p - y|, by the smooth rule on the surface nodes.  One CTA per
// point, R right-hand sides at a time (R <= MAXR).
__global__ void field_kernel(const qd4* __restrict__ x, const qd4* __restrict__ n, long long N,
                             const double2* __restrict__ mu, int R, int r0, int rc,
                             const double* __restrict__ pts, double k, double eta,
                             double2* __restrict__ u) {
  __shared__ double2 red[256];
  __shared__ double2 ph[PH_N];
  phase_table_fill(ph);
  __syncthreads();
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
    sincos_table(k * rho, ph, &sn, &cs);
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

// sigma = w mu as float-float (re hi, re lo, im hi, im lo), [N][R]
__global__ void sigma_ff_kernel(const qd4* __restrict__ x, const double2* __restrict__ mu, float4* __restrict__ out,
                                long long N, int R) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N * R) return;
  const double w = x[idx / R].w;
  const double2 v = mu[idx];
  const ff re = ff_from_double(v.x * w), im = ff_from_double(v.y * w);
  out[idx] = make_float4(re.hi, re.lo, im.hi, im.lo);
}

// Far field with the per-node work in float-float: for body b with centre c_b
// and local nodes x~ = y - c_b,
//   e^{-ik xhat.y} = e^{-ik xhat.c_b} e^{-ik xhat.x~},
// the first factor in FP64 once per (direction, body), the second and the
// amplitude -i (k xhat.n + eta) w mu per node in float-float (FP32 pipe).
// One CTA per direction; bodies in chunks of FF_BCHUNK for the FP64 factors.
constexpr int FF_BCHUNK = 256;

template <int RC>
__global__ void farfield_ff_kernel(const qd4* __restrict__ centers, const long long* __restrict__ boff, int nb,
                                   const float4* __restrict__ xhi, const float4* __restrict__ xlo,
                                   const float4* __restrict__ nhi, const float4* __restrict__ nlo,
                                   const float4* __restrict__ sig, int R, int r0,
                                   const double* __restrict__ dirs, double k, double eta,
                                   double2* __restrict__ uinf) {
  __shared__ float4 tab[256];
  __shared__ double2 ph0[FF_BCHUNK];
  __shared__ double2 red[256];
  ff_phase_table_fill(tab);
  const int m = blockIdx.x, tid = threadIdx.x;
  const double hx = dirs[3 * m], hy = dirs[3 * m + 1], hz = dirs[3 * m + 2];
  const ff hxf = ff_from_double(hx), hyf = ff_from_double(hy), hzf = ff_from_double(hz);
  const ff kf = ff_from_double(k), mkf = ff_from_double(-k), etaf = ff_from_double(eta);
  double2 tot[RC];
#pragma unroll
  for (int r = 0; r < RC; ++r) tot[r] = make_double2(0.0, 0.0);
  for (int b0 = 0; b0 < nb; b0 += FF_BCHUNK) {
    const int nbc = min(FF_BCHUNK, nb - b0);
    __syncthreads();
    for (int b = tid; b < nbc; b += blockDim.x) {
      const qd4 c = centers[b0 + b];
      double sn, cs;
      sincos(-k * (hx * c.x + hy * c.y + hz * c.z), &sn, &cs);
      ph0[b] = make_double2(cs, sn);
    }
    __syncthreads();
    for (int b = 0; b < nbc; ++b) {
      const long long send = boff[b0 + b + 1];
      ff ar[RC], ai[RC];
#pragma unroll
      for (int r = 0; r < RC; ++r) ar[r] = ai[r] = ff{0.f, 0.f};
      for (long long s = boff[b0 + b] + tid; s < send; s += blockDim.x) {
        const float4 ph = xhi[s], pl = xlo[s], qh = nhi[s], ql = nlo[s];
        const ff dot = ff_add(ff_add(ff_mul(hxf, ff{ph.x, pl.x}), ff_mul(hyf, ff{ph.y, pl.y})),
                              ff_mul(hzf, ff{ph.z, pl.z}));
        ff sn, cs;
        ff_sincos(ff_mul(mkf, dot), tab, &sn, &cs);
        const ff hn = ff_add(ff_add(ff_mul(hxf, ff{qh.x, ql.x}), ff_mul(hyf, ff{qh.y, ql.y})),
                             ff_mul(hzf, ff{qh.z, ql.z}));
        const ff a = ff_add(ff_mul(kf, hn), etaf);
        // -i a (cos + i sin) = a sin - i a cos
        const ff fre = ff_mul(a, sn), fim = ff_neg(ff_mul(a, cs));
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          const float4 v = sig[s * R + r0 + r];
          const ff vr{v.x, v.y}, vi{v.z, v.w};
          ar[r] = ff_add(ar[r], ff_sub(ff_mul(fre, vr), ff_mul(fim, vi)));
          ai[r] = ff_add(ai[r], ff_add(ff_mul(fre, vi), ff_mul(fim, vr)));
        }
      }
      const double2 e0 = ph0[b];
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        const double xr = ff_to_double(ar[r]), xi = ff_to_double(ai[r]);
        tot[r].x += e0.x * xr - e0.y * xi;
        tot[r].y += e0.x * xi + e0.y * xr;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    red[tid] = tot[r];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (tid < w) {
        red[tid].x += red[tid + w].x;
        red[tid].y += red[tid + w].y;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const double f = 0.079577471545947667884;
      uinf[(long long)m * R + r0 + r] = make_double2(red[0].x * f, red[0].y * f);
    }
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
  DeviceBuf sg;
  if ((rc = qams_dev_alloc(c, &sg, sizeof(float4) * (size_t)c->N * R))) {
    qams_dev_free(c, &d);
    return rc;
  }
  const long long n = c->N * R;
  sigma_ff_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const qd4*)c->x64.p, (const double2*)mu,
                                                                (float4*)sg.p, c->N, R); qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  for (int r0 = 0; r0 < R;) {
    const int left = R - r0;
    const int cnt = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    auto go = [&](auto kern) {
      kern<<<M, 256, 0, st>>>((const qd4*)c->centers.p, (const long long*)c->boff.p, (int)c->bodies.size(),
                              (const float4*)c->x32.p, (const float4*)c->x32lo.p, (const float4*)c->n32.p,
                              (const float4*)c->n32lo.p, (const float4*)sg.p, R, r0, (const double*)d.p, c->k,
                              c->eta, (double2*)uinf);
      qams_count_launch();
    };
    switch (cnt) {
      case 16: go(farfield_ff_kernel<16>); break;
      case 8: go(farfield_ff_kernel<8>); break;
      case 4: go(farfield_ff_kernel<4>); break;
      case 2: go(farfield_ff_kernel<2>); break;
      default: go(farfield_ff_kernel<1>); break;
    }
    QAMS_CUDA(cudaGetLastError());
    r0 += cnt;
  }
  QAMS_CUDA(cudaStreamSynchronize(st));
  qams_dev_free(c, &sg);
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
  return qams_near_correction(c, R, mu, M, pts_host, u, st);
}
