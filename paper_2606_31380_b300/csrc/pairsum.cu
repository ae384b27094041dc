// Inter-body pair sum (Eq. multi2part): the off-diagonal blocks of Eq.
// linearsys applied matrix-free,
//   y_t = sum_{s not in body(t)} K(x_t, y_s) sigma_s,
//   K   = e^{ik rho}/(4 pi rho) [(ik/rho - 1/rho^2) n_s.(y_s - x_t) - i eta].
//
// Work decomposition: a CTA owns TILE consecutive targets of one body (one
// per thread) and a contiguous range of source bodies; sources are staged
// CHUNK at a time in shared memory and read as broadcasts.  With several
// source ranges per tile the partial sums go to a [split][N][rc] buffer and
// a second kernel adds them in a fixed order (deterministic result).
//
// FP32 path: positions are body-local, x = c_b + x~.  For a body pair (a,b)
// with dc = c_a - c_b (FP64), rho0 = |dc| and d = x~_t - y~_s:
//   rho^2 = rho0^2 + e,  e = 2 dc.d + |d|^2,  rho - rho0 = e/(rho + rho0),
// so the phase k(rho - rho0) is formed from O(|d|) quantities and the large
// part e^{ik rho0} is applied once per (target, source body) in FP64.
#include <cmath>

#include "ffloat.cuh"
#include "phase.cuh"
#include "qams_internal.h"

namespace {

constexpr int TILE = 128;
constexpr int CHUNK = 128;
constexpr int BODY_BATCH = 32;  // source bodies whose body-pair constants are formed together
constexpr float INV_2PI = 0.15915494309189535f;
constexpr float TWO_PI_HI = 6.28318548202514648f;    // float(2 pi)
constexpr float TWO_PI_LO = -1.7484555314695172e-7f;  // 2 pi - TWO_PI_HI

// TT targets per thread (tile of TT x TILE targets): each source read from
// shared memory serves TT independent pair evaluations.
template <int RC, int TT>
__global__ void __launch_bounds__(TILE) pairsum_f32_kernel(
    const TargetTile* __restrict__ tiles, const SourceSplit* __restrict__ splits,
    const long long* __restrict__ boff, const qd4* __restrict__ centers,
    const float4* __restrict__ x32, const float4* __restrict__ n32, const float2* __restrict__ sigma,
    int R, int r0, double k, double eta, float2* __restrict__ out, long long split_stride, int out_ld,
    int out_r0) {
  __shared__ float4 sp[CHUNK];
  __shared__ float4 sq[CHUNK];
  __shared__ float2 ss[CHUNK][RC];
  __shared__ float4 bdc[BODY_BATCH];  // per source body: dc = c_a - c_b (x, y, z), rho0
  __shared__ float4 bph[BODY_BATCH];  // rho0^2, cos k rho0, sin k rho0

  const TargetTile tile = tiles[blockIdx.x];
  const SourceSplit split = splits[blockIdx.y];
  const int tid = threadIdx.x;
  bool active[TT];
  long long t[TT];
  float4 xt[TT];
#pragma unroll
  for (int u = 0; u < TT; ++u) {
    active[u] = tid + u * TILE < tile.count;
    t[u] = tile.start + (active[u] ? tid + u * TILE : 0);
    xt[u] = x32[t[u]];
  }
  const float kf = (float)k, etaf = (float)eta;

  float2 tot[TT][RC];
#pragma unroll
  for (int u = 0; u < TT; ++u)
#pragma unroll
    for (int r = 0; r < RC; ++r) tot[u][r] = make_float2(0.f, 0.f);

  for (int bb = split.begin; bb < split.end; bb += BODY_BATCH) {
    // the tile's targets share one body: its FP64 body-pair constants are
    // formed once per CTA, one source body per lane of the first warp
    __syncthreads();
    if (tid < BODY_BATCH && bb + tid < split.end) {
      const qd4 ca = centers[tile.body], cb = centers[bb + tid];
      const double dcx = ca.x - cb.x, dcy = ca.y - cb.y, dcz = ca.z - cb.z;
      const double rho0 = sqrt(dcx * dcx + dcy * dcy + dcz * dcz);
      double s0d, c0d;
      sincos(k * rho0, &s0d, &c0d);
      bdc[tid] = make_float4((float)dcx, (float)dcy, (float)dcz, (float)rho0);
      bph[tid] = make_float4((float)(rho0 * rho0), (float)c0d, (float)s0d, 0.f);
    }
    __syncthreads();
  for (int b = bb; b < min(split.end, bb + BODY_BATCH); ++b) {
    if (b == tile.body) continue;
    const float4 dcv = bdc[b - bb], phv = bph[b - bb];
    const float fx = dcv.x, fy = dcv.y, fz = dcv.z;
    const float rho0f = dcv.w;
    const float r02 = phv.x;
    float At[TT];
#pragma unroll
    for (int u = 0; u < TT; ++u) At[u] = fx * xt[u].x + fy * xt[u].y + fz * xt[u].z;

    float2 acc[TT][RC];
#pragma unroll
    for (int u = 0; u < TT; ++u)
#pragma unroll
      for (int r = 0; r < RC; ++r) acc[u][r] = make_float2(0.f, 0.f);

    const long long send = boff[b + 1];
    for (long long s0 = boff[b]; s0 < send; s0 += CHUNK) {
      __syncthreads();
      const long long i = s0 + tid;
      if (i < send) {
        float4 p = x32[i];
        float4 q = n32[i];
        p.w = fx * p.x + fy * p.y + fz * p.z;  // dc . y~_s
        q.w = fx * q.x + fy * q.y + fz * q.z;  // n_s . dc
        sp[tid] = p;
        sq[tid] = q;
#pragma unroll
        for (int r = 0; r < RC; ++r) ss[tid][r] = sigma[i * R + r0 + r];
      }
      __syncthreads();
      const int cnt = (int)min((long long)CHUNK, send - s0);
#pragma unroll (TT == 1 ? 4 : 2)
      for (int j = 0; j < cnt; ++j) {
        const float4 p = sp[j];
        const float4 q = sq[j];
#pragma unroll
        for (int u = 0; u < TT; ++u) {
          const float dx = xt[u].x - p.x, dy = xt[u].y - p.y, dz = xt[u].z - p.z;
          const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float e = fmaf(2.f, At[u] - p.w, dd);
          const float r2 = r02 + e;
          const float rinv = rsqrtf(r2);
          const float rho = r2 * rinv;
          const float delta = __fdividef(e, rho + rho0f);
          const float ph = kf * delta;
          const float nq = rintf(ph * INV_2PI);
          float red = fmaf(-nq, TWO_PI_HI, ph);
          red = fmaf(-nq, TWO_PI_LO, red);
          float sn, cs;
          __sincosf(red, &sn, &cs);
          const float nyx = -(q.w + fmaf(q.x, dx, fmaf(q.y, dy, q.z * dz)));
          const float are = -nyx * rinv * rinv;
          const float aim = fmaf(kf * nyx, rinv, -etaf);
          const float kre = (cs * are - sn * aim) * rinv;
          const float kim = (sn * are + cs * aim) * rinv;
#pragma unroll
          for (int r = 0; r < RC; ++r) {
            const float2 sg = ss[j][r];
            acc[u][r].x = fmaf(kre, sg.x, fmaf(-kim, sg.y, acc[u][r].x));
            acc[u][r].y = fmaf(kre, sg.y, fmaf(kim, sg.x, acc[u][r].y));
          }
        }
      }
    }
    const float c0 = phv.y, s0f = phv.z;
#pragma unroll
    for (int u = 0; u < TT; ++u)
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        tot[u][r].x += c0 * acc[u][r].x - s0f * acc[u][r].y;
        tot[u][r].y += c0 * acc[u][r].y + s0f * acc[u][r].x;
      }
  }
  }
  const float inv4pi = 0.079577471545947668f;
#pragma unroll
  for (int u = 0; u < TT; ++u) {
    if (!active[u]) continue;
    float2* o = out + split_stride * blockIdx.y + t[u] * out_ld + out_r0;
#pragma unroll
    for (int r = 0; r < RC; ++r) o[r] = make_float2(tot[u][r].x * inv4pi, tot[u][r].y * inv4pi);
  }
}

template <int RC>
__global__ void __launch_bounds__(TILE) pairsum_f64_kernel(
    const TargetTile* __restrict__ tiles, const SourceSplit* __restrict__ splits,
    const long long* __restrict__ boff, const qd4* __restrict__ x64, const qd4* __restrict__ n64,
    const double2* __restrict__ sigma, int R, int r0, double k, double eta, double2* __restrict__ out,
    long long split_stride, int out_ld, int out_r0) {
  __shared__ qd4 sp[CHUNK];
  __shared__ qd4 sq[CHUNK];
  __shared__ double2 ss[CHUNK][RC];
  __shared__ double2 ph[PH_N];

  phase_table_fill(ph);
  const TargetTile tile = tiles[blockIdx.x];
  const SourceSplit split = splits[blockIdx.y];
  const int tid = threadIdx.x;
  const bool active = tid < tile.count;
  const long long t = tile.start + (active ? tid : 0);
  const qd4 xt = x64[t];

  double2 acc[RC];
#pragma unroll
  for (int r = 0; r < RC; ++r) acc[r] = make_double2(0.0, 0.0);

  for (int b = split.begin; b < split.end; ++b) {
    if (b == tile.body) continue;
    const long long send = boff[b + 1];
    for (long long s0 = boff[b]; s0 < send; s0 += CHUNK) {
      __syncthreads();
      const long long i = s0 + tid;
      if (i < send) {
        sp[tid] = x64[i];
        sq[tid] = n64[i];
#pragma unroll
        for (int r = 0; r < RC; ++r) ss[tid][r] = sigma[i * R + r0 + r];
      }
      __syncthreads();
      const int cnt = (int)min((long long)CHUNK, send - s0);
#pragma unroll 2
      for (int j = 0; j < cnt; ++j) {
        const qd4 p = sp[j];
        const qd4 q = sq[j];
        const double dx = p.x - xt.x, dy = p.y - xt.y, dz = p.z - xt.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = rsqrt(r2);
        const double rho = r2 * rinv;
        double sn, cs;
        sincos_table(k * rho, ph, &sn, &cs);
        const double nyx = q.x * dx + q.y * dy + q.z * dz;
        const double are = -nyx * rinv * rinv;
        const double aim = k * nyx * rinv - eta;
        const double kre = (cs * are - sn * aim) * rinv;
        const double kim = (sn * are + cs * aim) * rinv;
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          const double2 s = ss[j][r];
          acc[r].x += kre * s.x - kim * s.y;
          acc[r].y += kre * s.y + kim * s.x;
        }
      }
    }
  }
  if (active) {
    const double inv4pi = 0.079577471545947667884;
    double2* o = out + split_stride * blockIdx.y + t * out_ld + out_r0;
#pragma unroll
    for (int r = 0; r < RC; ++r) o[r] = make_double2(acc[r].x * inv4pi, acc[r].y * inv4pi);
  }
}

// Float-float path (FP64-accurate result from FP32 arithmetic, ~48 bits):
// the same body-local decomposition as the FP32 path,
//   rho^2 = rho0^2 + e,  e = 2 dc.d + |d|^2,  rho - rho0 = e/(rho + rho0),
// with every per-pair quantity in float-float.  The body-pair constants
// (dc, rho0, dc.x~_t, dc.y~_s, n_s.dc) are formed in FP64 once per target or
// per staged source; the per-pair work has no FP64 instruction.  Partial sums
// go to FP64 every CHUNK sources, and e^{ik rho0} is applied in FP64 per
// source body.  sigma and the result are complex128.
template <int RC>
__global__ void __launch_bounds__(TILE) pairsum_ff_kernel(
    const TargetTile* __restrict__ tiles, const SourceSplit* __restrict__ splits,
    const long long* __restrict__ boff, const qd4* __restrict__ centers, const float4* __restrict__ xhi,
    const float4* __restrict__ xlo, const float4* __restrict__ nhi, const float4* __restrict__ nlo,
    const double2* __restrict__ sigma, int R, int r0, double k, double eta, double2* __restrict__ out,
    long long split_stride, int out_ld, int out_r0) {
  __shared__ float4 sph[CHUNK], spl[CHUNK];  // y~_s (hi / lo), .w = dc.y~_s (hi / lo)
  __shared__ float4 snh[CHUNK], snl[CHUNK];  // n_s (hi / lo), .w = n_s.dc (hi / lo)
  __shared__ float4 ssg[CHUNK][RC];          // sigma: re hi, re lo, im hi, im lo
  __shared__ float4 tab[256];
  __shared__ qd4 bdd[BODY_BATCH];      // per source body: dc (x, y, z), rho0
  __shared__ double2 bcs[BODY_BATCH];  // cos k rho0, sin k rho0

  ff_phase_table_fill(tab);
  const TargetTile tile = tiles[blockIdx.x];
  const SourceSplit split = splits[blockIdx.y];
  const int tid = threadIdx.x;
  const bool active = tid < tile.count;
  const long long t = tile.start + (active ? tid : 0);
  const float4 th = xhi[t], tl = xlo[t];
  const ff xtx{th.x, tl.x}, xty{th.y, tl.y}, xtz{th.z, tl.z};
  const qd4 ca = centers[tile.body];
  const ff kf = ff_from_double(k);
  const ff etaf = ff_from_double(eta);

  double2 tot[RC];
#pragma unroll
  for (int r = 0; r < RC; ++r) tot[r] = make_double2(0.0, 0.0);

  for (int bb = split.begin; bb < split.end; bb += BODY_BATCH) {
    // body-pair constants once per CTA (the tile's targets share one body)
    __syncthreads();
    if (tid < BODY_BATCH && bb + tid < split.end) {
      const qd4 cb = centers[bb + tid];
      const double dcx = ca.x - cb.x, dcy = ca.y - cb.y, dcz = ca.z - cb.z;
      const double rho0 = sqrt(dcx * dcx + dcy * dcy + dcz * dcz);
      double s0d, c0d;
      sincos(k * rho0, &s0d, &c0d);
      qd4 v;
      v.x = dcx;
      v.y = dcy;
      v.z = dcz;
      v.w = rho0;
      bdd[tid] = v;
      bcs[tid] = make_double2(c0d, s0d);
    }
    __syncthreads();
  for (int b = bb; b < min(split.end, bb + BODY_BATCH); ++b) {
    if (b == tile.body) continue;
    const qd4 dv = bdd[b - bb];
    const double dcx = dv.x, dcy = dv.y, dcz = dv.z, rho0 = dv.w;
    const double c0d = bcs[b - bb].x, s0d = bcs[b - bb].y;
    const ff r0f = ff_from_double(rho0);
    const ff r02 = ff_from_double(rho0 * rho0);
    const ff At = ff_from_double(dcx * ((double)th.x + tl.x) + dcy * ((double)th.y + tl.y) +
                                 dcz * ((double)th.z + tl.z));

    double2 bacc[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) bacc[r] = make_double2(0.0, 0.0);

    const long long send = boff[b + 1];
    for (long long s0 = boff[b]; s0 < send; s0 += CHUNK) {
      __syncthreads();
      const long long i = s0 + tid;
      if (i < send) {
        const float4 ph = xhi[i], pl = xlo[i], qh = nhi[i], ql = nlo[i];
        const double yx = (double)ph.x + pl.x, yy = (double)ph.y + pl.y, yz = (double)ph.z + pl.z;
        const double nx = (double)qh.x + ql.x, ny = (double)qh.y + ql.y, nz = (double)qh.z + ql.z;
        const ff bs = ff_from_double(dcx * yx + dcy * yy + dcz * yz);
        const ff ns = ff_from_double(nx * dcx + ny * dcy + nz * dcz);
        sph[tid] = make_float4(ph.x, ph.y, ph.z, bs.hi);
        spl[tid] = make_float4(pl.x, pl.y, pl.z, bs.lo);
        snh[tid] = make_float4(qh.x, qh.y, qh.z, ns.hi);
        snl[tid] = make_float4(ql.x, ql.y, ql.z, ns.lo);
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          const double2 v = sigma[i * R + r0 + r];
          const ff re = ff_from_double(v.x), im = ff_from_double(v.y);
          ssg[tid][r] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
      }
      __syncthreads();
      const int cnt = (int)min((long long)CHUNK, send - s0);
      ff ar[RC], ai[RC];
#pragma unroll
      for (int r = 0; r < RC; ++r) ar[r] = ai[r] = ff{0.0f, 0.0f};
      for (int j = 0; j < cnt; ++j) {
        const float4 ph = sph[j], pl = spl[j], qh = snh[j], ql = snl[j];
        const ff dx = ff_sub(xtx, ff{ph.x, pl.x});
        const ff dy = ff_sub(xty, ff{ph.y, pl.y});
        const ff dz = ff_sub(xtz, ff{ph.z, pl.z});
        const ff dd = ff_add(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
        const ff e = ff_add(ff_mul_f(ff_sub(At, ff{ph.w, pl.w}), 2.0f), dd);
        const ff rho = ff_sqrt(ff_add(r02, e));
        const ff rinv = ff_rcp(rho);
        const ff delta = ff_div(e, ff_add(rho, r0f));
        ff sn, cs;
        ff_sincos(ff_mul(kf, delta), tab, &sn, &cs);
        // n_s.(y_s - x_t) = -(n_s.dc + n_s.d)
        const ff nd = ff_add(ff_add(ff_mul(ff{qh.x, ql.x}, dx), ff_mul(ff{qh.y, ql.y}, dy)),
                             ff_add(ff_mul(ff{qh.z, ql.z}, dz), ff{qh.w, ql.w}));
        const ff rinv2 = ff_mul(rinv, rinv);
        const ff are = ff_mul(nd, rinv2);                                  // -nyx / rho^2 with nyx = -nd
        const ff aim = ff_sub(ff_mul(ff_mul(kf, ff_neg(nd)), rinv), etaf);  // k nyx / rho - eta
        const ff kre = ff_mul(ff_sub(ff_mul(cs, are), ff_mul(sn, aim)), rinv);
        const ff kim = ff_mul(ff_add(ff_mul(sn, are), ff_mul(cs, aim)), rinv);
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          const float4 sg = ssg[j][r];
          const ff sre{sg.x, sg.y}, sim{sg.z, sg.w};
          ar[r] = ff_add(ar[r], ff_sub(ff_mul(kre, sre), ff_mul(kim, sim)));
          ai[r] = ff_add(ai[r], ff_add(ff_mul(kre, sim), ff_mul(kim, sre)));
        }
      }
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        bacc[r].x += ff_to_double(ar[r]);
        bacc[r].y += ff_to_double(ai[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      tot[r].x += c0d * bacc[r].x - s0d * bacc[r].y;
      tot[r].y += c0d * bacc[r].y + s0d * bacc[r].x;
    }
  }
  }
  if (active) {
    const double inv4pi = 0.079577471545947667884;
    double2* o = out + split_stride * blockIdx.y + t * out_ld + out_r0;
#pragma unroll
    for (int r = 0; r < RC; ++r) o[r] = make_double2(tot[r].x * inv4pi, tot[r].y * inv4pi);
  }
}

// y[t][r0 + r] = sum over splits of part[split][t][r], r < rc (fixed order)
template <typename C>
__global__ void reduce_splits_kernel(const C* __restrict__ part, int S, long long N, int rc, C* __restrict__ y,
                                     int R, int r0) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N * rc) return;
  const long long t = idx / rc;
  const int r = (int)(idx % rc);
  C s = part[idx];
  for (int q = 1; q < S; ++q) {
    const C v = part[q * N * rc + idx];
    s.x += v.x;
    s.y += v.y;
  }
  y[t * R + r0 + r] = s;
}

int pick_rc(int left) {
  if (left >= 16) return 16;
  if (left >= 8) return 8;
  if (left >= 4) return 4;
  if (left >= 2) return 2;
  return 1;
}

template <int RC>
void launch_f32(qams_ctx* c, dim3 grid, const float2* sigma, int R, int r0, float2* out, long long stride,
                int ld, int or0, cudaStream_t st) {
  if (c->ps_tt == 2) {
    grid.x = (unsigned)c->tiles2.size();
    pairsum_f32_kernel<RC, 2><<<grid, TILE, 0, st>>>(
        (const TargetTile*)c->d_tiles2.p, (const SourceSplit*)c->d_splits.p, (const long long*)c->boff.p,
        (const qd4*)c->centers.p, (const float4*)c->x32.p, (const float4*)c->n32.p, sigma, R, r0, c->k,
        c->eta, out, stride, ld, or0);
  } else {
    pairsum_f32_kernel<RC, 1><<<grid, TILE, 0, st>>>(
        (const TargetTile*)c->d_tiles.p, (const SourceSplit*)c->d_splits.p, (const long long*)c->boff.p,
        (const qd4*)c->centers.p, (const float4*)c->x32.p, (const float4*)c->n32.p, sigma, R, r0, c->k,
        c->eta, out, stride, ld, or0);
  }
  qams_count_launch();
}

template <int RC>
void launch_f64(qams_ctx* c, dim3 grid, const double2* sigma, int R, int r0, double2* out, long long stride,
                int ld, int or0, cudaStream_t st) {
  pairsum_f64_kernel<RC><<<grid, TILE, 0, st>>>(
      (const TargetTile*)c->d_tiles.p, (const SourceSplit*)c->d_splits.p, (const long long*)c->boff.p,
      (const qd4*)c->x64.p, (const qd4*)c->n64.p, sigma, R, r0, c->k, c->eta, out, stride, ld, or0); qams_count_launch();
}

template <int RC>
void launch_ff(qams_ctx* c, dim3 grid, const double2* sigma, int R, int r0, double2* out, long long stride,
               int ld, int or0, cudaStream_t st) {
  pairsum_ff_kernel<RC><<<grid, TILE, 0, st>>>(
      (const TargetTile*)c->d_tiles.p, (const SourceSplit*)c->d_splits.p, (const long long*)c->boff.p,
      (const qd4*)c->centers.p, (const float4*)c->x32.p, (const float4*)c->x32lo.p, (const float4*)c->n32.p,
      (const float4*)c->n32lo.p, sigma, R, r0, c->k, c->eta, out, stride, ld, or0); qams_count_launch();
}

}  // namespace

// Build target tiles and source splits for the current bodies.
int qams_pairsum_prepare(qams_ctx* c) {
  c->tiles.clear();
  for (int b = 0; b < (int)c->bodies.size(); ++b) {
    const BodyHost& bh = c->bodies[b];
    for (int s = 0; s < bh.n; s += TILE) c->tiles.push_back({b, std::min(TILE, bh.n - s), bh.offset + s});
  }
  // tiles of two targets per thread (2 TILE nodes of one body)
  c->tiles2.clear();
  for (int b = 0; b < (int)c->bodies.size(); ++b) {
    const BodyHost& bh = c->bodies[b];
    for (int s = 0; s < bh.n; s += 2 * TILE) c->tiles2.push_back({b, std::min(2 * TILE, bh.n - s), bh.offset + s});
  }
  qams_dev_free(c, &c->d_tiles);
  qams_dev_free(c, &c->d_tiles2);
  int rc = qams_dev_alloc(c, &c->d_tiles, sizeof(TargetTile) * c->tiles.size());
  if (rc) return rc;
  if ((rc = qams_dev_alloc(c, &c->d_tiles2, sizeof(TargetTile) * c->tiles2.size()))) return rc;
  QAMS_CUDA(cudaMemcpy(c->d_tiles.p, c->tiles.data(), sizeof(TargetTile) * c->tiles.size(),
                       cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->d_tiles2.p, c->tiles2.data(), sizeof(TargetTile) * c->tiles2.size(),
                       cudaMemcpyHostToDevice));
  return qams_pairsum_set_splits(c, qams_pairsum_default_splits(c, 8));
}

// Source splits for about mult x SMs CTAs (at least 1, at most one per body).
int qams_pairsum_default_splits(const qams_ctx* c, int mult) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const long long want = (long long)mult * sms;
  const long long nt = std::max<long long>(1, (long long)c->tiles.size());
  return (int)std::max(1LL, std::min<long long>((long long)c->bodies.size(), (want + nt - 1) / nt));
}

// S contiguous source-body ranges of about N/S nodes each, and the partial-sum
// buffer they need (S > 1).  Blocking.
int qams_pairsum_set_splits(qams_ctx* c, int S) {
  const int nb = (int)c->bodies.size();
  S = std::max(1, std::min(S, nb));
  c->splits.clear();
  long long per = (c->N + S - 1) / S, acc = 0;
  int begin = 0;
  for (int b = 0; b < nb; ++b) {
    acc += c->bodies[b].n;
    if (acc >= per * ((long long)c->splits.size() + 1) || b == nb - 1) {
      c->splits.push_back({begin, b + 1});
      begin = b + 1;
    }
  }
  qams_dev_free(c, &c->d_splits);
  int rc = qams_dev_alloc(c, &c->d_splits, sizeof(SourceSplit) * c->splits.size());
  if (rc) return rc;
  QAMS_CUDA(cudaMemcpy(c->d_splits.p, c->splits.data(), sizeof(SourceSplit) * c->splits.size(),
                       cudaMemcpyHostToDevice));
  const size_t need = c->splits.size() > 1 ? sizeof(double2) * 16 * (size_t)c->N * c->splits.size() : 0;
  if (c->partial.bytes < need || (need == 0 && c->partial.p)) {
    qams_dev_free(c, &c->partial);
    if (need && (rc = qams_dev_alloc(c, &c->partial, need))) return rc;
  }
  return QAMS_OK;
}

int qams_pairsum_launch(qams_ctx* c, int R, const void* sigma, void* y, int precision, cudaStream_t st) {
  if (c->lat.on && c->lat.use && c->lat.ready) return qams_lattice_pairsum(c, R, sigma, y, precision, st);
  const int S = (int)c->splits.size();
  dim3 grid((unsigned)c->tiles.size(), (unsigned)S);
  if (precision == QAMS_PREC_FP32 && R >= c->tc_pair_min_r && R <= 16) {
    // multiply-accumulate on the tensor cores, all right-hand sides in one launch
    float2* out = S > 1 ? (float2*)c->partial.p : (float2*)y;
    cudaEvent_t pe = qams_prof_begin(c, QAMS_PROF_PAIRSUM_TC, st);
    int rc = qams_pairsum_tc_launch(c, R, sigma, out, S > 1 ? c->N * R : 0, R, st);
    qams_prof_end(c, QAMS_PROF_PAIRSUM_TC, st, pe);
    if (rc) return rc;
    if (S > 1) {
      const long long n = c->N * R;
      reduce_splits_kernel<float2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float2*)c->partial.p, S, c->N,
                                                                              R, (float2*)y, R, 0);
      qams_count_launch();
      QAMS_CUDA(cudaGetLastError());
    }
    return QAMS_OK;
  }
  for (int r0 = 0; r0 < R;) {
    const int rc = pick_rc(R - r0);
    if (precision == QAMS_PREC_FP32) {
      float2* out = S > 1 ? (float2*)c->partial.p : (float2*)y;
      const long long stride = S > 1 ? c->N * rc : 0;
      const int ld = S > 1 ? rc : R, or0 = S > 1 ? 0 : r0;
      const float2* sg = (const float2*)sigma;
      cudaEvent_t pe = qams_prof_begin(c, QAMS_PROF_PAIRSUM_FP32, st);
      switch (rc) {
        case 16: launch_f32<16>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
        case 8: launch_f32<8>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
        case 4: launch_f32<4>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
        case 2: launch_f32<2>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
        default: launch_f32<1>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
      }
      qams_prof_end(c, QAMS_PROF_PAIRSUM_FP32, st, pe);
      QAMS_CUDA(cudaGetLastError());
      if (S > 1) {
        const long long n = c->N * rc;
        reduce_splits_kernel<float2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            (const float2*)c->partial.p, S, c->N, rc, (float2*)y, R, r0); qams_count_launch();
        QAMS_CUDA(cudaGetLastError());
      }
    } else {
      double2* out = S > 1 ? (double2*)c->partial.p : (double2*)y;
      const long long stride = S > 1 ? c->N * rc : 0;
      const int ld = S > 1 ? rc : R, or0 = S > 1 ? 0 : r0;
      const double2* sg = (const double2*)sigma;
      const int slot = precision == QAMS_PREC_FF ? QAMS_PROF_PAIRSUM_FF : QAMS_PROF_PAIRSUM_FP64;
      cudaEvent_t pe = qams_prof_begin(c, slot, st);
      if (precision == QAMS_PREC_FF) {
        switch (rc) {
          case 16: launch_ff<16>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
          case 8: launch_ff<8>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
          case 4: launch_ff<4>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
          case 2: launch_ff<2>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
          default: launch_ff<1>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
        }
      } else {
        switch (rc) {
          case 16: launch_f64<16>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
          case 8: launch_f64<8>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
          case 4: launch_f64<4>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
          case 2: launch_f64<2>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
          default: launch_f64<1>(c, grid, sg, R, r0, out, stride, ld, or0, st); break;
        }
      }
      qams_prof_end(c, slot, st, pe);
      QAMS_CUDA(cudaGetLastError());
      if (S > 1) {
        const long long n = c->N * rc;
        reduce_splits_kernel<double2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            (const double2*)c->partial.p, S, c->N, rc, (double2*)y, R, r0); qams_count_launch();
        QAMS_CUDA(cudaGetLastError());
      }
    }
    r0 += rc;
  }
  return QAMS_OK;
}

// ---------------------------------------------------------------------------
// Pair sum without device allocation.
//
// For callers that cannot call cudaMalloc -- for example a host framework
// that reserves all device memory for its own pool up front, or a
// latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronisation -- this variant takes every input and output from the
// caller and keeps its own scratch (launch tables and the per-split partial
// sums) in the file-scope array below, which every GPU that loads the
// library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t STATIC_SCRATCH_BYTES = 32u << 20;  // 32 MiB
constexpr int STATIC_MAX_BODIES = 4096;
constexpr int STATIC_MAX_TILES = 65536;
constexpr int STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch per device (host code cannot use the
// symbol's name as a device pointer); looked up once, on the first call on a
// device.  A cudaDeviceReset ends the context the address belongs to, so
// this entry point must not be used again in a process that reset the device.
static void* g_static_ptr[STATIC_MAX_DEVICES];

}  // namespace

extern "C" int qams_pairsum_f32_static(int n_bodies, const long long* body_offsets_host, const double* centers_host,
                                       const void* x32_dev, const void* n32_dev, int R, const void* sigma_dev,
                                       void* y_dev, double k, double eta, void* stream) {
  if (n_bodies < 1 || !body_offsets_host || !centers_host || !x32_dev || !n32_dev || R < 1 || !sigma_dev ||
      !y_dev || !(k > 0) || !std::isfinite(k) || !std::isfinite(eta))
    return QAMS_EINVAL;
  if (n_bodies > STATIC_MAX_BODIES) return QAMS_ESCRATCH;
  const long long N = body_offsets_host[n_bodies];
  if (body_offsets_host[0] != 0 || N < 1) return QAMS_EINVAL;
  for (int b = 0; b < n_bodies; ++b)
    if (body_offsets_host[b + 1] <= body_offsets_host[b]) return QAMS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // the call waits for its own copies before returning; on a stream that is
  // being captured that wait would invalidate the caller's capture
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  QAMS_CUDA(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) return QAMS_EINVAL;
  int dev = 0;
  QAMS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= STATIC_MAX_DEVICES) return QAMS_ESCRATCH;
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    QAMS_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_ptr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_static_ptr[dev];

  // launch tables, built like qams_pairsum_prepare's (host memory only)
  std::vector<TargetTile> tiles;
  for (int b = 0; b < n_bodies; ++b) {
    const long long o = body_offsets_host[b], n = body_offsets_host[b + 1] - o;
    for (long long s = 0; s < n; s += TILE) tiles.push_back({b, (int)std::min<long long>(TILE, n - s), o + s});
  }
  if ((long long)tiles.size() > STATIC_MAX_TILES) return QAMS_ESCRATCH;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) & ~(size_t)255;
    return base + at;
  };
  long long* d_boff = (long long*)carve(sizeof(long long) * (n_bodies + 1));
  qd4* d_cent = (qd4*)carve(sizeof(qd4) * n_bodies);
  TargetTile* d_tiles = (TargetTile*)carve(sizeof(TargetTile) * tiles.size());
  SourceSplit* d_splits = (SourceSplit*)carve(sizeof(SourceSplit) * n_bodies);
  const size_t fixed = off;
  if (fixed >= STATIC_SCRATCH_BYTES) return QAMS_ESCRATCH;
  const size_t room = STATIC_SCRATCH_BYTES - fixed;

  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rc_max = pick_rc(R);
  long long want = std::max(1LL, std::min<long long>(n_bodies, (8LL * sms + (long long)tiles.size() - 1) /
                                                                   (long long)tiles.size()));
  // partial sums must fit in the remaining scratch
  const long long fit = (long long)(room / (sizeof(float2) * (size_t)N * rc_max));
  const int S = (int)std::max(1LL, std::min(want, fit));
  std::vector<SourceSplit> splits;
  const long long per = (N + S - 1) / S;
  long long acc = 0;
  int begin = 0;
  for (int b = 0; b < n_bodies; ++b) {
    acc += body_offsets_host[b + 1] - body_offsets_host[b];
    if (acc >= per * ((long long)splits.size() + 1) || b == n_bodies - 1) {
      splits.push_back({begin, b + 1});
      begin = b + 1;
    }
  }
  const int Sr = (int)splits.size();
  float2* d_part = (float2*)carve(0);
  std::vector<qd4> cent(n_bodies);
  for (int b = 0; b < n_bodies; ++b) {
    cent[b].x = centers_host[3 * b];
    cent[b].y = centers_host[3 * b + 1];
    cent[b].z = centers_host[3 * b + 2];
    cent[b].w = 0.0;
  }
  // every table entry and every partial sum is written before it is read,
  // so nothing left in the array by an earlier call needs clearing
  QAMS_CUDA(cudaMemcpyAsync(d_boff, body_offsets_host, sizeof(long long) * (n_bodies + 1), cudaMemcpyHostToDevice, st));
  QAMS_CUDA(cudaMemcpyAsync(d_cent, cent.data(), sizeof(qd4) * n_bodies, cudaMemcpyHostToDevice, st));
  QAMS_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TargetTile) * tiles.size(), cudaMemcpyHostToDevice, st));
  QAMS_CUDA(cudaMemcpyAsync(d_splits, splits.data(), sizeof(SourceSplit) * Sr, cudaMemcpyHostToDevice, st));

  dim3 grid((unsigned)tiles.size(), (unsigned)Sr);
  for (int r0 = 0; r0 < R;) {
    const int rcur = pick_rc(R - r0);
    float2* out = Sr > 1 ? d_part : (float2*)y_dev;
    const long long stride = Sr > 1 ? N * rcur : 0;
    const int ld = Sr > 1 ? rcur : R, or0 = Sr > 1 ? 0 : r0;
    const float2* sg = (const float2*)sigma_dev;
#define QAMS_STATIC_LAUNCH(RCV)                                                                                  \
  pairsum_f32_kernel<RCV, 1><<<grid, TILE, 0, st>>>(d_tiles, d_splits, d_boff, d_cent, (const float4*)x32_dev, \
                                                 (const float4*)n32_dev, sg, R, r0, k, eta, out, stride, ld, or0)
    switch (rcur) {
      case 16: QAMS_STATIC_LAUNCH(16); break;
      case 8: QAMS_STATIC_LAUNCH(8); break;
      case 4: QAMS_STATIC_LAUNCH(4); break;
      case 2: QAMS_STATIC_LAUNCH(2); break;
      default: QAMS_STATIC_LAUNCH(1); break;
    }
#undef QAMS_STATIC_LAUNCH
    qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
    if (Sr > 1) {
      const long long n = N * rcur;
      reduce_splits_kernel<float2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_part, Sr, N, rcur, (float2*)y_dev,
                                                                                R, r0);
      qams_count_launch();
      QAMS_CUDA(cudaGetLastError());
    }
    r0 += rcur;
  }
  // the host tables above are read by the copies: finish them before returning
  QAMS_CUDA(cudaStreamSynchronize(st));
  return QAMS_OK;
}
