// Near-field correction of the field at off-surface points (Sec. 6, the
// point-source check of Eq. artificial point source solution).  The smooth
// rule loses accuracy for points within a few node spacings of a surface
// (the integrand's nearest singularity comes within the reach of the
// nodes).  For such a point x and body b the body's contribution is
// replaced by the product-integration rule of the self blocks, taken at an
// off-surface target: x = y(s*, theta*) + v with (s*, theta*) the nearest
// surface point, the azimuthal integrals by the modal Green's functions of
// the source rings seen from x, the outer integral graded toward s*.  The
// self-block kernel returns, per (x, b), the row of those weights minus the
// smooth rule's on the near panels; this file finds the pairs and adds
//   u(x) += sum_col row[col] mu[col].
#include <algorithm>
#include <cmath>
#include <vector>

#include "qams_internal.h"

namespace {

constexpr int MAXR = 16;

// one warp per corrected point: its (point, body) pairs T[beg[k]..beg[k+1]) in
// order, u[m][r0 + r] += sum over the pairs of row . mu_b[:, r0 + r]
// (one writer per point: the sum does not depend on scheduling)
__global__ void near_apply_kernel(const NearTarget* __restrict__ T, const int* __restrict__ beg, int npts,
                                  const double2* __restrict__ rows, const double2* __restrict__ mu, int R, int r0,
                                  int rc, double2* u) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= npts) return;
  double ar[MAXR], ai[MAXR];
  for (int r = 0; r < rc; ++r) ar[r] = ai[r] = 0.0;
  int m = 0;
  for (int k = beg[w]; k < beg[w + 1]; ++k) {
    const NearTarget t = T[k];
    m = t.m;
    const double2* row = rows + t.row;
    for (int col = lane; col < t.n; col += 32) {
      const double2 a = row[col];
      const double2* mv = mu + (t.node0 + col) * R + r0;
      for (int r = 0; r < rc; ++r) {
        const double2 v = mv[r];
        ar[r] += a.x * v.x - a.y * v.y;
        ai[r] += a.x * v.y + a.y * v.x;
      }
    }
  }
  for (int r = 0; r < rc; ++r) {
    for (int o = 16; o > 0; o >>= 1) {
      ar[r] += __shfl_xor_sync(0xffffffffu, ar[r], o);
      ai[r] += __shfl_xor_sync(0xffffffffu, ai[r], o);
    }
    if (lane == 0) {
      double2* dst = u + (long long)m * R + r0 + r;
      dst->x += ar[r];
      dst->y += ai[r];
    }
  }
}

// largest distance between neighbouring nodes (along theta and along s within a
// panel) of body b: the length scale of its smooth rule
double node_spacing(const qams_ctx* c, const BodyHost& b) {
  const double* x = c->hx.data() + 3 * b.offset;
  const int nth = b.d.n_theta, order = b.d.order;
  double h2 = 0.0;
  auto d2 = [&](long long i, long long j) {
    const double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
    return dx * dx + dy * dy + dz * dz;
  };
  for (int p = 0; p < b.d.n_panels; ++p)
    for (int l = 0; l < order; ++l)
      for (int j = 0; j < nth; ++j) {
        const long long t = ((long long)p * order + l) * nth + j;
        h2 = std::max(h2, d2(t, ((long long)p * order + l) * nth + (j + 1) % nth));
        if (l + 1 < order) h2 = std::max(h2, d2(t, t + nth));
      }
  return std::sqrt(h2);
}

}  // namespace

int qams_near_correction(qams_ctx* c, int R, const void* mu, int M, const double* pts, void* u, cudaStream_t st) {
  c->near_pairs = 0;
  if (c->near_factor <= 0) return QAMS_OK;
  const int nb = (int)c->bodies.size();
  // node spacing per class of congruent bodies
  std::vector<double> hcls(c->class_rep.size());
  for (size_t k = 0; k < c->class_rep.size(); ++k) hcls[k] = node_spacing(c, c->bodies[c->class_rep[k]]);
  std::vector<NearTarget> tg;
  double r_extra = 0.0;
  long long entries = 0;
  for (int m = 0; m < M; ++m) {
    const double* x = pts + 3 * m;
    for (int b = 0; b < nb; ++b) {
      const BodyHost& B = c->bodies[b];
      const double dnear = c->near_factor * hcls[c->body_class[b]];
      const double dx = x[0] - B.d.center[0], dy = x[1] - B.d.center[1], dz = x[2] - B.d.center[2];
      if (dx * dx + dy * dy + dz * dz > (B.radius + dnear) * (B.radius + dnear)) continue;
      NearTarget t{};
      double dist;
      qams_nearest_point(B, c->hx.data() + 3 * B.offset, x, &t.s, &t.th, &t.panel, &dist, &t.ds, t.v);
      if (!(dist < dnear)) continue;
      t.cls = c->body_class[b];
      for (int q = 0; q < 3; ++q) t.x[q] = x[q];
      t.node0 = B.offset;
      t.row = entries;
      t.m = m;
      t.n = B.n;
      entries += B.n;
      r_extra = std::max(r_extra, dist);
      tg.push_back(t);
    }
  }
  c->near_pairs = (long long)tg.size();
  if (tg.empty()) return QAMS_OK;
  // rows in chunks of at most ~1 GB
  const long long cap = std::max<long long>(1LL << 26, tg.front().n);
  int rc = QAMS_OK;
  for (size_t i0 = 0; i0 < tg.size() && !rc;) {
    // a chunk ends on a point boundary (pairs are generated point by point)
    size_t i1 = i0;
    const long long base = tg[i0].row;
    while (i1 < tg.size() && tg[i1].row + tg[i1].n - base <= cap) ++i1;
    if (i1 == i0) i1 = i0 + 1;
    while (i1 < tg.size() && i1 > i0 + 1 && tg[i1].m == tg[i1 - 1].m) --i1;
    while (i1 < tg.size() && tg[i1].m == tg[i1 - 1].m) ++i1;
    std::vector<NearTarget> part(tg.begin() + i0, tg.begin() + i1);
    std::vector<int> beg{0};
    for (size_t k = 1; k < part.size(); ++k)
      if (part[k].m != part[k - 1].m) beg.push_back((int)k);
    beg.push_back((int)part.size());
    const int npts = (int)beg.size() - 1;
    for (NearTarget& t : part) t.row -= base;
    const long long ent = part.back().row + part.back().n;
    DeviceBuf d_t, d_rows, d_beg;
    rc = qams_dev_alloc(c, &d_t, sizeof(NearTarget) * part.size());
    if (!rc) rc = qams_dev_alloc(c, &d_beg, sizeof(int) * beg.size());
    if (!rc) rc = qams_dev_alloc(c, &d_rows, sizeof(double2) * (size_t)ent);
    if (!rc && (cudaMemcpyAsync(d_t.p, part.data(), sizeof(NearTarget) * part.size(), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(d_beg.p, beg.data(), sizeof(int) * beg.size(), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess))
      rc = QAMS_ECUDA;
    if (!rc) rc = qams_near_rows_launch(c, (const NearTarget*)d_t.p, (long long)part.size(), r_extra,
                                        (double2*)d_rows.p, st);
    if (!rc) {
      const long long threads = (long long)npts * 32;
      for (int r0 = 0; r0 < R; r0 += MAXR) {
        const int cnt = std::min(MAXR, R - r0);
        near_apply_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
            (const NearTarget*)d_t.p, (const int*)d_beg.p, npts, (const double2*)d_rows.p, (const double2*)mu, R, r0,
            cnt, (double2*)u);
        qams_count_launch();
      }
      if (cudaGetLastError() != cudaSuccess) rc = QAMS_ECUDA;
      if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = QAMS_ECUDA;
    }
    qams_dev_free(c, &d_t);
    qams_dev_free(c, &d_beg);
    qams_dev_free(c, &d_rows);
    i0 = i1;
  }
  return rc;
}
