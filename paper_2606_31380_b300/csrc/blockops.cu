// Self-block products and the full operator apply (Eq. linearsys):
//   y = blockdiag(A_b) x + sum_{b' != b} D_{b,b'} (w x),
// the diagonal blocks from the assembled self blocks (HBM-streaming,
// one warp per row) and the off-diagonal part from the pair sum.
#include <algorithm>

#include "qams_internal.h"

namespace {

__global__ void to_fp32_kernel(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

template <typename T2>
struct Acc;
template <>
struct Acc<double2> {
  using R = double;
};
template <>
struct Acc<float2> {
  using R = float;
};

// One warp per row g: y[g][r0+r] (+)= sum_col A_b[t][col] x[off+col][r0+r],
// U block entries in flight per lane (the row streams from HBM; x is re-read
// from L1/L2 by every row of the body).
template <typename T2, int RC>
__global__ void block_apply_kernel(const T2* __restrict__ blocks, const long long* __restrict__ blk_off,
                                   const long long* __restrict__ boff, int nb, long long N,
                                   const T2* __restrict__ x, T2* __restrict__ y, int R, int r0, int accumulate) {
  using F = typename Acc<T2>::R;
  constexpr int U = RC >= 8 ? 2 : 4;
  const long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= N) return;
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (boff[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const long long off = boff[lo];
  const int n = (int)(boff[lo + 1] - off);
  const T2* row = blocks + blk_off[lo] + (g - off) * n;
  F ar[RC], ai[RC];
#pragma unroll
  for (int r = 0; r < RC; ++r) ar[r] = ai[r] = F(0);
  for (int c0 = lane; c0 < n; c0 += 32 * U) {
    T2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c0 + 32 * u < n) {
        v[u] = row[c0 + 32 * u];
      } else {
        v[u].x = F(0);
        v[u].y = F(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int col = c0 + 32 * u;
      if (col >= n) break;
      const T2* xv = x + (off + col) * R + r0;
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        const T2 w = xv[r];
        ar[r] += v[u].x * w.x - v[u].y * w.y;
        ai[r] += v[u].x * w.y + v[u].y * w.x;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    for (int o = 16; o > 0; o >>= 1) {
      ar[r] += __shfl_xor_sync(0xffffffffu, ar[r], o);
      ai[r] += __shfl_xor_sync(0xffffffffu, ai[r], o);
    }
  }
  if (lane == 0) {
    T2* yv = y + g * R + r0;
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      T2 v;
      v.x = ar[r];
      v.y = ai[r];
      if (accumulate) {
        v.x += yv[r].x;
        v.y += yv[r].y;
      }
      yv[r] = v;
    }
  }
}

// sigma = w x (quadrature weights folded into the density)
template <typename T2, typename P4>
__global__ void weight_kernel(const P4* __restrict__ xw, const T2* __restrict__ x, T2* __restrict__ s, long long N,
                              int R) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N * R) return;
  const auto w = xw[i / R].w;
  T2 v = x[i];
  v.x *= w;
  v.y *= w;
  s[i] = v;
}

template <typename T2, int RC>
void launch_block(qams_ctx* c, const void* blocks, const void* x, void* y, int R, int r0, int acc, cudaStream_t st) {
  const long long threads = c->N * 32;
  block_apply_kernel<T2, RC><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      (const T2*)blocks, (const long long*)c->blk_off.p, (const long long*)c->boff.p, (int)c->bodies.size(), c->N,
      (const T2*)x, (T2*)y, R, r0, acc); qams_count_launch();
}

template <typename T2>
void block_dispatch(qams_ctx* c, const void* blocks, const void* x, void* y, int R, int acc, cudaStream_t st) {
  const int slot = sizeof(T2) == sizeof(double2) ? QAMS_PROF_BLOCK_FP64 : QAMS_PROF_BLOCK_FP32;
  cudaEvent_t pe = qams_prof_begin(c, slot, st);
  for (int r0 = 0; r0 < R;) {
    const int left = R - r0;
    int rc = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    switch (rc) {
      case 16: launch_block<T2, 16>(c, blocks, x, y, R, r0, acc, st); break;
      case 8: launch_block<T2, 8>(c, blocks, x, y, R, r0, acc, st); break;
      case 4: launch_block<T2, 4>(c, blocks, x, y, R, r0, acc, st); break;
      case 2: launch_block<T2, 2>(c, blocks, x, y, R, r0, acc, st); break;
      default: launch_block<T2, 1>(c, blocks, x, y, R, r0, acc, st); break;
    }
    r0 += rc;
  }
  qams_prof_end(c, slot, st, pe);
}

}  // namespace

int qams_blocks_to_fp32(qams_ctx* c, cudaStream_t st) {
  qams_dev_free(c, &c->blocks32);
  int rc = qams_dev_alloc(c, &c->blocks32, sizeof(float2) * (size_t)c->block_entries);
  if (rc) return rc;
  const long long n = c->block_entries;
  to_fp32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double2*)c->blocks64.p, (float2*)c->blocks32.p, n); qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  // split copies for the tensor-core product (the preconditioner's follow its build)
  c->tc_pinv_ok = false;
  if ((rc = qams_tc_groups(c))) return rc;
  return qams_tc_prepare(c, 0, st);
}

namespace {
// The tensor-core product when it applies (FP32, enough right-hand sides,
// split copy available); QAMS_EINVAL means "use the CUDA-core kernel".
int try_tc(qams_ctx* c, const void* blocks, int R, const void* x, void* y, bool accumulate, cudaStream_t st) {
  if (R < c->tc_min_r) return QAMS_EINVAL;
  const int which = blocks == c->blocks32.p ? 0 : blocks == c->pinv32.p ? 1 : -1;
  if (which < 0) return QAMS_EINVAL;
  return qams_tc_block_apply(c, which, R, x, y, accumulate, st);
}
}  // namespace

int qams_block_apply(qams_ctx* c, int R, const void* x, void* y, int precision, bool accumulate, cudaStream_t st) {
  if (precision == QAMS_PREC_FP64) {
    block_dispatch<double2>(c, c->blocks64.p, x, y, R, accumulate ? 1 : 0, st);
  } else {
    const int rc = try_tc(c, c->blocks32.p, R, x, y, accumulate, st);
    if (rc != QAMS_EINVAL) return rc;
    block_dispatch<float2>(c, c->blocks32.p, x, y, R, accumulate ? 1 : 0, st);
  }
  QAMS_CUDA(cudaGetLastError());
  return QAMS_OK;
}

int qams_block_apply_ptr(qams_ctx* c, const void* blocks, int R, const void* x, void* y, int precision,
                         bool accumulate, cudaStream_t st) {
  if (precision == QAMS_PREC_FP64) {
    block_dispatch<double2>(c, blocks, x, y, R, accumulate ? 1 : 0, st);
  } else {
    const int rc = try_tc(c, blocks, R, x, y, accumulate, st);
    if (rc != QAMS_EINVAL) return rc;
    block_dispatch<float2>(c, blocks, x, y, R, accumulate ? 1 : 0, st);
  }
  QAMS_CUDA(cudaGetLastError());
  return QAMS_OK;
}

int qams_apply_launch(qams_ctx* c, int R, const void* x, void* y, int precision, cudaStream_t st) {
  const size_t need = sizeof(double2) * (size_t)c->N * R;
  if (c->ws_sigma.bytes < need) {
    qams_dev_free(c, &c->ws_sigma);
    int rc = qams_dev_alloc(c, &c->ws_sigma, need);
    if (rc) return rc;
  }
  const long long n = c->N * R;
  if (precision != QAMS_PREC_FP32) {
    weight_kernel<double2, qd4><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const qd4*)c->x64.p, (const double2*)x, (double2*)c->ws_sigma.p, c->N, R);
  } else {
    weight_kernel<float2, float4><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const float4*)c->x32.p, (const float2*)x, (float2*)c->ws_sigma.p, c->N, R);
  }
  qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  int rc = qams_pairsum_launch(c, R, c->ws_sigma.p, y, precision, st);
  if (rc) return rc;
  return qams_block_apply(c, R, x, y, precision == QAMS_PREC_FF ? QAMS_PREC_FP64 : precision, true, st);
}
