// Launch-shape autotuner for the FP32 operator apply (no counterpart in the
// paper: it chooses between kernels that compute the same sums up to
// rounding).
//
// For R right-hand sides on a context's bodies it times, with CUDA events on
// the caller's stream (one warm-up and two timed launches each):
//   * the FP32 pair sum with its multiply-accumulate on the CUDA cores (one
//     or two targets per thread) or on the tensor cores (R <= 16), for every
//     distinct source-split count
//     S(m) = clamp(ceil(m SMs / target tiles), 1, bodies), m in {1,2,4,8,16};
//   * for R >= 8, the FP32 self-block product on the CUDA cores or on the
//     tensor cores (when the split copy exists).
// The fastest choice is kept in the context (split tables, thresholds) and
// in a process-wide cache keyed by (device, body sizes, R), so later
// contexts of the same shape reuse it without timing.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qams_internal.h"

namespace {

std::mutex g_tune_mu;
std::map<std::string, qams_tuning> g_tune_cache;

std::string key_of(const qams_ctx* c, int R) {
  std::string k = std::to_string(c->device) + "|" + std::to_string(R) + "|";
  // run-length list of body sizes (the kernels' cost depends on sizes, not shapes)
  int prev = -1, run = 0;
  for (const BodyHost& b : c->bodies) {
    if (b.n == prev) {
      ++run;
      continue;
    }
    if (run) k += std::to_string(prev) + "x" + std::to_string(run) + ",";
    prev = b.n;
    run = 1;
  }
  k += std::to_string(prev) + "x" + std::to_string(run);
  return k;
}

// deterministic test vector: components in (-1, 1) from an integer hash
__global__ void fill_kernel(float2* v, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned h = (unsigned)(i * 2654435761ull) ^ 0x9e3779b9u;
  h ^= h >> 15;
  h *= 0x2c1b3c6du;
  h ^= h >> 12;
  const float a = (float)(h & 0xffff) / 32768.f - 1.f, b = (float)(h >> 16) / 32768.f - 1.f;
  v[i] = make_float2(a, b);
}

int time_ms(cudaStream_t st, float* ms, int (*fn)(void*), void* arg) {
  int rc = fn(arg);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  QAMS_CUDA(cudaEventCreate(&e0));
  QAMS_CUDA(cudaEventCreate(&e1));
  QAMS_CUDA(cudaEventRecord(e0, st));
  for (int i = 0; i < 2 && !rc; ++i) rc = fn(arg);
  QAMS_CUDA(cudaEventRecord(e1, st));
  QAMS_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / 2;
  return rc;
}

struct Job {
  qams_ctx* c;
  int R;
  const void* x;
  void* y;
  cudaStream_t st;
};

int run_pair(void* p) {
  Job* j = (Job*)p;
  return qams_pairsum_launch(j->c, j->R, j->x, j->y, QAMS_PREC_FP32, j->st);
}

int run_block(void* p) {
  Job* j = (Job*)p;
  return qams_block_apply(j->c, j->R, j->x, j->y, QAMS_PREC_FP32, false, j->st);
}

void apply_tuning(qams_ctx* c, const qams_tuning& t) {
  c->tc_pair_min_r = t.pair_tc ? t.R : std::min(17, t.R + 1);
  c->ps_tt = t.pair_targets;
  if (t.block_tc >= 0) c->tc_min_r = t.block_tc ? t.R : std::min(17, t.R + 1);
}

}  // namespace

extern "C" int qams_autotune(qams_ctx* c, int R, qams_tuning* out, void* stream) {
  if (!c || R < 1 || R > 16 || c->bodies.empty() || !c->have_k) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const std::string key = key_of(c, R);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      qams_tuning t = it->second;
      int rc = qams_pairsum_set_splits(c, t.pair_splits);
      if (rc) return rc;
      apply_tuning(c, t);
      t.cached = 1;
      if (out) *out = t;
      return QAMS_OK;
    }
  }
  DeviceBuf x, y;
  int rc = qams_dev_alloc(c, &x, sizeof(float2) * (size_t)c->N * R);
  if (!rc) rc = qams_dev_alloc(c, &y, sizeof(float2) * (size_t)c->N * R);
  if (rc) {
    qams_dev_free(c, &x);
    qams_dev_free(c, &y);
    return rc;
  }
  const long long n = c->N * R;
  fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((float2*)x.p, n);
  qams_count_launch();
  qams_tuning best{};
  best.R = R;
  best.pair_ms = 1e30;
  best.block_tc = -1;
  Job job{c, R, x.p, y.p, st};
  std::vector<int> cands;
  for (int m : {1, 2, 4, 8, 16}) {
    const int S = qams_pairsum_default_splits(c, m);
    if (std::find(cands.begin(), cands.end(), S) == cands.end()) cands.push_back(S);
  }
  const int saved_pair = c->tc_pair_min_r, saved_blk = c->tc_min_r, saved_tt = c->ps_tt;
  for (int S : cands) {
    if ((rc = qams_pairsum_set_splits(c, S))) break;
    // variants: CUDA cores with 1 or 2 targets per thread, tensor cores
    for (int v = 0; v < 3 && !rc; ++v) {
      c->tc_pair_min_r = v == 2 ? 1 : 17;
      c->ps_tt = v == 1 ? 2 : 1;
      float ms = 0.f;
      rc = time_ms(st, &ms, run_pair, &job);
      if (!rc && ms < best.pair_ms) {
        best.pair_ms = ms;
        best.pair_tc = v == 2;
        best.pair_targets = v == 1 ? 2 : 1;
        best.pair_splits = S;
      }
    }
    if (rc) break;
  }
  // block products: below 8 right-hand sides they stream HBM on the CUDA cores
  // at a fraction of a percent of the apply, and the split-FP16 product's
  // ~22-bit accumulation costs the refinement an extra step, so the tensor
  // path is only considered from 8 up
  if (!rc && c->assembled && R >= 8) {
    float ms[2] = {0.f, 0.f};
    best.block_tc = 0;
    c->tc_min_r = 17;
    rc = time_ms(st, &ms[0], run_block, &job);
    best.block_ms = ms[0];
    if (!rc && c->tc_blk_ok) {
      c->tc_min_r = 1;
      rc = time_ms(st, &ms[1], run_block, &job);
      if (!rc && ms[1] < ms[0]) {
        best.block_tc = 1;
        best.block_ms = ms[1];
      }
    }
  }
  c->tc_pair_min_r = saved_pair;
  c->tc_min_r = saved_blk;
  c->ps_tt = saved_tt;
  if (!rc) rc = qams_tc_check(c, st);
  if (!rc) rc = qams_pairsum_set_splits(c, best.pair_splits);
  qams_dev_free(c, &x);
  qams_dev_free(c, &y);
  if (rc) return rc;
  apply_tuning(c, best);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  if (out) *out = best;
  return QAMS_OK;
}
