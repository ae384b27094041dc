// Block-Jacobi preconditioner (Sec. 6 solver description: GMRES with a
// block-diagonal preconditioner built from the factorisation of the self
// matrix): P_b = A_b^{-1} for every body, in complex64, by blocked
// Gauss-Jordan elimination on the body's self block.
//
// For block column k (width b <= 64) of W (n x n, row-major, W = A_b on entry):
//   P = W_kk^{-1}                       (own kernel, partial pivoting inside the block)
//   R = P W_k,:                         (GEMM)
//   C = W_:,k                           (copy)
//   W -= C R                            (GEMM, rank-b update of the whole matrix)
//   T = -C P                            (GEMM)
//   W_k,: = R,  W_:,k = T,  W_kk = P    (own kernel)
// after which W = A_b^{-1}.  The GEMMs are plain cuBLAS complex64 GEMMs,
// batched over bodies of equal size.  Pivoting is local to the diagonal
// blocks; the self blocks of the second-kind combined-field operator
// (1/2 I plus a smoothing part) keep them well conditioned, and a
// vanishing pivot is reported as QAMS_ENUMERIC.
#include <cublas_v2.h>

#include <algorithm>
#include <map>
#include <vector>

#include "qams_internal.h"

namespace {

constexpr int BW = 64;

// Inverse of the b x b diagonal block of every body (one CTA per body) by
// Gauss-Jordan on [W_kk | I] with partial pivoting; the inverse is written
// to P (b x b per body, row-major).
__global__ void __launch_bounds__(256) pivot_inverse_kernel(float2* const* __restrict__ W, int n, int k0, int b,
                                                            float2* __restrict__ P, int* __restrict__ status) {
  extern __shared__ float2 aug[];  // [b][2b]
  __shared__ float2 fcol[64];      // column c before its elimination
  __shared__ int piv;
  const float2* Wb = W[blockIdx.x];
  const int ld = 2 * b;
  for (int e = threadIdx.x; e < b * ld; e += blockDim.x) {
    const int r = e / ld, c = e % ld;
    aug[e] = c < b ? Wb[(long long)(k0 + r) * n + k0 + c] : make_float2(c - b == r ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int c = 0; c < b; ++c) {
    if (threadIdx.x < 32) {
      float best = -1.f;
      int bi = c;
      for (int r = c + threadIdx.x; r < b; r += 32) {
        const float2 v = aug[r * ld + c];
        const float m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        piv = bi;
        if (!(best > 0.f)) atomicExch(status, 1);
      }
    }
    __syncthreads();
    const int pr = piv;
    if (pr != c)
      for (int j = threadIdx.x; j < ld; j += blockDim.x) {
        const float2 t = aug[c * ld + j];
        aug[c * ld + j] = aug[pr * ld + j];
        aug[pr * ld + j] = t;
      }
    __syncthreads();
    const float2 d = aug[c * ld + c];
    const float den = d.x * d.x + d.y * d.y;
    const float2 inv = den > 0.f ? make_float2(d.x / den, -d.y / den) : make_float2(0.f, 0.f);
    __syncthreads();
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
      const float2 v = aug[c * ld + j];
      aug[c * ld + j] = make_float2(v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x);
    }
    // the multipliers are read before any thread overwrites column c
    for (int r = threadIdx.x; r < b; r += blockDim.x) fcol[r] = aug[r * ld + c];
    __syncthreads();
    for (int e = threadIdx.x; e < b * ld; e += blockDim.x) {
      const int r = e / ld, j = e % ld;
      if (r == c) continue;
      const float2 f = fcol[r];
      const float2 v = aug[c * ld + j];
      aug[e].x -= f.x * v.x - f.y * v.y;
      aug[e].y -= f.x * v.y + f.y * v.x;
    }
    __syncthreads();
  }
  float2* Pb = P + (long long)blockIdx.x * b * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) Pb[e] = aug[(e / b) * ld + b + e % b];
}

// C = W_:,k (n x b, row-major) for every body
__global__ void copy_col_block_kernel(float2* const* __restrict__ W, int n, int k0, int b, float2* __restrict__ C) {
  const long long body = blockIdx.y;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * b) return;
  const int i = (int)(e / b), c = (int)(e % b);
  C[body * n * b + e] = W[body][(long long)i * n + k0 + c];
}

// W_k,: = R (off the diagonal block), W_:,k = T (off the diagonal block), W_kk = P
__global__ void fix_kernel(float2* const* __restrict__ W, int n, int k0, int b, const float2* __restrict__ R,
                           const float2* __restrict__ T, const float2* __restrict__ P) {
  const long long body = blockIdx.y;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float2* Wb = W[body];
  if (e < (long long)b * n) {  // row block
    const int r = (int)(e / n), j = (int)(e % n);
    const bool diag = j >= k0 && j < k0 + b;
    Wb[(long long)(k0 + r) * n + j] = diag ? P[body * b * b + r * b + (j - k0)] : R[body * b * n + e];
  }
  if (e < (long long)n * b) {  // column block
    const int i = (int)(e / b), c = (int)(e % b);
    if (i < k0 || i >= k0 + b) Wb[(long long)i * n + k0 + c] = T[body * n * b + e];
  }
}

__global__ void widen_blocks_kernel(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2(a[i].x, a[i].y);
}

#define QAMS_CUBLAS(call)                                        \
  do {                                                           \
    cublasStatus_t s_ = (call);                                  \
    if (s_ != CUBLAS_STATUS_SUCCESS) {                           \
      qams_internal_last_cuda_error(cudaErrorUnknown, #call);    \
      rc = QAMS_ECUDA;                                           \
      goto done;                                                 \
    }                                                            \
  } while (0)

}  // namespace

int qams_precond_launch(qams_ctx* c, cudaStream_t st) {
  const int nb = (int)c->bodies.size();
  int rc = QAMS_OK;
  qams_dev_free(c, &c->pinv32);
  qams_dev_free(c, &c->pinv64);
  if ((rc = qams_dev_alloc(c, &c->pinv32, sizeof(float2) * (size_t)c->block_entries))) return rc;
  if ((rc = qams_dev_alloc(c, &c->pinv64, sizeof(double2) * (size_t)c->block_entries))) return rc;
  QAMS_CUDA(cudaMemcpyAsync(c->pinv32.p, c->blocks32.p, sizeof(float2) * (size_t)c->block_entries,
                            cudaMemcpyDeviceToDevice, st));
  // group bodies by size
  std::map<int, std::vector<int>> groups;
  std::vector<long long> boff(nb);
  long long off = 0;
  for (int b = 0; b < nb; ++b) {
    boff[b] = off;
    off += (long long)c->bodies[b].n * c->bodies[b].n;
    groups[c->bodies[b].n].push_back(b);
  }
  cublasHandle_t h = nullptr;
  DeviceBuf ptrs, Rb, Cb, Tb, Pb, stat;
  size_t maxg = 0, maxn = 0;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return QAMS_ECUDA;
  cublasSetStream(h, st);
  cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST);
  for (auto& g : groups) {
    maxg = std::max(maxg, g.second.size());
    maxn = std::max(maxn, (size_t)g.first);
  }
  if ((rc = qams_dev_alloc(c, &ptrs, sizeof(void*) * 6 * maxg))) goto done;
  if ((rc = qams_dev_alloc(c, &Rb, sizeof(float2) * maxg * BW * maxn))) goto done;
  if ((rc = qams_dev_alloc(c, &Cb, sizeof(float2) * maxg * BW * maxn))) goto done;
  if ((rc = qams_dev_alloc(c, &Tb, sizeof(float2) * maxg * BW * maxn))) goto done;
  if ((rc = qams_dev_alloc(c, &Pb, sizeof(float2) * maxg * BW * BW))) goto done;
  if ((rc = qams_dev_alloc(c, &stat, sizeof(int)))) goto done;
  if (cudaMemsetAsync(stat.p, 0, sizeof(int), st) != cudaSuccess) { rc = QAMS_ECUDA; goto done; }
  if (cudaFuncSetAttribute(pivot_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float2) * BW * 2 * BW)) != cudaSuccess) { rc = QAMS_ECUDA; goto done; }
  for (auto& g : groups) {
    const int n = g.first;
    const int G = (int)g.second.size();
    // pointer table: W[body], then per-body pointers of the GEMM operands
    std::vector<void*> hp(6 * (size_t)G);
    for (int q = 0; q < G; ++q) hp[q] = (float2*)c->pinv32.p + boff[g.second[q]];
    float2** dW = (float2**)ptrs.p;
    const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f),
                    mone = make_cuComplex(-1.f, 0.f);
    for (int k0 = 0; k0 < n; k0 += BW) {
      const int b = std::min(BW, n - k0);
      for (int q = 0; q < G; ++q) {
        float2* W = (float2*)hp[q];
        hp[G + q] = W + (long long)k0 * n;                 // W_k,: (row-major b x n)
        hp[2 * G + q] = (float2*)Rb.p + (long long)q * b * n;
        hp[3 * G + q] = (float2*)Cb.p + (long long)q * n * b;
        hp[4 * G + q] = (float2*)Pb.p + (long long)q * b * b;
        hp[5 * G + q] = (float2*)Tb.p + (long long)q * n * b;
      }
      if (cudaMemcpyAsync(ptrs.p, hp.data(), sizeof(void*) * 6 * G, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = QAMS_ECUDA;
        goto done;
      }
      if (cudaStreamSynchronize(st) != cudaSuccess) { rc = QAMS_ECUDA; goto done; }  // hp is rewritten next step
      pivot_inverse_kernel<<<G, 256, sizeof(float2) * b * 2 * b, st>>>(dW, n, k0, b, (float2*)Pb.p, (int*)stat.p);
      qams_count_launch();
      {
        const long long nbk = (long long)n * b;
        copy_col_block_kernel<<<dim3((unsigned)((nbk + 255) / 256), G), 256, 0, st>>>(dW, n, k0, b, (float2*)Cb.p);
        qams_count_launch();
      }
      {
        // column-major views: R^T (n x b) = W_k,:^T (n x b, ld n) * P^T (b x b, ld b)
        const cuComplex** A = (const cuComplex**)(dW + G);
        const cuComplex** B = (const cuComplex**)(dW + 4 * G);
        cuComplex** Cc = (cuComplex**)(dW + 2 * G);
        QAMS_CUBLAS(cublasCgemmBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, n, b, b, &one, A, n, B, b, &zero, Cc, n, G));
      }
      {
        // W^T (n x n) -= R^T (n x b, ld n) * C^T (b x n, ld b)
        const cuComplex** A = (const cuComplex**)(dW + 2 * G);
        const cuComplex** B = (const cuComplex**)(dW + 3 * G);
        cuComplex** Cc = (cuComplex**)dW;
        QAMS_CUBLAS(cublasCgemmBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, n, n, b, &mone, A, n, B, b, &one, Cc, n, G));
      }
      {
        // T^T (b x n, ld b) = -P^T (b x b) * C^T (b x n, ld b)
        const cuComplex** A = (const cuComplex**)(dW + 4 * G);
        const cuComplex** B = (const cuComplex**)(dW + 3 * G);
        cuComplex** Cc = (cuComplex**)(dW + 5 * G);
        QAMS_CUBLAS(cublasCgemmBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, b, n, b, &mone, A, b, B, b, &zero, Cc, b, G));
      }
      {
        const long long nbk = (long long)n * b;
        fix_kernel<<<dim3((unsigned)((nbk + 255) / 256), G), 256, 0, st>>>(dW, n, k0, b, (const float2*)Rb.p,
                                                                         (const float2*)Tb.p, (const float2*)Pb.p);
        qams_count_launch();
      }
      if (cudaGetLastError() != cudaSuccess) { rc = QAMS_ECUDA; goto done; }
    }
  }
  {
    const long long n = c->block_entries;
    widen_blocks_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float2*)c->pinv32.p,
                                                                     (double2*)c->pinv64.p, n);
    qams_count_launch();
    int hs = 0;
    if (cudaMemcpyAsync(&hs, stat.p, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = QAMS_ECUDA;
      goto done;
    }
    if (hs) rc = QAMS_ENUMERIC;
  }
done:
  if (h) cublasDestroy(h);
  for (DeviceBuf* b : {&ptrs, &Rb, &Cb, &Tb, &Pb, &stat}) qams_dev_free(c, b);
  return rc;
}
