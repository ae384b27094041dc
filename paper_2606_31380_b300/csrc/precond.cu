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
// after which W = A_b^{-1}.  The three products run in an own tiled
// complex64 GEMM kernel (64 x 64 output tiles, 16-wide K chunks staged in
// shared memory, 4 x 4 complex outputs per thread), batched over bodies of
// equal size in one launch per product.  Pivoting is local to the diagonal
// blocks; the self blocks of the second-kind combined-field operator
// (1/2 I plus a smoothing part) keep them well conditioned, and a
// vanishing pivot is reported as QAMS_ENUMERIC.
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

// One GEMM operand per batch entry z: tab[z] + off when a pointer table is
// given, else base + z * bstride + off; row-major with leading dimension ld.
struct Opnd {
  float2* const* tab;
  float2* base;
  long long off, bstride;
  int ld;
};

__device__ __forceinline__ float2* opnd_ptr(const Opnd& o, int z) {
  return o.tab ? o.tab[z] + o.off : o.base + (long long)z * o.bstride + o.off;
}

constexpr int GT = 64;  // output tile (rows and columns)
constexpr int GK = 16;  // K chunk

// D = alpha A B (+ D when accumulate) for complex64 row-major A (M x K),
// B (K x N), D (M x N); grid (N tiles, M tiles, batch).
__global__ void __launch_bounds__(256) cgemm_kernel(Opnd A, Opnd B, Opnd D, int M, int N, int K, float2 alpha,
                                                    int accumulate) {
  __shared__ float2 As[GK][GT + 1];
  __shared__ float2 Bs[GK][GT];
  const int z = blockIdx.z;
  const float2* a = opnd_ptr(A, z);
  const float2* b = opnd_ptr(B, z);
  float2* d = opnd_ptr(D, z);
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = t + 256 * q;
      const int am = idx >> 4, ak = idx & 15;  // A tile: 64 rows x 16
      As[ak][am] = (m0 + am < M && k0 + ak < K) ? a[(long long)(m0 + am) * A.ld + k0 + ak] : make_float2(0.f, 0.f);
      const int bk = idx >> 6, bn = idx & 63;  // B tile: 16 rows x 64
      Bs[bk][bn] = (k0 + bk < K && n0 + bn < N) ? b[(long long)(k0 + bk) * B.ld + n0 + bn] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      float2 av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(av[i].x, bv[j].x, fmaf(-av[i].y, bv[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(av[i].x, bv[j].y, fmaf(av[i].y, bv[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      float2* o = d + (long long)m * D.ld + n;
      float2 v = make_float2(alpha.x * acc[i][j].x - alpha.y * acc[i][j].y,
                             alpha.x * acc[i][j].y + alpha.y * acc[i][j].x);
      if (accumulate) {
        v.x += o->x;
        v.y += o->y;
      }
      *o = v;
    }
  }
}

void cgemm(const Opnd& A, const Opnd& B, const Opnd& D, int M, int N, int K, float2 alpha, int accumulate, int G,
           cudaStream_t st) {
  const dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)((M + GT - 1) / GT), (unsigned)G);
  cgemm_kernel<<<grid, 256, 0, st>>>(A, B, D, M, N, K, alpha, accumulate);
  qams_count_launch();
}

__global__ void widen_blocks_kernel(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2(a[i].x, a[i].y);
}

}  // namespace

int qams_precond_launch(qams_ctx* c, cudaStream_t st) {
  int rc = QAMS_OK;
  qams_dev_free(c, &c->pinv32);
  qams_dev_free(c, &c->pinv64);
  if ((rc = qams_dev_alloc(c, &c->pinv32, sizeof(float2) * (size_t)c->block_entries))) return rc;
  if ((rc = qams_dev_alloc(c, &c->pinv64, sizeof(double2) * (size_t)c->block_entries))) return rc;
  QAMS_CUDA(cudaMemcpyAsync(c->pinv32.p, c->blocks32.p, sizeof(float2) * (size_t)c->block_entries,
                            cudaMemcpyDeviceToDevice, st));
  // one inverse per class of congruent bodies, grouped by size
  std::map<int, std::vector<int>> groups;
  std::vector<long long> boff(c->class_rep.size());
  for (size_t k = 0; k < c->class_rep.size(); ++k) {
    boff[k] = c->class_blk[k];
    groups[c->bodies[c->class_rep[k]].n].push_back((int)k);
  }
  DeviceBuf ptrs, Rb, Cb, Tb, Pb, stat;
  size_t maxg = 0, maxn = 0;
  for (auto& g : groups) {
    maxg = std::max(maxg, g.second.size());
    maxn = std::max(maxn, (size_t)g.first);
  }
  if ((rc = qams_dev_alloc(c, &ptrs, sizeof(void*) * maxg))) goto done;
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
    // pointer table of the group's matrices W (fixed for the whole elimination)
    std::vector<float2*> hp((size_t)G);
    for (int q = 0; q < G; ++q) hp[q] = (float2*)c->pinv32.p + boff[g.second[q]];
    float2** dW = (float2**)ptrs.p;
    if (cudaMemcpyAsync(ptrs.p, hp.data(), sizeof(float2*) * G, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = QAMS_ECUDA;
      goto done;
    }
    for (int k0 = 0; k0 < n; k0 += BW) {
      const int b = std::min(BW, n - k0);
      pivot_inverse_kernel<<<G, 256, sizeof(float2) * b * 2 * b, st>>>(dW, n, k0, b, (float2*)Pb.p, (int*)stat.p);
      qams_count_launch();
      {
        const long long nbk = (long long)n * b;
        copy_col_block_kernel<<<dim3((unsigned)((nbk + 255) / 256), G), 256, 0, st>>>(dW, n, k0, b, (float2*)Cb.p);
        qams_count_launch();
      }
      const Opnd Wk{dW, nullptr, (long long)k0 * n, 0, n};              // W_k,: (b x n, ld n)
      const Opnd Wf{dW, nullptr, 0, 0, n};                              // W (n x n)
      const Opnd Ro{nullptr, (float2*)Rb.p, 0, (long long)b * n, n};   // R (b x n)
      const Opnd Co{nullptr, (float2*)Cb.p, 0, (long long)n * b, b};   // C (n x b)
      const Opnd Po{nullptr, (float2*)Pb.p, 0, (long long)b * b, b};   // P (b x b)
      const Opnd To{nullptr, (float2*)Tb.p, 0, (long long)n * b, b};   // T (n x b)
      cgemm(Po, Wk, Ro, b, n, b, make_float2(1.f, 0.f), 0, G, st);   // R = P W_k,:
      cgemm(Co, Ro, Wf, n, n, b, make_float2(-1.f, 0.f), 1, G, st);  // W -= C R
      cgemm(Co, Po, To, n, b, b, make_float2(-1.f, 0.f), 0, G, st);  // T = -C P
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
  if (rc == QAMS_OK) rc = qams_tc_prepare(c, 1, st);  // split copy for the tensor-core product
done:
  for (DeviceBuf* b : {&ptrs, &Rb, &Cb, &Tb, &Pb, &stat}) qams_dev_free(c, b);
  return rc;
}
