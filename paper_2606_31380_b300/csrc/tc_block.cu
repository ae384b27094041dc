// Self-block and preconditioner products on the tensor cores (tcgen05/TMEM).
//
// The FP32 operator applies, for every body b, Y_b = M_b X_b with M_b the
// complex n x n self block A_b or preconditioner block P_b (the dense
// diagonal blocks of Eq. linearsys) and X_b the body's [n][R] slice of the
// unknowns.  With many right-hand sides this is a dense GEMM.  Written as a
// real product it needs no rearrangement of the stored block: the row-major
// complex block read as floats is a real n x 2n matrix M' (re, im
// interleaved along the row), and
//     Y = M' B,   B[2s][r]   =  x_re(s,r),  B[2s+1][r]   = -x_im(s,r),
//                 B[2s][R+r] =  x_im(s,r),  B[2s+1][R+r] =  x_re(s,r),
// i.e. M = n (rows), K = 2n, N = 2R (real and imaginary output columns).
//
// Precision: FP16 operands with FP32 accumulation, each operand split in
// two FP16 parts, v = hi + lo / 2^11 (hi = fp16(v), lo = fp16((v - hi) 2^11)),
// after Ootomo and Yokota, "Recovering single precision accuracy from
// Tensor Cores while surpassing the FP32 theoretical peak performance"
// (IJHPCA 2022): M' B ~ M_hi B_hi + (M_hi B_lo + M_lo B_hi) / 2^11 keeps
// about 22 significant bits, FP32-level accuracy.  Each body's part of
// every column of x is scaled by a power of two so that its largest entry
// lies in [2^13, 2^14);
// blocks are used unscaled and must stay below 2^14 in magnitude (checked
// when the split copy is built; otherwise the CUDA-core product is used).
// The split copies hold 2 x 2 bytes per real entry: the same 8 bytes per
// complex entry that the complex64 product streams.
//
// Kernel: one CTA per (body, 128-row tile).  One thread issues TMA loads of
// 128 x 64 FP16 tiles of M_hi and M_lo and 2NH x 64 tiles of B (128-byte
// swizzle) into a 4-stage ring guarded by mbarriers; one thread issues, per
// 16-wide K step, two tcgen05.mma: D[:, 0:2NH] += M_hi [B_hi; B_lo] and
// D[:, NH:2NH] += M_lo B_hi, with D (128 x 2NH FP32) in tensor memory.
// Every wait is bounded (about 2^31 clock cycles); a timeout sets an error
// flag, the CTA drains what it issued, frees its tensor memory and returns.
// After the K loop four warps read D with tcgen05.ld, combine the parts,
// undo the column scales and write (or add to) y.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qams_internal.h"
#include "tc_common.cuh"

namespace {

constexpr int BM = 128;       // rows per tile (M of the MMA)
constexpr int BK = 64;        // FP16 elements per K chunk (128 bytes: one swizzle span)
constexpr int STAGES = 4;
constexpr int A_TILE = BM * BK * 2;  // 16 KB
constexpr int B_TILE = 64 * BK * 2;  // up to 2NH = 64 rows: 8 KB
constexpr int SMEM_BYTES = STAGES * (2 * A_TILE + B_TILE) + 256 + 1024;

struct TcParams {
  int n;            // rows of each block (K = 2n)
  int mtiles;       // ceil(n / BM)
  int R, NH;        // right-hand sides; half width of the B tile (multiple of 16, >= 2R)
  long long node0;  // first node of the group's first body
  const unsigned* colmax;  // [bodies][R] largest |x| of each body's column (float bits)
  float2* y;
  int accumulate;
  int* err;
};

// power-of-two scale putting the column maximum in [2^13, 2^14), and its inverse
__device__ __forceinline__ void col_scale(unsigned bits, float* sc, float* inv) {
  const float m = __uint_as_float(bits);
  if (!(m > 0.f)) {
    *sc = 1.f;
    *inv = 1.f;
    return;
  }
  int e;
  frexpf(m, &e);  // m < 2^e
  *sc = ldexpf(1.f, 14 - e);
  *inv = ldexpf(1.f, e - 14);
}

template <int NH>
__global__ void __launch_bounds__(128, 1) tc_block_kernel(const __grid_constant__ CUtensorMap mAhi,
                                                          const __grid_constant__ CUtensorMap mAlo,
                                                          const __grid_constant__ CUtensorMap mB, TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment of the shared-space address (the swizzle pattern repeats every 8 rows of 128 B)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* a_hi = smem;
  uint8_t* a_lo = smem + STAGES * A_TILE;
  uint8_t* b_t = smem + 2 * STAGES * A_TILE;
  uint64_t* full = (uint64_t*)(b_t + STAGES * B_TILE);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  constexpr int NCOL = 2 * NH <= 32 ? 32 : 64;  // tensor-memory columns (power of two >= 32)

  const int body = blockIdx.x / p.mtiles;
  const int mt = blockIdx.x % p.mtiles;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nK = (2 * p.n + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA ring
    constexpr uint32_t bytes = 2 * A_TILE + 2 * NH * BK * 2;
    int issued = 0;
    for (int kc = 0; kc < nK; ++kc) {
      const int s = kc % STAGES;
      if (!mbar_wait(&empty[s], ((kc / STAGES) & 1) ^ 1, p.err)) break;
      mbar_expect_tx(&full[s], bytes);
      tma_load_3d(a_hi + s * A_TILE, &mAhi, &full[s], kc * BK, mt * BM, body);
      tma_load_3d(a_lo + s * A_TILE, &mAlo, &full[s], kc * BK, mt * BM, body);
      tma_load_3d(b_t + s * B_TILE, &mB, &full[s], kc * BK, 0, body);
      issued = kc + 1;
    }
    if (issued < nK) {
      // gave up: wait (bounded) until every issued copy has landed
      for (int kc = issued > STAGES ? issued - STAGES : 0; kc < issued; ++kc)
        mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1, p.err);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t id_full = idesc_f16(BM, 2 * NH), id_half = idesc_f16(BM, NH);
    for (int kc = 0; kc < nK; ++kc) {
      const int s = kc % STAGES;
      if (!mbar_wait(&full[s], (kc / STAGES) & 1, p.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t dh = sdesc_sw128(a_hi + s * A_TILE), dl = sdesc_sw128(a_lo + s * A_TILE),
                     db = sdesc_sw128(b_t + s * B_TILE);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        // +32 bytes per 16-element K step inside the 128-byte swizzle span
        mma_f16(tmem, dh + 2 * k, db + 2 * k, id_full, (kc | k) != 0);
        mma_f16(tmem + NH, dl + 2 * k, db + 2 * k, id_half, 1u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);  // also after an early exit: the epilogue waits for what was issued
  }
  __syncwarp();

  // epilogue: all four warps, one TMEM lane (tile row) per thread
  const bool ok = mbar_wait(done, 0, p.err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float d[2 * NH];
#pragma unroll
  for (int c = 0; c < 2 * NH; c += 16) ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, d + c);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  const int m = mt * BM + warp * 32 + lane;
  if (ok && m < p.n && !*(volatile int*)p.err) {
    float2* yr = p.y + (p.node0 + (long long)body * p.n + m) * p.R;
    const float lo_w = 1.f / 2048.f;
    for (int r = 0; r < p.R; ++r) {
      float sc, inv;
      col_scale(p.colmax[body * p.R + r], &sc, &inv);
      float2 v = make_float2((d[r] + lo_w * d[NH + r]) * inv, (d[p.R + r] + lo_w * d[NH + p.R + r]) * inv);
      if (p.accumulate) {
        const float2 o = yr[r];
        v.x += o.x;
        v.y += o.y;
      }
      yr[r] = v;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
}

// hi/lo FP16 split of an FP32 array (the blocks, read as floats); largest
// magnitude to *amax (float bits, atomicMax on non-negative floats)
__global__ void split_blocks_kernel(const float* __restrict__ a, __half* __restrict__ hi, __half* __restrict__ lo,
                                    long long n, unsigned* __restrict__ amax) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = a[i];
    const __half h = __float2half_rn(v);
    hi[i] = h;
    lo[i] = __float2half_rn((v - __half2float(h)) * 2048.f);
    m = fmaxf(m, fabsf(v));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

// largest |re|, |im| of every (body, column) of x [N][R] within one size
// group: cm[b R + r] for the group's bodies b (n nodes each from node0)
__global__ void colmax_kernel(const float2* __restrict__ x, long long node0, int n, int nb, int R,
                              unsigned* __restrict__ cm) {
  const long long total = (long long)nb * n * R;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = x[node0 * R + i];
    const float m = fmaxf(fabsf(v.x), fabsf(v.y));
    const long long node = i / R;
    if (m > 0.f) atomicMax(&cm[(node / n) * R + i % R], __float_as_uint(m));
  }
}

// B tiles of one size group: Bt[body][j][k], j < NH the scaled hi parts,
// NH <= j < 2NH the lo parts (see the header for the row/column meaning)
__global__ void split_x_kernel(const float2* __restrict__ x, long long node0, int n, int nb, int R, int NH,
                               const unsigned* __restrict__ cm, __half* __restrict__ bt) {
  const long long total = (long long)nb * n * R;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i % n);
    const long long q = i / n;
    const int r = (int)(q % R);
    const int b = (int)(q / R);
    float sc, inv;
    col_scale(cm[b * R + r], &sc, &inv);
    const float2 v = x[(node0 + (long long)b * n + s) * R + r];
    const float xr = v.x * sc, xi = v.y * sc;
    const long long K = 2LL * n;
    __half* base = bt + (long long)b * 2 * NH * K;
    const float vals[4] = {xr, -xi, xi, xr};  // rows r (k = 2s, 2s+1) and R + r
    const int rows[2] = {r, R + r};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float w = vals[2 * h + c];
        const __half hv = __float2half_rn(w);
        const __half lv = __float2half_rn((w - __half2float(hv)) * 2048.f);
        base[(long long)rows[h] * K + 2 * s + c] = hv;
        base[(long long)(NH + rows[h]) * K + 2 * s + c] = lv;
      }
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 3-D FP16 map {2n (K), rows, bodies} with a {64, box_rows, 1} box, 128-byte swizzle
int encode_map(CUtensorMap* map, const void* base, int n, int rows, int nb, int box_rows) {
  auto fn = get_encode();
  if (!fn) return QAMS_ECUDA;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * n), (cuuint64_t)rows, (cuuint64_t)nb};
  const cuuint64_t strides[2] = {(cuuint64_t)(4 * n), (cuuint64_t)(4LL * n * rows)};
  const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    qams_internal_last_cuda_error(cudaErrorInvalidValue, "cuTensorMapEncodeTiled");
    return QAMS_ECUDA;
  }
  return QAMS_OK;
}

}  // namespace

// Contiguous runs of equal-size bodies (one tensor map each); empty when a
// body size does not suit the tensor path (n % 8 != 0).
int qams_tc_groups(qams_ctx* c) {
  c->tc_groups.clear();
  const int nb = (int)c->bodies.size();
  // the tensor maps address one block per body: with congruent bodies sharing
  // blocks the CUDA-core product (which follows the per-body offsets) is used
  if ((int)c->class_rep.size() != nb) return QAMS_OK;
  long long elem = 0;
  for (int b = 0; b < nb;) {
    const int n = c->bodies[b].n;
    if (n % 8 != 0) {
      c->tc_groups.clear();
      return QAMS_OK;
    }
    TcGroup g{b, 0, n, c->bodies[b].offset, elem};
    while (b < nb && c->bodies[b].n == n) {
      ++g.nb;
      elem += (long long)n * n;
      ++b;
    }
    c->tc_groups.push_back(g);
  }
  return QAMS_OK;
}

// Split copy (FP16 hi/lo) of a complex64 block set for the tensor path.
// which = 0: self blocks, 1: preconditioner.  Blocking (reads back the
// largest magnitude).
int qams_tc_prepare(qams_ctx* c, int which, cudaStream_t st) {
  DeviceBuf& hi = which ? c->tc_pinv_hi : c->tc_blk_hi;
  DeviceBuf& lo = which ? c->tc_pinv_lo : c->tc_blk_lo;
  bool& ok = which ? c->tc_pinv_ok : c->tc_blk_ok;
  const void* src = which ? c->pinv32.p : c->blocks32.p;
  ok = false;
  qams_dev_free(c, &hi);
  qams_dev_free(c, &lo);
  if (c->tc_groups.empty() || !src) return QAMS_OK;
  const long long nf = 2 * c->block_entries;  // floats
  int rc;
  if ((rc = qams_dev_alloc(c, &hi, sizeof(__half) * nf))) return rc;
  if ((rc = qams_dev_alloc(c, &lo, sizeof(__half) * nf))) return rc;
  if (!c->tc_amax.p && (rc = qams_dev_alloc(c, &c->tc_amax, 256))) return rc;
  QAMS_CUDA(cudaMemsetAsync(c->tc_amax.p, 0, sizeof(unsigned), st));
  split_blocks_kernel<<<1184, 256, 0, st>>>((const float*)src, (__half*)hi.p, (__half*)lo.p, nf,
                                            (unsigned*)c->tc_amax.p);
  qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  unsigned bits = 0;
  QAMS_CUDA(cudaMemcpyAsync(&bits, c->tc_amax.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  QAMS_CUDA(cudaStreamSynchronize(st));
  float amax;
  std::memcpy(&amax, &bits, sizeof(float));
  ok = std::isfinite(amax) && amax < 16384.f;
  if (!ok) {
    qams_dev_free(c, &hi);
    qams_dev_free(c, &lo);
  }
  return QAMS_OK;
}

// y (+)= M x on the tensor cores for the complex64 vectors x, y [N][R],
// M = self blocks (which = 0) or preconditioner (1).  QAMS_EINVAL when the
// split copy is not available (the caller then uses the CUDA-core product).
int qams_tc_block_apply(qams_ctx* c, int which, int R, const void* x, void* y, bool accumulate, cudaStream_t st) {
  const bool ok = which ? c->tc_pinv_ok : c->tc_blk_ok;
  if (!ok || R < 1 || R > 16 || c->tc_groups.empty()) return QAMS_EINVAL;
  const DeviceBuf& hi = which ? c->tc_pinv_hi : c->tc_blk_hi;
  const DeviceBuf& lo = which ? c->tc_pinv_lo : c->tc_blk_lo;
  const int NH = 2 * R <= 16 ? 16 : 32;
  int rc;
  // B tiles for the largest group, zero rows beyond 2R kept zero
  size_t need = 0;
  for (const TcGroup& g : c->tc_groups) need = std::max(need, sizeof(__half) * (size_t)g.nb * 2 * NH * 2 * g.n);
  if (c->tc_bt.bytes < need) {
    qams_dev_free(c, &c->tc_bt);
    if ((rc = qams_dev_alloc(c, &c->tc_bt, need))) return rc;
    c->tc_bt_R = -1;
  }
  if (!c->tc_err.p) {
    if ((rc = qams_dev_alloc(c, &c->tc_err, 64))) return rc;
    QAMS_CUDA(cudaMemsetAsync(c->tc_err.p, 0, 64, st));
  }
  int maxnb = 0;
  for (const TcGroup& g : c->tc_groups) maxnb = std::max(maxnb, g.nb);
  const size_t cm_bytes = sizeof(unsigned) * (1 + (size_t)maxnb * 16);
  if (c->tc_amax.bytes < cm_bytes) {
    qams_dev_free(c, &c->tc_amax);
    if ((rc = qams_dev_alloc(c, &c->tc_amax, cm_bytes))) return rc;
  }
  unsigned* cm = (unsigned*)c->tc_amax.p + 1;  // [bodies of the group][R] column maxima
  static bool attr = false;
  if (!attr) {
    QAMS_CUDA(cudaFuncSetAttribute(tc_block_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    QAMS_CUDA(cudaFuncSetAttribute(tc_block_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr = true;
  }
  for (const TcGroup& g : c->tc_groups) {
    if (c->tc_bt_R != R || c->tc_groups.size() > 1)
      QAMS_CUDA(cudaMemsetAsync(c->tc_bt.p, 0, sizeof(__half) * (size_t)g.nb * 2 * NH * 2 * g.n, st));
    const long long work = (long long)g.nb * g.n * R;
    QAMS_CUDA(cudaMemsetAsync(cm, 0, sizeof(unsigned) * (size_t)g.nb * R, st));
    colmax_kernel<<<(unsigned)std::min<long long>(2368, (work + 255) / 256), 256, 0, st>>>(
        (const float2*)x, g.node0, g.n, g.nb, R, cm);
    qams_count_launch();
    split_x_kernel<<<(unsigned)std::min<long long>(4096, (work + 255) / 256), 256, 0, st>>>(
        (const float2*)x, g.node0, g.n, g.nb, R, NH, cm, (__half*)c->tc_bt.p);
    qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
    CUtensorMap mh, ml, mb;
    const size_t eoff = (size_t)g.elem0 * 2;  // FP16 elements before the group's first block
    if ((rc = encode_map(&mh, (const __half*)hi.p + eoff, g.n, g.n, g.nb, BM))) return rc;
    if ((rc = encode_map(&ml, (const __half*)lo.p + eoff, g.n, g.n, g.nb, BM))) return rc;
    if ((rc = encode_map(&mb, c->tc_bt.p, g.n, 2 * NH, g.nb, 2 * NH))) return rc;
    TcParams p{g.n, (g.n + BM - 1) / BM, R, NH, g.node0, cm, (float2*)y, accumulate ? 1 : 0, (int*)c->tc_err.p};
    const unsigned grid = (unsigned)(g.nb * p.mtiles);
    cudaEvent_t pe = qams_prof_begin(c, QAMS_PROF_BLOCK_TC, st);
    if (NH == 16)
      tc_block_kernel<16><<<grid, 128, SMEM_BYTES, st>>>(mh, ml, mb, p);
    else
      tc_block_kernel<32><<<grid, 128, SMEM_BYTES, st>>>(mh, ml, mb, p);
    qams_prof_end(c, QAMS_PROF_BLOCK_TC, st, pe);
    qams_count_launch();
    QAMS_CUDA(cudaGetLastError());
  }
  c->tc_bt_R = R;
  return QAMS_OK;
}

// Timeout flag of the tensor-core kernels (a bounded wait gave up).
int qams_tc_check(qams_ctx* c, cudaStream_t st) {
  if (!c->tc_err.p) return QAMS_OK;
  int e = 0;
  QAMS_CUDA(cudaMemcpyAsync(&e, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  QAMS_CUDA(cudaStreamSynchronize(st));
  return e ? QAMS_ETIMEOUT : QAMS_OK;
}

namespace {
// One CTA waits, as the tensor-core kernels do, on an mbarrier that nothing
// completes; the bounded wait gives up after `cycles` and records it.
__global__ void wait_selftest_kernel(int* err, long long cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, err, cycles);
}
}  // namespace

extern "C" int qams_selftest_timeout(int cuda_device, long long cycles, void* stream) {
  if (cycles < 1 || cycles > (1LL << 32)) return QAMS_EINVAL;
  int count = 0;
  QAMS_CUDA(cudaGetDeviceCount(&count));
  if (cuda_device < 0 || cuda_device >= count) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(cuda_device));
  cudaStream_t st = (cudaStream_t)stream;
  int* d_err = nullptr;
  QAMS_CUDA(cudaMalloc(&d_err, sizeof(int)));
  int e = 0;
  cudaError_t ce = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (ce == cudaSuccess) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(d_err, cycles);
    qams_count_launch();
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  cudaFree(d_err);
  if (ce != cudaSuccess) {
    qams_internal_last_cuda_error(ce, "qams_selftest_timeout");
    return QAMS_ECUDA;
  }
  return e ? QAMS_ETIMEOUT : QAMS_OK;
}
