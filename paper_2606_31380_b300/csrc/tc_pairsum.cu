// FP32 inter-body pair sum (Eq. multi2part) with its multiply-accumulate on
// the tensor cores (tcgen05, kind::tf32).
//
// For the targets t of one tile and the sources s of the other bodies,
//   y_t[r] = sum_s K(x_t, y_s) sigma_s[r],
// K as in pairsum.cu.  With R right-hand sides the CUDA-core kernel spends
// 4R FP32 FMAs per pair on this product besides the ~30 operations and 4
// MUFU evaluations of K.  Here the product is a GEMM: per CTA, 128 targets
// (rows, M = 128) times a running K dimension of 2 x (sources) real columns
// (re, im of K), times B = [sigma' re-columns | im-columns] with
//   B[2s][r] = sigma'_re, B[2s+1][r] = -sigma'_im, B[2s][R+r] = sigma'_im,
//   B[2s+1][R+r] = sigma'_re,   sigma' = sigma e^{ik rho_0(a, b)},
// so the body-pair phase e^{ik rho_0} (FP64, once per CTA and source body)
// is folded into the 16 x R sigma values of each sub-chunk rather than into
// every pair.  Operands are split for FP32-level accuracy:
// v = hi + lo with hi = v rounded to TF32 (11 significant bits) and lo the
// exact remainder (read as TF32 again), D = K_hi [S_hi; S_lo] + K_lo S_hi,
// i.e. about 22 bits per product with FP32 accumulation.
//
// CTA: eight K-evaluation warps for 128 targets -- warps w and w + 4 own the
// same tensor-memory lanes (targets) and evaluate the first and second 8 of
// each 16-source sub-chunk -- and one MMA warp.  The evaluation warps write
// their K_hi and K_lo values (16 columns each) to tensor memory with
// tcgen05.st and the sigma' tile (2NH rows x 32 FP32 = one 128-byte swizzle
// span) to shared memory in the 128-byte-swizzled K-major layout, then each
// arrives on the sub-chunk's "full" mbarrier.  The MMA warp waits for all
// eight, issues 4 K steps x 2 MMAs with A read from tensor memory and B from
// shared memory, and commits them to the buffer's "empty" mbarrier.  A and B
// are double-buffered, so the evaluation warps run up to two sub-chunks
// ahead of the MMAs; only body batches and 128-source staging steps
// synchronise the CTA.  D (128 x 2NH FP32) stays in
// tensor memory.  Accumulated in one D over all 511,488 sources of the
// 1000-body workload, the sums came out ~2e-3 too small in magnitude -- the
// signature of an accumulation that truncates each addition; so D is
// restarted every FLUSH sub-chunks (at most 64 additions per block), two D
// buffers alternate, and one sub-chunk after a block ends (once the regular
// buffer wait has shown its MMAs complete) warps 0-3 add it to FP32
// registers with round-to-nearest.  Waits are bounded; a timeout sets the
// error flag (QAMS_ETIMEOUT).
#include <cmath>

#include "qams_internal.h"
#include "tc_common.cuh"

namespace {

constexpr int TPT = 128;  // targets per CTA (MMA M)
constexpr int NCW = 8;               // K-evaluation warps: two threads per target
constexpr int NTH = (NCW + 1) * 32;  // plus one warp that issues the MMAs
constexpr int SRC = 128;  // sources staged in shared memory at a time
constexpr int SUB = 16;   // sources per sub-chunk (K = 32 TF32 values)
constexpr int BB = 32;    // source bodies whose body-pair constants are formed together
constexpr int TMEM_COLS = 256;  // D blocks at columns 0 and 64, A buffers at 128 and 192
constexpr int FLUSH = 8;        // sub-chunks accumulated in one D block
constexpr float INV_2PI_F = 0.15915494309189535f;
constexpr float TWO_PI_HI_F = 6.28318548202514648f;    // float(2 pi)
constexpr float TWO_PI_LO_F = -1.7484555314695172e-7f;  // 2 pi - TWO_PI_HI_F

struct TcPairArgs {
  const TargetTile* tiles;
  const SourceSplit* splits;
  const long long* boff;
  const qd4* centers;
  const float4* x32;
  const float4* n32;
  const float2* sigma;
  int R;
  double k, eta;
  float2* out;
  long long split_stride;
  int out_ld;
  int* err;
};

__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// byte offset of FP32 element (row, kc) in a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t sw128_off(int row, int kc) {
  return (uint32_t)(row * 128 + ((((kc >> 2) ^ (row & 7)) & 7) << 4) + ((kc & 3) << 2));
}

template <int NH>
__global__ void __launch_bounds__(NTH, 2) pairsum_tc_kernel(TcPairArgs a) {
  __shared__ float4 sp[SRC];
  __shared__ float4 sq[SRC];
  __shared__ float4 bdc[BB];  // dc = c_a - c_b (x, y, z), rho0
  __shared__ float4 bph[BB];  // rho0^2, cos k rho0, sin k rho0
  __shared__ uint64_t afull[2];   // a sub-chunk's K and sigma' are in place (one arrival per evaluation warp)
  __shared__ uint64_t aempty[2];  // its MMAs completed (tcgen05.commit)
  __shared__ uint64_t done;
  __shared__ uint32_t tslot;
  extern __shared__ uint8_t dsm[];
  constexpr int BT = 2 * NH * 128;  // bytes of one sigma' tile
  uint8_t* btile = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);

  const TargetTile tile = a.tiles[blockIdx.x];
  const SourceSplit split = a.splits[blockIdx.y];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = warp == NCW;         // the MMA warp
  const int row = (warp & 3) * 32 + lane;  // target within the tile = tensor-memory lane
  const int half = (warp >> 2) & 1;        // which 8 sources of a sub-chunk
  const bool active = !issuer && row < tile.count;
  const long long t = tile.start + (active ? row : 0);
  const float4 xt = a.x32[t];
  const float kf = (float)a.k, etaf = (float)a.eta;
  const int R = a.R;

  for (int i = tid; i < 2 * BT / 4; i += NTH) ((float*)btile)[i] = 0.f;  // rows beyond 2R stay zero
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&afull[i], NCW);
      mbar_init(&aempty[i], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tslot, TMEM_COLS);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeroed tiles, for the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);

  int g = 0;         // sub-chunks so far
  bool bad = false;  // a bounded wait gave up
  float acc[NH];     // warps 0-3: y columns (re R, im R) summed over finished D blocks
#pragma unroll
  for (int c = 0; c < NH; ++c) acc[c] = 0.f;
  // add D block `blk` (both its parts) to acc; warps 0-3 only, after its MMAs completed
  auto fold = [&](int blk) {
    const uint32_t base = lane_base + 64 * (blk & 1);
#pragma unroll
    for (int c = 0; c < NH; c += 16) {  // 16 columns of each part at a time (register pressure)
      float d0[16], d1[16];
      ld16(base + c, d0);
      ld16(base + NH + c, d1);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[c + i] += d0[i] + d1[i];
    }
  };

  for (int bb = split.begin; bb < split.end; bb += BB) {
    __syncthreads();
    if (tid < BB && bb + tid < split.end) {
      const qd4 ca = a.centers[tile.body], cb = a.centers[bb + tid];
      const double dcx = ca.x - cb.x, dcy = ca.y - cb.y, dcz = ca.z - cb.z;
      const double rho0 = sqrt(dcx * dcx + dcy * dcy + dcz * dcz);
      double s0d, c0d;
      sincos(a.k * rho0, &s0d, &c0d);
      bdc[tid] = make_float4((float)dcx, (float)dcy, (float)dcz, (float)rho0);
      bph[tid] = make_float4((float)(rho0 * rho0), (float)c0d, (float)s0d, 0.f);
    }
    __syncthreads();
    for (int b = bb; b < min(split.end, bb + BB); ++b) {
      if (b == tile.body) continue;
      const float4 dcv = bdc[b - bb], phv = bph[b - bb];
      const float fx = dcv.x, fy = dcv.y, fz = dcv.z, rho0f = dcv.w, r02 = phv.x;
      const float At = fx * xt.x + fy * xt.y + fz * xt.z;
      const long long send = a.boff[b + 1];
      for (long long s0 = a.boff[b]; s0 < send; s0 += SRC) {
        const int cnt = (int)min((long long)SRC, send - s0);
        if (issuer) {
          // MMA warp: per sub-chunk, wait until the evaluation warps filled it,
          // then 4 K steps x 2 MMAs into the current D block
          for (int j0 = 0; j0 < cnt; j0 += SUB, ++g) {
            const int p = g & 1;
            if (!bad) bad = !mbar_wait(&afull[p], (g >> 1) & 1, a.err);
            if (lane == 0) {
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              constexpr uint32_t id_full = idesc_tf32(TPT, 2 * NH), id_half = idesc_tf32(TPT, NH);
              const uint64_t bd = sdesc_sw128(btile + p * BT);
              const uint32_t ah = tmem + 128 + 64 * p, al = ah + 32;
              const uint32_t dt = tmem + 64 * ((g / FLUSH) & 1);
              const int f = g % FLUSH;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                mma_tf32_ts(dt, ah + 8 * kk, bd + 2 * kk, id_full, (f | kk) != 0);
                mma_tf32_ts(dt + NH, al + 8 * kk, bd + 2 * kk, id_half, 1u);
              }
              mma_commit(&aempty[p]);
            }
            __syncwarp();
          }
          continue;
        }
        // evaluation warps: stage the chunk's sources (named barrier of the 8 warps)
        asm volatile("bar.sync 1, %0;" ::"r"(NCW * 32) : "memory");
        if (tid < SRC) {
          const long long i = s0 + tid;
          if (i < send) {
            float4 p = a.x32[i];
            float4 q = a.n32[i];
            p.w = fx * p.x + fy * p.y + fz * p.z;  // dc . y~_s
            q.w = fx * q.x + fy * q.y + fz * q.z;  // n_s . dc
            sp[tid] = p;
            sq[tid] = q;
          }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(NCW * 32) : "memory");
        for (int j0 = 0; j0 < cnt; j0 += SUB, ++g) {
          const int p = g & 1;
          // buffers p (K in tensor memory, sigma' tile) are free once sub-chunk g-2's MMAs completed
          if (g >= 2 && !bad) bad = !mbar_wait(&aempty[p], ((g - 2) >> 1) & 1, a.err);
          // the previous D block ended with sub-chunk g - 2: add it to the registers
          if (g % FLUSH == 1 && g / FLUSH >= 1 && warp < 4) fold(g / FLUSH - 1);
          // sigma' tile: thread (s, r) writes its 4 hi and 4 lo values
          uint8_t* bt = btile + p * BT;
          if (tid < SUB * R) {
            const int s = tid / R, r = tid - s * R;
            float2 v = make_float2(0.f, 0.f);
            if (j0 + s < cnt) {
              const float2 sg = a.sigma[(s0 + j0 + s) * R + r];
              v = make_float2(phv.y * sg.x - phv.z * sg.y, phv.y * sg.y + phv.z * sg.x);
            }
            const float vals[4] = {v.x, -v.y, v.y, v.x};  // (row r: 2s, 2s+1), (row R + r: 2s, 2s+1)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int rr = (q < 2 ? r : R + r), kc = 2 * s + (q & 1);
              const float h = tf32_rn(vals[q]);
              *(float*)(bt + sw128_off(rr, kc)) = h;
              *(float*)(bt + sw128_off(NH + rr, kc)) = vals[q] - h;
            }
          }
          // K for this thread's 8 sources of the sub-chunk
          float vh[16], vl[16];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int j = j0 + half * 8 + u;
            float kre = 0.f, kim = 0.f;
            if (j < cnt) {
              const float4 ps = sp[j];
              const float4 qs = sq[j];
              const float dx = xt.x - ps.x, dy = xt.y - ps.y, dz = xt.z - ps.z;
              const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              const float e = fmaf(2.f, At - ps.w, dd);
              const float r2 = r02 + e;
              const float rinv = rsqrtf(r2);
              const float rho = r2 * rinv;
              const float delta = __fdividef(e, rho + rho0f);
              const float ph = kf * delta;
              const float nq = rintf(ph * INV_2PI_F);
              float red = fmaf(-nq, TWO_PI_HI_F, ph);
              red = fmaf(-nq, TWO_PI_LO_F, red);
              float sn, cs;
              __sincosf(red, &sn, &cs);
              const float nyx = -(qs.w + fmaf(qs.x, dx, fmaf(qs.y, dy, qs.z * dz)));
              const float are = -nyx * rinv * rinv;
              const float aim = fmaf(kf * nyx, rinv, -etaf);
              kre = (cs * are - sn * aim) * rinv;
              kim = (sn * are + cs * aim) * rinv;
            }
            const float hr = tf32_rn(kre), hi = tf32_rn(kim);
            vh[2 * u] = hr;
            vh[2 * u + 1] = hi;
            vl[2 * u] = kre - hr;
            vl[2 * u + 1] = kim - hi;
          }
          const uint32_t abase = lane_base + 128 + 64 * p;
          st16(abase + half * 16, vh);
          st16(abase + 32 + half * 16, vl);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&afull[p])) : "memory");
        }
      }
    }
  }
  if (issuer && lane == 0) mma_commit(&done);  // arrives once every MMA issued above has completed
  __syncthreads();
  const bool have = g > 0;
  if (have && warp < 4 && !mbar_wait(&done, 0, a.err)) bad = true;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp < 4) {
    if (have) {
      const int last = (g - 1) / FLUSH;
      if ((g - 1) % FLUSH == 0 && last >= 1) fold(last - 1);  // its fold point never came
      fold(last);
    }
    if (active && !bad) {
      const float inv4pi = 0.079577471545947668f;
      float2* o = a.out + a.split_stride * blockIdx.y + t * a.out_ld;
      float re[16], im[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        re[r] = 0.f;
        im[r] = 0.f;
      }
      // acc holds the re columns 0..R-1 and the im columns R..2R-1
#pragma unroll
      for (int c = 0; c < NH; ++c) {
        if (c < R) re[c & 15] = acc[c];
        else if (c < 2 * R) im[(c - R) & 15] = acc[c];
      }
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (r < R) o[r] = make_float2(re[r] * inv4pi, im[r] * inv4pi);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

// Launch of the tensor-core FP32 pair sum for all R (<= 16) right-hand sides
// at once; out / split_stride / out_ld as in pairsum.cu (partial sums per
// source split when there are several).  Returns QAMS_EINVAL for R > 16.
int qams_pairsum_tc_launch(qams_ctx* c, int R, const void* sigma, void* out, long long split_stride, int out_ld,
                           cudaStream_t st) {
  if (R < 1 || R > 16) return QAMS_EINVAL;
  if (!c->tc_err.p) {
    int rc = qams_dev_alloc(c, &c->tc_err, 64);
    if (rc) return rc;
    QAMS_CUDA(cudaMemsetAsync(c->tc_err.p, 0, 64, st));
  }
  TcPairArgs a{(const TargetTile*)c->d_tiles.p, (const SourceSplit*)c->d_splits.p, (const long long*)c->boff.p,
               (const qd4*)c->centers.p, (const float4*)c->x32.p, (const float4*)c->n32.p, (const float2*)sigma,
               R, c->k, c->eta, (float2*)out, split_stride, out_ld, (int*)c->tc_err.p};
  const dim3 grid((unsigned)c->tiles.size(), (unsigned)c->splits.size());
  static bool attr = false;
  const int smem16 = 2 * 2 * 16 * 128 + 1024, smem32 = 2 * 2 * 32 * 128 + 1024;
  if (!attr) {
    QAMS_CUDA(cudaFuncSetAttribute(pairsum_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem16));
    QAMS_CUDA(cudaFuncSetAttribute(pairsum_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32));
    attr = true;
  }
  if (2 * R <= 16)
    pairsum_tc_kernel<16><<<grid, NTH, smem16, st>>>(a);
  else
    pairsum_tc_kernel<32><<<grid, NTH, smem32, st>>>(a);
  qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  return QAMS_OK;
}
