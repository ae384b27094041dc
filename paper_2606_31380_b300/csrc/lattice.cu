// Translation-invariant pair sum on a regular lattice of one rigid shape
// (Sec. 4, regular P x Q x R arrays with uniform spacing; Table
// tab:multibody_cubic).
//
// When every body is the same reference shape with the same rotation and
// the centres are c_{pqr} = c_0 + p a0 + q a1 + r a2, the inter-body block
// between bodies t and s depends only on their lattice displacement
// d = (p_t - p_s, q_t - q_s, r_t - r_s):
//   D_{t,s}[i][j] = T(d)[i][j] = K(x~_i + d0 a0 + d1 a1 + d2 a2, y~_j),
// with x~ the body-local nodes and K the kernel of Eq. multi2part (weights
// folded into sigma), T(0) = 0 (the self block is applied separately).  The
// pair sum is then a three-level block-Toeplitz product
//   y_t = sum_s T(t - s) sigma_s.
// The paper evaluates the (2P-1)(2Q-1)(2R-1) - 1 distinct blocks once and
// copies them into the dense matrix.  Here the distinct blocks are embedded
// in a circulant of period L_k = 2 P_k - 1 along each axis (every
// displacement in [-(P_k - 1), P_k - 1] lands on its own residue), which the
// 3-D discrete Fourier transform diagonalises:
//   y = IDFT_f( T^(f) DFT(sigma)(f) ),  T^(f) = sum_d T(d) e^{-2 pi i f.d/L},
// one dense n x n by n x R product per frequency f.  T^ is formed once per
// wavenumber (kernel values in FP64, the transform in float-float; kept in
// complex128 and rounded to complex64); an apply
// is three DFT passes over the zero-padded densities, the frequency
// products, and three inverse passes cropped to the lattice.  The DFTs are
// direct sums along one axis at a time (L_k <= 63), staged in shared memory.
#include <algorithm>
#include <cmath>

#include "ffloat.cuh"
#include "phase.cuh"
#include "qams_internal.h"

namespace {

constexpr int CB = 32;        // columns per CTA of a DFT pass (one warp wide)
constexpr int DFT_THREADS = 128;
constexpr int MAXL = 64;      // twiddle slots per table (L <= 63)

template <typename T2>
struct Real;
template <>
struct Real<double2> {
  using T = double;
};
template <>
struct Real<float2> {
  using T = float;
};

// T(d) of every residue of the circulant grid, FP64, layout [o0][o1][o2][i][j]
// (o_k = d_k mod L_k).  x64/n64 are the world nodes of the context; body 0's
// n nodes (centre c0) give the body-local positions.
__global__ void lattice_blocks_kernel(const qd4* __restrict__ x64, const qd4* __restrict__ n64,
                                      const qd4* __restrict__ centers, int n, int L0, int L1, int L2, int P0,
                                      int P1, int P2, double3 a0, double3 a1, double3 a2, double k, double eta,
                                      double2* __restrict__ T) {
  __shared__ double2 ptab[PH_N];
  phase_table_fill(ptab);
  __syncthreads();
  const long long nn = (long long)n * n;
  const long long total = (long long)L0 * L1 * L2 * nn;
  const qd4 c0 = centers[0];
  const double inv4pi = 0.07957747154594767;  // 1/(4 pi)
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long o = idx / nn;
    const int ij = (int)(idx - o * nn);
    const int i = ij / n, j = ij - (ij / n) * n;
    const int o2 = (int)(o % L2), o1 = (int)((o / L2) % L1), o0 = (int)(o / ((long long)L1 * L2));
    const int d0 = o0 < P0 ? o0 : o0 - L0, d1 = o1 < P1 ? o1 : o1 - L1, d2 = o2 < P2 ? o2 : o2 - L2;
    if (d0 == 0 && d1 == 0 && d2 == 0) {
      T[idx] = make_double2(0.0, 0.0);
      continue;
    }
    const qd4 xi = x64[i], yj = x64[j], nj = n64[j];
    // r = x~_i + d.A - y~_j, the centre c0 cancelling between x~ and y~
    const double rx = (xi.x - c0.x) - (yj.x - c0.x) + d0 * a0.x + d1 * a1.x + d2 * a2.x;
    const double ry = (xi.y - c0.y) - (yj.y - c0.y) + d0 * a0.y + d1 * a1.y + d2 * a2.y;
    const double rz = (xi.z - c0.z) - (yj.z - c0.z) + d0 * a0.z + d1 * a1.z + d2 * a2.z;
    const double rho = sqrt(rx * rx + ry * ry + rz * rz);
    const double inv = 1.0 / rho;
    const double nd = -(nj.x * rx + nj.y * ry + nj.z * rz);  // n_s . (y_s - x_t)
    double s, c;
    sincos_table(k * rho, ptab, &s, &c);
    const double g = inv * inv4pi;
    const double bre = -nd * inv * inv, bim = k * nd * inv - eta;
    T[idx] = make_double2(g * (c * bre - s * bim), g * (c * bim + s * bre));
  }
}

__global__ void round_kernel(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// One DFT pass along one lattice axis.  A line is a0 < n_a0, a1 < n_a1; its
// element j (< Jin) at column b (< B) is in[a0 is0 + a1 is1 + j iB + b],
// and output f (< Jout) goes to out[a0 os0 + a1 os1 + f oB + b]:
//   out_f = scale sum_{j < Jin} in_j tw[(j f) mod L].
// A CTA stages all Jin inputs of its CB columns before writing, and CTAs own
// disjoint (line, column) ranges, so in == out (same strides) is allowed.
struct AxisPass {
  long long B;
  int n_a0, n_a1;
  long long is0, is1, iB;
  long long os0, os1, oB;
  int Jin, Jout, L;
};

template <typename T2>
__global__ void __launch_bounds__(DFT_THREADS) axis_dft_kernel(const T2* in, T2* out, AxisPass p,
                                                               const T2* __restrict__ tw,
                                                               typename Real<T2>::T scale) {
  using F = typename Real<T2>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* s = reinterpret_cast<T2*>(smraw);  // [Jin][CB]
  T2* stw = s + p.Jin * CB;              // [L]
  const int line = blockIdx.y;
  const int a0 = line / p.n_a1, a1 = line - (line / p.n_a1) * p.n_a1;
  const long long b0 = (long long)blockIdx.x * CB;
  const long long ibase = a0 * p.is0 + a1 * p.is1 + b0, obase = a0 * p.os0 + a1 * p.os1 + b0;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < p.Jin * CB; idx += DFT_THREADS) {
    const int j = idx / CB, cc = idx - (idx / CB) * CB;
    T2 v;
    v.x = F(0);
    v.y = F(0);
    if (b0 + cc < p.B) v = in[ibase + j * p.iB + cc];
    s[idx] = v;
  }
  for (int m = tid; m < p.L; m += DFT_THREADS) stw[m] = tw[m];
  __syncthreads();
  const int cc = tid & (CB - 1), g = tid / CB;
  if (b0 + cc >= p.B) return;
  for (int f = g; f < p.Jout; f += DFT_THREADS / CB) {
    F ar = F(0), ai = F(0);
    int m = 0;
    for (int j = 0; j < p.Jin; ++j) {
      const T2 v = s[j * CB + cc], w = stw[m];
      ar += v.x * w.x - v.y * w.y;
      ai += v.x * w.y + v.y * w.x;
      m += f;
      if (m >= p.L) m -= p.L;
    }
    T2 o;
    o.x = ar * scale;
    o.y = ai * scale;
    out[obase + f * p.oB + cc] = o;
  }
}

// The same pass on complex128 data with the sums in float-float arithmetic
// (pairs of FP32, ~48 bits) on the FP32 pipe: the transform of the displacement
// blocks, where FP64 issue (1/64 of FP32 on this GPU) would bound the prepare.
__global__ void __launch_bounds__(DFT_THREADS) axis_dft_ff_kernel(const double2* in, double2* out, AxisPass p,
                                                                  const double2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* s = reinterpret_cast<float4*>(smraw);  // [Jin][CB] (re hi, re lo, im hi, im lo)
  float4* stw = s + p.Jin * CB;                  // [L]
  const int line = blockIdx.y;
  const int a0 = line / p.n_a1, a1 = line - (line / p.n_a1) * p.n_a1;
  const long long b0 = (long long)blockIdx.x * CB;
  const long long ibase = a0 * p.is0 + a1 * p.is1 + b0, obase = a0 * p.os0 + a1 * p.os1 + b0;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < p.Jin * CB; idx += DFT_THREADS) {
    const int j = idx / CB, cc = idx - (idx / CB) * CB;
    double2 v = make_double2(0.0, 0.0);
    if (b0 + cc < p.B) v = in[ibase + j * p.iB + cc];
    const ff re = ff_from_double(v.x), im = ff_from_double(v.y);
    s[idx] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
  for (int m = tid; m < p.L; m += DFT_THREADS) {
    const ff c = ff_from_double(tw[m].x), sn = ff_from_double(tw[m].y);
    stw[m] = make_float4(c.hi, c.lo, sn.hi, sn.lo);
  }
  __syncthreads();
  const int cc = tid & (CB - 1), g = tid / CB;
  if (b0 + cc >= p.B) return;
  for (int f = g; f < p.Jout; f += DFT_THREADS / CB) {
    ff ar{0.f, 0.f}, ai{0.f, 0.f};
    int m = 0;
    for (int j = 0; j < p.Jin; ++j) {
      const float4 v = s[j * CB + cc], w = stw[m];
      const ff vr{v.x, v.y}, vi{v.z, v.w}, wr{w.x, w.y}, wi{w.z, w.w};
      ar = ff_add(ar, ff_sub(ff_mul(vr, wr), ff_mul(vi, wi)));
      ai = ff_add(ai, ff_add(ff_mul(vr, wi), ff_mul(vi, wr)));
      m += f;
      if (m >= p.L) m -= p.L;
    }
    out[obase + f * p.oB + cc] = make_double2(ff_to_double(ar), ff_to_double(ai));
  }
}

int run_pass_ff(const double2* in, double2* out, const AxisPass& p, const double2* tw, cudaStream_t st) {
  if (p.n_a0 * (long long)p.n_a1 > 65535 || p.B <= 0) return QAMS_EINVAL;
  const dim3 grid((unsigned)((p.B + CB - 1) / CB), (unsigned)(p.n_a0 * p.n_a1));
  const size_t smem = sizeof(float4) * ((size_t)p.Jin * CB + p.L);
  axis_dft_ff_kernel<<<grid, DFT_THREADS, smem, st>>>(in, out, p, tw);
  qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  return QAMS_OK;
}

// Frequency products, one CTA per frequency f: x[f][:, r0..r0+RC) is staged in
// shared memory transposed ([r][j], so consecutive lanes read consecutive
// words), then one warp per row i streams A[f][i][:] from HBM (U loads in flight
// per lane; complex64 rows as pairs of entries, 16 bytes per lane) against it,
//   y[f][i][r0 + r] = sum_j A[f][i][j] x[f][j][r0 + r],  r < RC.
constexpr int FP_THREADS = 256;

template <typename F>
__device__ __forceinline__ void cmac(F& ar, F& ai, F vx, F vy, F wx, F wy) {
  ar += vx * wx - vy * wy;
  ai += vx * wy + vy * wx;
}

template <typename T2, int RC>
__global__ void __launch_bounds__(FP_THREADS) freq_product_kernel(const T2* __restrict__ A, const T2* __restrict__ x,
                                                                  T2* __restrict__ y, int n, int R, int r0) {
  using F = typename Real<T2>::T;
  constexpr int U = RC >= 8 ? 2 : 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* xs = reinterpret_cast<T2*>(smraw);  // [RC][n]
  const long long f = blockIdx.x;
  const T2* xf = x + f * n * R + r0;
  for (int e = threadIdx.x; e < n * RC; e += FP_THREADS) {
    const int j = e / RC, r = e - (e / RC) * RC;
    xs[r * n + j] = xf[(long long)j * R + r];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < n; i += FP_THREADS / 32) {
    F ar[RC], ai[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) ar[r] = ai[r] = F(0);
    bool pairs = false;
    if constexpr (sizeof(T2) == sizeof(float2)) {
      pairs = n >= 256;  // long complex64 rows: two entries (16 bytes) per lane and load
      // n is even (an even number of azimuths), so rows are 16-byte aligned pairs
      const float4* a = reinterpret_cast<const float4*>(A + (f * n + i) * n);
      const int n2 = pairs ? n >> 1 : 0;
      for (int j0 = lane; j0 < n2; j0 += 32 * U) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = j0 + 32 * u < n2 ? a[j0 + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j2 = j0 + 32 * u;
          if (j2 >= n2) break;
#pragma unroll
          for (int r = 0; r < RC; ++r) {
            const float4 w = *reinterpret_cast<const float4*>(xs + r * n + 2 * j2);
            cmac(ar[r], ai[r], v[u].x, v[u].y, w.x, w.y);
            cmac(ar[r], ai[r], v[u].z, v[u].w, w.z, w.w);
          }
        }
      }
    }
    if (!pairs) {
      const T2* a = A + (f * n + i) * n;
      for (int j0 = lane; j0 < n; j0 += 32 * U) {
        T2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (j0 + 32 * u < n) {
            v[u] = a[j0 + 32 * u];
          } else {
            v[u].x = F(0);
            v[u].y = F(0);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + 32 * u;
          if (j >= n) break;
#pragma unroll
          for (int r = 0; r < RC; ++r) {
            const T2 w = xs[r * n + j];
            cmac(ar[r], ai[r], v[u].x, v[u].y, w.x, w.y);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RC; ++r)
      for (int o = 16; o > 0; o >>= 1) {
        ar[r] += __shfl_xor_sync(0xffffffffu, ar[r], o);
        ai[r] += __shfl_xor_sync(0xffffffffu, ai[r], o);
      }
    if (lane == 0) {
      T2* yv = y + (f * n + i) * R + r0;
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        T2 w;
        w.x = ar[r];
        w.y = ai[r];
        yv[r] = w;
      }
    }
  }
}

int grid_for(long long work) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (work + 255) / 256;
  return (int)std::max(1LL, std::min<long long>(want, (long long)sms * 16));
}

template <typename T2>
int run_pass(const T2* in, T2* out, const AxisPass& p, const T2* tw, double scale, cudaStream_t st) {
  if (p.n_a0 * (long long)p.n_a1 > 65535 || p.B <= 0) return QAMS_EINVAL;
  const dim3 grid((unsigned)((p.B + CB - 1) / CB), (unsigned)(p.n_a0 * p.n_a1));
  const size_t smem = sizeof(T2) * ((size_t)p.Jin * CB + p.L);
  axis_dft_kernel<T2><<<grid, DFT_THREADS, smem, st>>>(in, out, p, tw, (typename Real<T2>::T)scale);
  qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  return QAMS_OK;
}

// twiddle table of axis `ax`, direction `dir` (0 forward e^{-2 pi i m/L}, 1 inverse)
template <typename T2>
const T2* twiddles(const qams_ctx* c, int ax, int dir) {
  const size_t off64 = sizeof(double2) * MAXL * 6;
  if (sizeof(T2) == sizeof(double2)) return (const T2*)((const char*)c->lat.tw.p + sizeof(double2) * MAXL * (2 * ax + dir));
  return (const T2*)((const char*)c->lat.tw.p + off64 + sizeof(float2) * MAXL * (2 * ax + dir));
}

template <typename T2, int RC>
int launch_product(const T2* A, const T2* x, T2* y, long long F, int n, int R, int r0, cudaStream_t st) {
  const size_t smem = sizeof(T2) * (size_t)n * RC;
  if (smem > 48 * 1024) {
    if (smem > 227 * 1024) return QAMS_EINVAL;
    QAMS_CUDA(cudaFuncSetAttribute(freq_product_kernel<T2, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  }
  freq_product_kernel<T2, RC><<<(unsigned)F, FP_THREADS, smem, st>>>(A, x, y, n, R, r0);
  qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  return QAMS_OK;
}

template <typename T2>
int lattice_apply(qams_ctx* c, int R, const T2* sigma, T2* y, const T2* that, cudaStream_t st) {
  const LatticeState& L = c->lat;
  const int n = L.n;
  const long long nR = (long long)n * R;
  const int P0 = L.P[0], P1 = L.P[1], P2 = L.P[2], L0 = L.L[0], L1 = L.L[1], L2 = L.L[2];
  const long long F = (long long)L0 * L1 * L2;
  const size_t need = sizeof(T2) * (size_t)(F * nR);
  for (DeviceBuf* b : {&c->lat.work, &c->lat.work2})
    if (b->bytes < need) {
      qams_dev_free(c, b);
      int rc = qams_dev_alloc(c, b, need);
      if (rc) return rc;
    }
  T2* w = (T2*)c->lat.work.p;
  T2* w2 = (T2*)c->lat.work2.p;
  int rc;
  // forward: axis 2 (sigma [p][q][r] -> w [p][q][f2]), axis 1, axis 0 (in place)
  AxisPass p{nR, P0, P1, (long long)P1 * P2 * nR, (long long)P2 * nR, nR,
             (long long)L1 * L2 * nR, (long long)L2 * nR, nR, P2, L2, L2};
  if ((rc = run_pass<T2>(sigma, w, p, twiddles<T2>(c, 2, 0), 1.0, st))) return rc;
  p = AxisPass{(long long)L2 * nR, P0, 1, (long long)L1 * L2 * nR, 0, (long long)L2 * nR,
               (long long)L1 * L2 * nR, 0, (long long)L2 * nR, P1, L1, L1};
  if ((rc = run_pass<T2>(w, w, p, twiddles<T2>(c, 1, 0), 1.0, st))) return rc;
  p = AxisPass{(long long)L1 * L2 * nR, 1, 1, 0, 0, (long long)L1 * L2 * nR, 0, 0, (long long)L1 * L2 * nR, P0, L0, L0};
  if ((rc = run_pass<T2>(w, w, p, twiddles<T2>(c, 0, 0), 1.0, st))) return rc;
  // products per frequency
  const int pslot = sizeof(T2) == sizeof(double2) ? QAMS_PROF_LATTICE_PRODUCT64 : QAMS_PROF_LATTICE_PRODUCT32;
  // right-hand sides per product launch: staged columns fit in 200 KB of shared memory
  const int max_rc = (int)std::min<long long>(16, (200LL * 1024) / ((long long)n * (long long)sizeof(T2)));
  if (max_rc < 1) return QAMS_EINVAL;
  for (int r0 = 0; r0 < R;) {
    const int left = std::min(R - r0, max_rc);
    const int rcn = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    cudaEvent_t pe = qams_prof_begin(c, pslot, st);
    switch (rcn) {
      case 16: rc = launch_product<T2, 16>(that, w, w2, F, n, R, r0, st); break;
      case 8: rc = launch_product<T2, 8>(that, w, w2, F, n, R, r0, st); break;
      case 4: rc = launch_product<T2, 4>(that, w, w2, F, n, R, r0, st); break;
      case 2: rc = launch_product<T2, 2>(that, w, w2, F, n, R, r0, st); break;
      default: rc = launch_product<T2, 1>(that, w, w2, F, n, R, r0, st); break;
    }
    qams_prof_end(c, pslot, st, pe);
    if (rc) return rc;
    r0 += rcn;
  }
  // inverse: axis 0, axis 1 (in place, cropped), axis 2 (-> y, scaled)
  p = AxisPass{(long long)L1 * L2 * nR, 1, 1, 0, 0, (long long)L1 * L2 * nR, 0, 0, (long long)L1 * L2 * nR, L0, P0, L0};
  if ((rc = run_pass<T2>(w2, w2, p, twiddles<T2>(c, 0, 1), 1.0, st))) return rc;
  p = AxisPass{(long long)L2 * nR, P0, 1, (long long)L1 * L2 * nR, 0, (long long)L2 * nR,
               (long long)L1 * L2 * nR, 0, (long long)L2 * nR, L1, P1, L1};
  if ((rc = run_pass<T2>(w2, w2, p, twiddles<T2>(c, 1, 1), 1.0, st))) return rc;
  p = AxisPass{nR, P0, P1, (long long)L1 * L2 * nR, (long long)L2 * nR, nR,
               (long long)P1 * P2 * nR, (long long)P2 * nR, nR, L2, P2, L2};
  return run_pass<T2>(w2, y, p, twiddles<T2>(c, 2, 1), 1.0 / (double)F, st);
}

}  // namespace

int qams_lattice_prepare_launch(qams_ctx* c, cudaStream_t st) {
  LatticeState& L = c->lat;
  if (!L.on || !c->have_k) return QAMS_EINVAL;
  L.ready = false;
  const int n = L.n;
  const long long F = (long long)L.L[0] * L.L[1] * L.L[2];
  const long long entries = F * n * (long long)n;
  int rc;
  if (L.that64.bytes < sizeof(double2) * (size_t)entries) {
    qams_dev_free(c, &L.that64);
    if ((rc = qams_dev_alloc(c, &L.that64, sizeof(double2) * (size_t)entries))) return rc;
  }
  if (L.that32.bytes < sizeof(float2) * (size_t)entries) {
    qams_dev_free(c, &L.that32);
    if ((rc = qams_dev_alloc(c, &L.that32, sizeof(float2) * (size_t)entries))) return rc;
  }
  // twiddles: [axis][dir][MAXL] complex128, then the same in complex64
  if (!L.tw.p && (rc = qams_dev_alloc(c, &L.tw, (sizeof(double2) + sizeof(float2)) * MAXL * 6))) return rc;
  std::vector<double2> t64(MAXL * 6, make_double2(0.0, 0.0));
  std::vector<float2> t32(MAXL * 6, make_float2(0.f, 0.f));
  for (int ax = 0; ax < 3; ++ax)
    for (int dir = 0; dir < 2; ++dir)
      for (int m = 0; m < L.L[ax]; ++m) {
        const double th = 2.0 * M_PI * (double)m / (double)L.L[ax];
        const double2 v = make_double2(std::cos(th), dir == 0 ? -std::sin(th) : std::sin(th));
        t64[MAXL * (2 * ax + dir) + m] = v;
        t32[MAXL * (2 * ax + dir) + m] = make_float2((float)v.x, (float)v.y);
      }
  QAMS_CUDA(cudaMemcpyAsync(L.tw.p, t64.data(), sizeof(double2) * MAXL * 6, cudaMemcpyHostToDevice, st));
  QAMS_CUDA(cudaMemcpyAsync((char*)L.tw.p + sizeof(double2) * MAXL * 6, t32.data(), sizeof(float2) * MAXL * 6,
                            cudaMemcpyHostToDevice, st));
  const double* A = L.basis;
  double2* T = (double2*)L.that64.p;
  lattice_blocks_kernel<<<grid_for(entries), 256, 0, st>>>(
      (const qd4*)c->x64.p, (const qd4*)c->n64.p, (const qd4*)c->centers.p, n, L.L[0], L.L[1], L.L[2], L.P[0],
      L.P[1], L.P[2], make_double3(A[0], A[1], A[2]), make_double3(A[3], A[4], A[5]),
      make_double3(A[6], A[7], A[8]), c->k, c->eta, T);
  qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  // forward DFT of the blocks along axes 2, 1, 0 (in place, all residues)
  const long long nn = (long long)n * n;
  const int L0 = L.L[0], L1 = L.L[1], L2 = L.L[2];
  AxisPass p{nn, L0, L1, (long long)L1 * L2 * nn, (long long)L2 * nn, nn,
             (long long)L1 * L2 * nn, (long long)L2 * nn, nn, L2, L2, L2};
  if ((rc = run_pass_ff(T, T, p, twiddles<double2>(c, 2, 0), st))) return rc;
  p = AxisPass{(long long)L2 * nn, L0, 1, (long long)L1 * L2 * nn, 0, (long long)L2 * nn,
               (long long)L1 * L2 * nn, 0, (long long)L2 * nn, L1, L1, L1};
  if ((rc = run_pass_ff(T, T, p, twiddles<double2>(c, 1, 0), st))) return rc;
  p = AxisPass{(long long)L1 * L2 * nn, 1, 1, 0, 0, (long long)L1 * L2 * nn, 0, 0, (long long)L1 * L2 * nn, L0, L0, L0};
  if ((rc = run_pass_ff(T, T, p, twiddles<double2>(c, 0, 0), st))) return rc;
  round_kernel<<<grid_for(entries), 256, 0, st>>>(T, (float2*)L.that32.p, entries);
  qams_count_launch();
  QAMS_CUDA(cudaGetLastError());
  L.ready = true;
  return QAMS_OK;
}

void qams_lattice_reset(qams_ctx* c) {
  for (DeviceBuf* b : {&c->lat.that64, &c->lat.that32, &c->lat.tw, &c->lat.work, &c->lat.work2}) qams_dev_free(c, b);
  c->lat.on = c->lat.ready = false;
}

int qams_lattice_pairsum(qams_ctx* c, int R, const void* sigma, void* y, int precision, cudaStream_t st) {
  cudaEvent_t pe = qams_prof_begin(c, QAMS_PROF_PAIRSUM_LATTICE, st);
  int rc;
  if (precision == QAMS_PREC_FP32)
    rc = lattice_apply<float2>(c, R, (const float2*)sigma, (float2*)y, (const float2*)c->lat.that32.p, st);
  else
    rc = lattice_apply<double2>(c, R, (const double2*)sigma, (double2*)y, (const double2*)c->lat.that64.p, st);
  qams_prof_end(c, QAMS_PROF_PAIRSUM_LATTICE, st, pe);
  return rc;
}
