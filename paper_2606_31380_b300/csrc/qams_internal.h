// Internal state of a libqams context (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qams.h"

// 32-byte aligned double4 (one 256-bit load); cudaMalloc and the shared
// arrays below satisfy the alignment.
typedef double4_32a qd4;

#define QAMS_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      qams_internal_last_cuda_error(e_, #call);          \
      return QAMS_ECUDA;                                 \
    }                                                    \
  } while (0)

void qams_internal_last_cuda_error(cudaError_t e, const char* what);

// Process-wide count of kernel launches made by the library.
void qams_count_launch(int n = 1);

// A validated copy of one body descriptor.  The arrays live in the vectors;
// d's own array pointers are cleared, so only the vectors are read.
struct BodyCopy {
  qams_body_desc d{};
  std::vector<double> a, b;     // kind 0: profile Fourier modes (n_modes each)
  std::vector<double> series;   // kind 1: [4][n_terms][3] (omega, A, B)
  std::vector<double> breaks;   // n_panels + 1 panel breakpoints (uniform if not given)
  double radius = 0.0;          // ball about the centre that holds the body
  double rmax = 0.0;            // bound on the ring radius r(s)
};

// Validates `src` and fills `out`; QAMS_OK or QAMS_EINVAL (the conditions of
// qams_body_desc).
int qams_copy_body(const qams_body_desc& src, BodyCopy* out);

// The descriptor with its array pointers aimed at the copy's vectors (valid
// while `bc` lives and is not moved).
qams_body_desc qams_desc_view(const BodyCopy& bc);

// The reference shape and discretisation of a body (everything but its
// rotation and centre): congruent bodies have equal keys and one self block.
std::string qams_shape_key(const BodyCopy& bc);

struct BodyHost : BodyCopy {
  long long offset = 0;  // first node
  int n = 0;             // nodes
};

// Nearest point of body b (world nodes hx_body [n][3]) to the world point x:
// surface parameters (s, th) and panel, distance, and v = x - y(s, th) in the
// frame the self-block kernel takes target offsets in (arc axis: (e1, e2,
// e3)(s); ring-series shapes: the body frame).
void qams_nearest_point(const BodyHost& b, const double* hx_body, const double x[3], double* s, double* th,
                        int* panel, double* dist, double* ds, double v[3]);

// One target tile of the pair sum: up to TILE consecutive nodes of one body.
struct TargetTile {
  int body;
  int count;
  long long start;
};

// A contiguous range of source bodies handled by one grid row.
struct SourceSplit {
  int begin, end;
};

struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// First-fit allocator over [0, size) with coalescing of freed neighbours;
// offsets and lengths are multiples of 256 bytes.  Thread-safe.
class FitAlloc {
 public:
  void init(size_t size);
  long long alloc(size_t bytes);  // offset, or -1 when no free range fits
  void release(size_t off, size_t bytes);
  size_t size() const { return size_; }
  size_t largest_free();

 private:
  size_t size_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  std::mutex mu_;
};

// Device memory region handed to a context: qams_dev_alloc/free draw from
// it instead of cudaMalloc/cudaFree (a serving slot's reservation).
struct DevArena {
  char* base = nullptr;
  FitAlloc fa;
};

// Per-launch device times of the hot kernels (CUDA events on the launching
// stream), recorded while profiling is switched on (qams_profile_enable).
struct ProfSlot {
  long long launches = 0;
  double ms = 0.0;
  std::vector<cudaEvent_t> pending;  // start/stop pairs not yet read
};

// A contiguous run of equal-size bodies: one tensor map per operand in the
// tensor-core block product.
struct TcGroup {
  int first, nb, n;    // first body, bodies, nodes per body
  long long node0;     // first node of the first body
  long long elem0;     // first complex block entry of the first body
};

// A regular lattice of one rigid shape (qams_set_lattice): bodies
// (p Q + q) R + r at c_0 + p a0 + q a1 + r a2, all with one rotation.  The
// pair sum then runs through the circulant embedding of lattice.cu.
struct LatticeState {
  bool on = false;           // bodies were set by qams_set_lattice
  bool use = true;           // QAMS_OPT_LATTICE
  bool ready = false;        // transformed blocks built for the current wavenumber
  int P[3] = {1, 1, 1};      // bodies along each lattice vector
  int L[3] = {1, 1, 1};      // circulant periods 2 P - 1
  double basis[9] = {};      // lattice vectors a0, a1, a2 (rows)
  int n = 0;                 // nodes per body
  DeviceBuf that64, that32;  // [L0 L1 L2][n][n] transformed displacement blocks
  DeviceBuf tw;              // twiddle tables
  DeviceBuf work, work2;     // [L0 L1 L2][n][R] transform workspaces
};

struct qams_ctx {
  int device = 0;
  size_t budget = 0;
  size_t allocated = 0;
  std::vector<BodyHost> bodies;
  long long N = 0;
  double k = 0.0, eta = 1.0;
  bool have_k = false;
  const int* cancel = nullptr;  // set by the server: checked between GMRES restart cycles
  DevArena* arena = nullptr;    // set by the server: device memory comes from the request's reservation

  // host node tables (FP64, world frame)
  std::vector<double> hx, hn, hw, hj;  // [N][3], [N][3], [N], [N] (|J|)

  // device node tables
  DeviceBuf x64;     // double4 [N]: world position, w in .w
  DeviceBuf n64;     // double4 [N]: world normal
  DeviceBuf x32;     // float4  [N]: body-local position x - c_b, w in .w
  DeviceBuf n32;     // float4  [N]: world normal
  DeviceBuf x32lo;   // float4  [N]: x - c_b - x32 (float-float tails)
  DeviceBuf n32lo;   // float4  [N]: normal - n32
  DeviceBuf centers; // double4 [nb]
  DeviceBuf boff;    // long long [nb+1]
  DeviceBuf jac64;   // double [N]: |J| at the nodes

  // congruent bodies share a self block (Sec. 4: D_tt computed once for
  // identical bodies): body_class[b] = index into class_rep, the first body
  // of each class; class_blk[k] = first block entry of class k
  std::vector<int> body_class, class_rep;
  std::vector<long long> class_blk;

  // self blocks (row-major n_b x n_b per class of congruent bodies, back to back)
  DeviceBuf blocks64;  // complex128
  DeviceBuf blocks32;  // complex64 copy for the FP32 path
  DeviceBuf blk_off;   // long long [nb+1]: first entry of each block
  long long block_entries = 0;
  bool assembled = false;
  long long asm_counts[2] = {0, 0};  // outer quadrature nodes of the last assembly: modal, far

  // block-Jacobi preconditioner: inverses of the self blocks (same layout)
  DeviceBuf pinv32;  // complex64, computed
  DeviceBuf pinv64;  // complex128 widening of pinv32 (an exact linear map for the FP64 path)
  bool have_precond = false;

  // apply workspaces
  DeviceBuf ws_sigma, ws_y;

  // tensor-core block products (tc_block.cu): FP16 hi/lo split copies of the
  // complex64 blocks, B-tile workspace, column maxima, timeout flag
  std::vector<TcGroup> tc_groups;
  DeviceBuf tc_blk_hi, tc_blk_lo, tc_pinv_hi, tc_pinv_lo, tc_bt, tc_amax, tc_err;
  bool tc_blk_ok = false, tc_pinv_ok = false;
  int tc_bt_R = -1;
  int tc_min_r = 8;       // right-hand sides from which the FP32 block products use the tensor cores
  int tc_pair_min_r = 8;  // ... and from which the FP32 pair sum accumulates on them

  // launch timing of the hot kernels (QAMS_PROF_* slots of qams.h)
  bool prof = false;
  ProfSlot prof_slots[QAMS_PROF_COUNT];

  // pair-sum launch tables
  std::vector<TargetTile> tiles;
  std::vector<TargetTile> tiles2;  // tiles of 2 TILE targets (two per thread)
  DeviceBuf d_tiles2;
  int ps_tt = 1;                   // targets per thread of the CUDA-core FP32 pair sum (1 or 2)
  std::vector<SourceSplit> splits;
  DeviceBuf d_tiles, d_splits;
  DeviceBuf partial;  // [splits][N][rc] partial sums (complex, largest precision)

  LatticeState lat;

  // near-field correction of qams_field (QAMS_OPT_NEAR_FIELD): points closer
  // than near_factor node spacings to a body get the product-integration rows
  int near_factor = 6;
  long long near_pairs = 0;  // (point, body) pairs corrected by the last qams_field

  ~qams_ctx();
};

// Bracket one kernel launch with events when profiling is on (slot = QAMS_PROF_*).
cudaEvent_t qams_prof_begin(qams_ctx* c, int slot, cudaStream_t st);
void qams_prof_end(qams_ctx* c, int slot, cudaStream_t st, cudaEvent_t start);

int qams_dev_alloc(qams_ctx* c, DeviceBuf* b, size_t bytes);
void qams_dev_free(qams_ctx* c, DeviceBuf* b);

// geometry.cpp
int qams_build_nodes(qams_ctx* c);
void qams_gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// pairsum.cu
int qams_pairsum_launch(qams_ctx* c, int R, const void* sigma, void* y, int precision, cudaStream_t st);
int qams_pairsum_prepare(qams_ctx* c);
int qams_pairsum_set_splits(qams_ctx* c, int S);
int qams_pairsum_default_splits(const qams_ctx* c, int mult);

// An off-surface target near one body (the near-field rows of selfblock.cu):
// x = y(s, th) + v with v = nu n^(s, th), the unit normal's components taken in
// the target ring's frame (e1, e2, e3)(s) for arc-axis bodies and in the
// body frame for ring-series bodies.
struct NearTarget {
  int cls;          // class of congruent bodies (index into class_rep)
  int panel;        // panel holding s
  double s, th;     // closest surface point
  double ds;        // distance to the surface in units of s (|x - y| / |d_s y|)
  double v[3];      // offset x - y(s, th)
  double x[3];      // world position (for the smooth-rule subtraction)
  long long node0;  // first node of the body
  long long row;    // first entry of the target's row in the output
  int m;            // target point (row of the field output)
  int n;            // nodes of the body (row length)
};

// selfblock.cu
int qams_assemble_launch(qams_ctx* c, cudaStream_t st);
int qams_near_rows_launch(qams_ctx* c, const NearTarget* targets, long long n, double r_extra, double2* rows,
                          cudaStream_t st);

// blockops.cu
int qams_blocks_to_fp32(qams_ctx* c, cudaStream_t st);
int qams_block_apply(qams_ctx* c, int R, const void* x, void* y, int precision, bool accumulate, cudaStream_t st);
int qams_apply_launch(qams_ctx* c, int R, const void* x, void* y, int precision, cudaStream_t st);
int qams_block_apply_ptr(qams_ctx* c, const void* blocks, int R, const void* x, void* y, int precision,
                         bool accumulate, cudaStream_t st);

// precond.cu
int qams_precond_launch(qams_ctx* c, cudaStream_t st);

// tc_block.cu
int qams_tc_groups(qams_ctx* c);
int qams_tc_prepare(qams_ctx* c, int which, cudaStream_t st);
int qams_tc_block_apply(qams_ctx* c, int which, int R, const void* x, void* y, bool accumulate, cudaStream_t st);
int qams_tc_check(qams_ctx* c, cudaStream_t st);

// tc_pairsum.cu
int qams_pairsum_tc_launch(qams_ctx* c, int R, const void* sigma, void* out, long long split_stride, int out_ld,
                           cudaStream_t st);

// lattice.cu
int qams_lattice_prepare_launch(qams_ctx* c, cudaStream_t st);
int qams_lattice_pairsum(qams_ctx* c, int R, const void* sigma, void* y, int precision, cudaStream_t st);
void qams_lattice_reset(qams_ctx* c);

// fields.cu
int qams_incident_launch(qams_ctx* c, int R, const double* dirs_host, void* rhs, cudaStream_t st);
int qams_field_launch(qams_ctx* c, int R, const void* mu, int M, const double* pts_host, void* u,
                      cudaStream_t st);

// nearfield.cu: adds the near-field rows' contributions to a smooth-rule field
int qams_near_correction(qams_ctx* c, int R, const void* mu, int M, const double* pts_host, void* u,
                         cudaStream_t st);
int qams_farfield_launch(qams_ctx* c, int R, const void* mu, int M, const double* dirs_host, void* uinf,
                         cudaStream_t st);
