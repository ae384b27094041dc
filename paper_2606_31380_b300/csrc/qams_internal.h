// Internal state of a libqams context (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
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

struct BodyHost : BodyCopy {
  long long offset = 0;  // first node
  int n = 0;             // nodes
};

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

struct qams_ctx {
  int device = 0;
  size_t budget = 0;
  size_t allocated = 0;
  std::vector<BodyHost> bodies;
  long long N = 0;
  double k = 0.0, eta = 1.0;
  bool have_k = false;
  const int* cancel = nullptr;  // set by the server: checked between GMRES restart cycles

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

  // self blocks (row-major n_b x n_b per body, bodies back to back)
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

  // pair-sum launch tables
  std::vector<TargetTile> tiles;
  std::vector<SourceSplit> splits;
  DeviceBuf d_tiles, d_splits;
  DeviceBuf partial;  // [splits][N][rc] partial sums (complex, largest precision)

  ~qams_ctx();
};

int qams_dev_alloc(qams_ctx* c, DeviceBuf* b, size_t bytes);
void qams_dev_free(qams_ctx* c, DeviceBuf* b);

// geometry.cpp
int qams_build_nodes(qams_ctx* c);
void qams_gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// pairsum.cu
int qams_pairsum_launch(qams_ctx* c, int R, const void* sigma, void* y, int precision, cudaStream_t st);
int qams_pairsum_prepare(qams_ctx* c);

// selfblock.cu
int qams_assemble_launch(qams_ctx* c, cudaStream_t st);

// blockops.cu
int qams_blocks_to_fp32(qams_ctx* c, cudaStream_t st);
int qams_block_apply(qams_ctx* c, int R, const void* x, void* y, int precision, bool accumulate, cudaStream_t st);
int qams_apply_launch(qams_ctx* c, int R, const void* x, void* y, int precision, cudaStream_t st);
int qams_block_apply_ptr(qams_ctx* c, const void* blocks, int R, const void* x, void* y, int precision,
                         bool accumulate, cudaStream_t st);

// precond.cu
int qams_precond_launch(qams_ctx* c, cudaStream_t st);

// fields.cu
int qams_incident_launch(qams_ctx* c, int R, const double* dirs_host, void* rhs, cudaStream_t st);
int qams_field_launch(qams_ctx* c, int R, const void* mu, int M, const double* pts_host, void* u,
                      cudaStream_t st);
int qams_farfield_launch(qams_ctx* c, int R, const void* mu, int M, const double* dirs_host, void* uinf,
                         cudaStream_t st);
