/*
 * qams.h -- C ABI of the B300 multi-body Nystrom operator library (libqams).
 *
 * Problem (Sec. 2, Sec. 4): sound-soft scattering by several bodies, each a
 * rigid motion x = R x0 + c (Sec. 6.5) of a quasi-axisymmetric reference
 * shape (Eq. para_quasi, generalised to a planar-arc axis), solved with the
 * combined-layer representation u = (D - i eta S)[mu] (Sec. 2, Remark) as the
 * block system (Eq. linearsys)
 *
 *     (1/2 I + D - i eta S) mu = -u^inc .
 *
 * Conventions
 *  - Every call returns int: QAMS_OK (0) or a negative QAMS_E* code;
 *    qams_strerror() names it.  On error nothing has been launched unless
 *    the code is QAMS_ECUDA.
 *  - "_dev" pointers are caller-owned device buffers on the context's
 *    device; "_host" pointers are caller-owned host buffers that are only
 *    read (or written) during the call.
 *  - Unknown vectors are [N][R] interleaved complex, node-major with the R
 *    right-hand sides innermost: complex128 (double re, im) for
 *    QAMS_PREC_FP64, complex64 (float re, im) for QAMS_PREC_FP32.
 *    Node order: body -> panel -> Gauss-Legendre node -> azimuth (theta
 *    fastest), the order of Eq. sx; qams_get_nodes() exposes it.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default).
 *    Calls enqueue work on it and do not synchronise the device, except
 *    where a call is documented as blocking.
 *  - The library owns and frees (qams_destroy) its node tables, self
 *    blocks, preconditioner and workspaces.  Host descriptors are copied.
 */
#ifndef QAMS_H
#define QAMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  QAMS_OK = 0,
  QAMS_EINVAL = -1,     /* bad argument or call order                     */
  QAMS_EBUDGET = -2,    /* footprint above the context's HBM budget       */
  QAMS_EGEOM = -3,      /* bodies overlap / closer than the minimum gap  */
  QAMS_ENOCONV = -4,    /* iteration limit reached; stats still filled    */
  QAMS_ENUMERIC = -5,   /* NaN/Inf in a residual                          */
  QAMS_ETIMEOUT = -6,   /* a bounded device wait gave up                  */
  QAMS_ECANCELLED = -7, /* cancelled between restart cycles               */
  QAMS_ECUDA = -8,      /* a CUDA runtime call failed                     */
  QAMS_ESCRATCH = -9,   /* problem too large for the static scratch       */
  QAMS_EAGAIN = -10     /* request not finished yet (qams_poll)           */
};

/* Arithmetic of the operator calls.  QAMS_PREC_FF: complex128 vectors and
 * FP64 block products, with the pair sum in float-float arithmetic (pairs of
 * FP32 numbers, ~48 bits: relative error ~1e-14 per pair) -- FP64-accurate
 * results without B300's slow FP64 pipe.  Used by qams_pairsum and qams_apply. */
enum { QAMS_PREC_FP64 = 0, QAMS_PREC_FP32 = 1, QAMS_PREC_FF = 2 };

typedef struct qams_ctx qams_ctx; /* opaque, library-owned */

/* One body (all FP64, host memory, copied at qams_set_bodies).
 *
 * profile_kind 0 -- reference shape on a planar-arc axis, s in [-pi/2, pi/2],
 * u = (1 + sin s)/2, l = L (u - 1/2):
 *   rho(u) = base_radius (1 + sum_m mode_cos[m-1] cos 2 pi m u + mode_sin[m-1] sin 2 pi m u)
 *   r(s)   = rho(u) cos s          (closed at both poles)
 *   axis   = planar circular arc of curvature `curvature` and arclength L
 *            with a rotation-minimising frame; 0 = straight (a body of
 *            revolution);
 *   y(s,theta) = gamma(l) + r(s) (cos theta e1(l) + sin theta e2).
 *
 * profile_kind 1 -- horizontal rings with a moving centre, the family of the
 * paper's own shapes (Eq. para_quasi; Eqs. quasiwave and geometries):
 *   y(s,theta) = (x_c(s) + r(s) cos theta, y_c(s) + r(s) sin theta, z(s)),
 * each of x_c, y_c, z, r = sum_j A_j cos(omega_j s) + B_j sin(omega_j s),
 * given in `series` as [4][n_terms][3] = (omega, A, B) (pad with zeros).
 * r must be positive inside (-pi/2, pi/2) and vanish at both ends, z must
 * increase.  base_radius, modes, axis_length and curvature are ignored.
 *
 * Discretisation (Sec. 3.1): n_panels panels in s -- uniform, or with the
 * n_panels + 1 increasing breakpoints `panel_breaks` from -pi/2 to pi/2
 * (e.g. dyadic refinement toward the poles, Sec. 6.1) -- with `order`
 * Gauss-Legendre nodes each, and n_theta = 2N equispaced azimuths.
 * Panels within one index of the target's panel are integrated with the
 * modal product rules, the others with the plain rule (Eq. sx).
 *
 * QAMS_EINVAL from qams_set_bodies: sizes out of range, a profile that is
 * not positive (kind 0: sum of |modes| >= 1 or kappa rho >= 1; kind 1: r <= 0
 * inside, r != 0 at an end, z not increasing), n_terms outside 1..8, or
 * breakpoints that are not increasing from -pi/2 to pi/2. */
typedef struct {
  int n_panels, order, n_theta;
  double base_radius;
  int n_modes; /* <= 8; mode_cos / mode_sin each hold n_modes values (NULL = zeros) */
  const double* mode_cos;
  const double* mode_sin;
  double axis_length, curvature;
  double rotation[9]; /* row-major R, world = R * local + center */
  double center[3];
  int profile_kind;           /* 0 or 1, see above */
  int n_terms;                /* kind 1: terms per function, 1..8 */
  const double* series;       /* kind 1: [4][n_terms][3]; ignored for kind 0 */
  const double* panel_breaks; /* n_panels + 1 values, or NULL = uniform panels */
} qams_body_desc;

const char* qams_strerror(int code);

/* Number of CUDA kernels the library has launched in this process (all
 * contexts); lets callers attribute device work to the library. */
long long qams_kernel_launches(void);

/* Launch timing of the hot kernels (a measurement hook; the paper has no
 * counterpart).  While enabled, every launch of the kernels below is
 * bracketed by two CUDA events on the stream it is launched on; read
 * returns the number of launches timed and their summed device time since
 * the last enable (blocking: waits for the recorded events).  Enabling
 * again clears the sums; disabling stops recording.
 * Errors: QAMS_EINVAL (NULL context or pointer, slot out of range), QAMS_ECUDA. */
enum {
  QAMS_PROF_PAIRSUM_FP32 = 0, /* inter-body pair sum, FP32 */
  QAMS_PROF_PAIRSUM_FF = 1,   /* inter-body pair sum, float-float */
  QAMS_PROF_PAIRSUM_FP64 = 2, /* inter-body pair sum, FP64 */
  QAMS_PROF_BLOCK_FP32 = 3,   /* self-block / preconditioner products, complex64 */
  QAMS_PROF_BLOCK_FP64 = 4,   /* self-block / preconditioner products, complex128 */
  QAMS_PROF_ASSEMBLY = 5,     /* self-block assembly kernel */
  QAMS_PROF_BLOCK_TC = 6,     /* self-block / preconditioner products on the tensor cores */
  QAMS_PROF_PAIRSUM_TC = 7,   /* FP32 pair sum with its accumulation on the tensor cores */
  QAMS_PROF_PAIRSUM_LATTICE = 8, /* pair sum of a lattice through the circulant embedding (all passes) */
  QAMS_PROF_LATTICE_PRODUCT32 = 9,  /* its per-frequency products, complex64 */
  QAMS_PROF_LATTICE_PRODUCT64 = 10, /* its per-frequency products, complex128 */
  QAMS_PROF_COUNT = 11
};
int qams_profile_enable(qams_ctx* ctx, int on);
int qams_profile_read(qams_ctx* ctx, int slot, long long* launches, double* total_ms);

/* Tuning options of a context (no counterpart in the paper: they choose
 * between equivalent kernels and launch shapes, never the arithmetic's
 * result beyond rounding).
 *   QAMS_OPT_TC_MIN_RHS  FP32 self-block / preconditioner products run on
 *                        the tensor cores when R >= value (default 8;
 *                        17 = never).
 *   QAMS_OPT_TC_PAIR_MIN_RHS  the FP32 pair sum accumulates on the tensor
 *                        cores when R >= value (default 8; 17 = never).
 *   QAMS_OPT_PAIR_TARGETS  targets per thread of the CUDA-core FP32 pair sum,
 *                        1 (default) or 2 (each staged source serves two).
 *   QAMS_OPT_NEAR_FIELD  qams_field's near-field correction for points within
 *                        value node spacings of a body (0 = smooth rule
 *                        only; 1..64; default 6).
 *   QAMS_OPT_LATTICE     on a context set by qams_set_lattice: 1 (default)
 *                        applies the pair sum through the circulant
 *                        embedding once qams_lattice_prepare (or
 *                        qams_assemble) has built it; 0 = the direct pair
 *                        sum over all node pairs.
 * Errors: QAMS_EINVAL (NULL context or pointer, unknown key, value out of
 * range). */
enum { QAMS_OPT_TC_MIN_RHS = 0, QAMS_OPT_TC_PAIR_MIN_RHS = 1, QAMS_OPT_PAIR_TARGETS = 2, QAMS_OPT_LATTICE = 3,
       QAMS_OPT_NEAR_FIELD = 4 };
int qams_set_option(qams_ctx* ctx, int key, long long value);
int qams_get_option(const qams_ctx* ctx, int key, long long* value);

/* Launch-shape autotuner (no counterpart in the paper; every candidate
 * computes the same sums up to rounding).  For R (1..16) right-hand sides on
 * the context's bodies it times, with CUDA events on `stream`, the FP32 pair
 * sum with its multiply-accumulate on the CUDA cores (one or two targets per
 * thread) or on the tensor cores, for each distinct source-split count
 * (about 1, 2, 4, 8 and 16 CTAs per SM), and, after qams_assemble and for
 * R >= 8, the FP32 self-block product on the CUDA cores or on the tensor
 * cores.  The fastest choices are installed in the context (split tables;
 * QAMS_OPT_PAIR_TARGETS, QAMS_OPT_TC_PAIR_MIN_RHS and QAMS_OPT_TC_MIN_RHS set so
 * that R takes them) and cached for the process under (device, body sizes,
 * R): a later call for the same shape installs the cached choice without
 * timing (cached = 1).  Needs the bodies and the wavenumber.  Blocking.
 * Errors: QAMS_EINVAL, QAMS_EBUDGET (scratch vectors), QAMS_ETIMEOUT,
 * QAMS_ECUDA. */
typedef struct {
  int R;
  int pair_tc;      /* 1: pair sum on the tensor cores */
  int pair_targets; /* CUDA-core pair sum: targets per thread (1 or 2) */
  int pair_splits;  /* source splits (grid rows) of the pair sum */
  int block_tc;     /* 1: block products on the tensor cores; -1: not timed (no assembly) */
  double pair_ms;   /* device time of one FP32 pair sum with the choice */
  double block_ms;  /* device time of one FP32 self-block product with the choice */
  int cached;       /* 1: taken from the process-wide cache */
} qams_tuning;
int qams_autotune(qams_ctx* ctx, int R, qams_tuning* out, void* stream);

/* Self-test of the bounded device waits (no counterpart in the paper).  The
 * tensor-core kernels wait on mbarriers with a bound of about 2^31 clock
 * cycles; a wait that gives up sets an error flag, the kernel drains what it
 * issued and returns, and the call reports QAMS_ETIMEOUT.  This call
 * launches one CTA that waits in the same way, for at most `cycles` (1 ..
 * 2^32) clock cycles, on an mbarrier that nothing completes: it returns
 * QAMS_ETIMEOUT (the expected result) and the device stays usable.
 * Blocking.  Errors: QAMS_EINVAL, QAMS_ECUDA. */
int qams_selftest_timeout(int cuda_device, long long cycles, void* stream);

/* Create a context on CUDA device `cuda_device`.  hbm_budget_bytes = 0 means
 * no limit.  Errors: QAMS_EINVAL, QAMS_ECUDA. */
int qams_create(qams_ctx** out, int cuda_device, size_t hbm_budget_bytes);
void qams_destroy(qams_ctx* ctx);

/* Bodies and their Nystrom nodes (Sec. 3.1, Eq. sx).  Builds positions,
 * unit outward normals and weights w = |J| (pi/N) omega in FP64 on the host
 * and uploads them.  Rejects (QAMS_EGEOM) bodies whose bounding balls come
 * closer than min_gap (Sec. 4 separation assumption).  Blocking.
 * Errors: QAMS_EINVAL (n_bodies < 1, n_theta odd or < 2, order < 1,
 * n_panels < 1, n_modes > 8), QAMS_EGEOM, QAMS_EBUDGET, QAMS_ECUDA. */
int qams_set_bodies(qams_ctx* ctx, int n_bodies, const qams_body_desc* bodies, double min_gap);

/* A regular lattice of one rigid shape (Sec. 4, regular P x Q x R arrays
 * with uniform spacing; Table tab:multibody_cubic).  Sets the context's
 * bodies to dims[0] dims[1] dims[2] copies of *body (same reference shape,
 * same rotation) with centres body->center + p a0 + q a1 + r a2, where a0,
 * a1, a2 are the rows of basis (row-major 3x3, host) and body index
 * (p dims[1] + q) dims[2] + r, so node order is p, q, r, then the body's own
 * order.  The inter-body block of bodies t and s then depends only on
 * their displacement d = (p_t - p_s, q_t - q_s, r_t - r_s) (the block
 * Toeplitz structure of Sec. 4).  qams_lattice_prepare (called by
 * qams_assemble) forms the (2 dims[0] - 1)(2 dims[1] - 1)(2 dims[2] - 1)
 * distinct blocks T(d)[i][j] = K(x~_i + d.A, y~_j) (values in FP64), embeds
 * them in a circulant of those periods and transforms them by the 3-D
 * discrete Fourier transform (float-float sums, ~1e-14 relative); from then
 * on qams_pairsum (and so qams_apply and qams_solve) computes the same sums
 * as the direct pair sum by per-frequency n x n products: complex64 blocks
 * and FP32 arithmetic for QAMS_PREC_FP32, complex128 blocks and FP64
 * arithmetic for QAMS_PREC_FF and QAMS_PREC_FP64 (no phase split is
 * needed).  Library-owned device memory: (16 + 8) n^2 prod(2 dims - 1)
 * bytes of blocks plus two [prod(2 dims - 1)][n][R] complex workspaces
 * sized at the first apply.  A later qams_set_bodies ends the lattice mode.
 * Checks and errors as qams_set_bodies; QAMS_EINVAL also for dims outside
 * 1..32 or a non-finite basis.  Blocking. */
int qams_set_lattice(qams_ctx* ctx, const qams_body_desc* body, const int dims_host[3], const double basis_host[9],
                     double min_gap);

/* Build the transformed displacement blocks of a lattice context for the
 * current wavenumber (see qams_set_lattice); qams_assemble calls it when
 * QAMS_OPT_LATTICE is on.  A new wavenumber invalidates them.  Blocking.
 * Errors: QAMS_EINVAL (not a lattice context, no wavenumber), QAMS_EBUDGET,
 * QAMS_ECUDA. */
int qams_lattice_prepare(qams_ctx* ctx, void* stream);

/* N (total nodes) and the first node of every body (n_bodies+1 offsets). */
int qams_node_count(const qams_ctx* ctx, long long* n_nodes);
int qams_body_offsets(const qams_ctx* ctx, long long* offsets_host);

/* Copy node tables to the host: x_host, n_host are [N][3], w_host is [N].
 * Any pointer may be NULL.  Blocking. */
int qams_get_nodes(const qams_ctx* ctx, double* x_host, double* n_host, double* w_host);

/* The Nystrom nodes of one body (Eq. para_quasi, Sec. 3.1, Eq. sx) without a
 * context or device: x_host, n_host [n][3] world positions and unit normals,
 * w_host [n] weights |J| (2 pi / n_theta) omega, n = n_panels order n_theta,
 * in the node order of qams_get_nodes.  Host only; any output may be NULL.
 * Errors: QAMS_EINVAL (the descriptor conditions of qams_set_bodies). */
int qams_body_nodes(const qams_body_desc* body, double* x_host, double* n_host, double* w_host);

/* The nearest surface point of one body to the world point x_host[3], as
 * qams_field's near-field correction finds it (Levenberg-Marquardt on
 * (s, theta) from the nearest node, a step taken only when it brings the
 * surface point closer): the surface parameters s_out in [-pi/2, pi/2]
 * (kept 1e-7 inside the poles) and theta_out in [0, 2 pi), and the distance.
 * Host only, no context or device.  Errors: QAMS_EINVAL (NULL pointers, the
 * descriptor conditions of qams_set_bodies). */
int qams_nearest_surface_point(const qams_body_desc* body, const double* x_host, double* s_out, double* theta_out,
                               double* dist_out);

/* Wavenumber k > 0 and combined-layer coupling eta (0 = pure double layer,
 * Eq. multi-double; 1 = the default of the Sec. 2 Remark). */
int qams_set_wavenumber(qams_ctx* ctx, double k, double eta);

/* Inter-body smooth sum (Eq. multi2part, the off-diagonal blocks of Eq.
 * linearsys applied matrix-free):
 *   y_t = sum_{s on other bodies} K(x_t, y_s) sigma_s,
 *   K   = e^{ik rho}/(4 pi rho) [(ik/rho - 1/rho^2) n_s.(y_s - x_t) - i eta],
 * sigma = w mu with the quadrature weights already folded in.  sigma_dev and
 * y_dev are [N][R] complex of the given precision; y is overwritten.
 * QAMS_PREC_FP32 evaluates each pair in FP32 with the phase split per body
 * pair, e^{ik rho} = e^{ik rho_0} e^{ik (rho - rho_0)}, rho_0 = |c_a - c_b|
 * in FP64; QAMS_PREC_FF does the same split in float-float arithmetic on
 * complex128 data.  Errors: QAMS_EINVAL (R < 1, no bodies, no wavenumber). */
int qams_pairsum(qams_ctx* ctx, int R, const void* sigma_dev, void* y_dev, int precision, void* stream);

/* Self-block assembly (Sec. 3.1-3.4): for every body the dense n_b x n_b
 * block of 1/2 I + D - i eta S, by product integration against the tensor
 * Lagrange interpolant of mu |J| (Gauss-Legendre in s, trigonometric in
 * theta) with modal Green's functions for the azimuthal integral (Eqs.
 * modalgreen, modal0, leg_recur, dleg_recur, conv, I1) and a composite
 * graded Gauss rule for the singular outer integral (in place of the
 * paper's generalised Gaussian tables).  Computed in FP64 on the device,
 * kept library-owned (complex128, plus a complex64 copy for the FP32
 * path).  Uses the wavenumber of qams_set_wavenumber.  Blocking.
 * Errors: QAMS_EINVAL (no bodies/wavenumber; order > 19 or n_theta > 64),
 * QAMS_EBUDGET, QAMS_ECUDA. */
int qams_assemble(qams_ctx* ctx, void* stream);

/* Work of the last assembly: counts[0] outer quadrature nodes evaluated with
 * the modal Green's functions, counts[1] far nodes evaluated by the
 * trapezoidal rule in theta (rings far from their target), summed over all
 * rows.  For throughput accounting. */
int qams_assembly_counts(const qams_ctx* ctx, long long* counts);

/* Copy body `body`'s assembled self block (row-major n_b x n_b complex128,
 * rows = targets, columns = sources, both in node order) to dst_dev. */
int qams_copy_selfblock(const qams_ctx* ctx, int body, void* dst_dev, void* stream);

/* Block-Jacobi preconditioner (Sec. 6: GMRES with a block-diagonal
 * preconditioner from the factorisation of the self matrix): P_b = A_b^{-1}
 * for every body, by blocked Gauss-Jordan elimination in complex64 (pivot
 * blocks of 64 inverted with partial pivoting, rank-64 updates as batched
 * complex64 GEMMs), kept library-owned in complex64 and widened to
 * complex128.  Requires qams_assemble; invalidated by the next assembly.
 * Blocking.  Errors: QAMS_EINVAL, QAMS_ENUMERIC (a vanishing pivot),
 * QAMS_EBUDGET, QAMS_ECUDA. */
int qams_build_preconditioner(qams_ctx* ctx, void* stream);

/* Copy body `body`'s preconditioner block P_b (row-major n_b x n_b
 * complex128) to dst_dev. */
int qams_copy_preconditioner(const qams_ctx* ctx, int body, void* dst_dev, void* stream);

/* Operator apply (Eq. linearsys): y = (1/2 I + D - i eta S) x for [N][R]
 * complex x (densities mu, weights not folded in), self blocks times x
 * plus the inter-body pair sum of w x.  QAMS_PREC_FP64 works in complex128,
 * QAMS_PREC_FP32 in complex64 with the complex64 block copy, QAMS_PREC_FF in
 * complex128 with the float-float pair sum and the complex128 blocks.  Requires
 * qams_assemble.  Uses a library-owned workspace of N*R complex. */
int qams_apply(qams_ctx* ctx, int R, const void* x_dev, void* y_dev, int precision, void* stream);

/* Block-diagonal products (the self-block and preconditioner rows of the
 * operator, Eq. linearsys): y_b = A_b x_b (qams_selfblock_apply) or
 * y_b = P_b x_b with P_b = A_b^{-1} (qams_precond_apply) for every body, no
 * inter-body part.  x, y: [N][R], complex128 (FP64, the complex128 blocks; the
 * preconditioner's complex64 inverse widened) or complex64 (FP32, the
 * complex64 copies).  QAMS_EINVAL before qams_assemble / before the
 * preconditioner exists.  HBM-bound: every call streams all blocks once per
 * 16 right-hand sides. */
int qams_selfblock_apply(qams_ctx* ctx, int R, const void* x_dev, void* y_dev, int precision, void* stream);
int qams_precond_apply(qams_ctx* ctx, int R, const void* x_dev, void* y_dev, int precision, void* stream);

/* Solver options (Sec. 6: GMRES; restart, tolerances and orthogonalisation
 * are not stated by the paper).  precision = QAMS_PREC_FP64: restarted
 * GMRES with the FP64 apply, stop at ||b - A mu|| <= tol ||b|| per column.
 * precision = QAMS_PREC_FP32: iterative refinement -- each correction solves
 * A d = r by GMRES with the FP32 apply to a relative reduction inner_tol,
 * then mu += d and r = b - A mu with the apply of `residual` (float-float by
 * default, FP64-accurate), until r meets tol.  The
 * Krylov basis and Gram-Schmidt (classical, applied twice) are FP64 in both
 * modes.  With precondition = 1 GMRES runs on A P^{-1} with the block-
 * Jacobi preconditioner of qams_build_preconditioner (built by the first
 * solve that asks for it) and returns mu = P^{-1} z.  A cancelled server
 * request stops between restart cycles with QAMS_ECANCELLED.
 * qams_solve_opts_default fills: FP32, restart 50, max_iters 1000,
 * tol 1e-11, inner_tol 1e-5, max_refine 12, precondition 1, residual FF. */
typedef struct {
  int precision;
  int restart;      /* m, 1..200 */
  int max_iters;    /* total Arnoldi steps */
  double tol;       /* on ||b - A mu|| / ||b|| (FP64 residual) */
  double inner_tol; /* FP32 mode: reduction per correction */
  int max_refine;   /* FP32 mode: corrections */
  int precondition; /* 1: right block-Jacobi preconditioning (built on first use) */
  int residual;     /* FP32 mode: arithmetic of the residual b - A mu, QAMS_PREC_FF
                       (default) or QAMS_PREC_FP64 */
} qams_solve_opts;

typedef struct {
  int iterations;      /* Arnoldi steps (all corrections)          */
  int refinements;     /* residual evaluations (FP32 mode)         */
  double rel_residual; /* max over columns of ||b - A mu|| / ||b|| */
  double solve_ms;     /* device time of the call (CUDA events)    */
  int applies_fp32;    /* operator applies with the FP32 path      */
  int applies_fp64;    /* FP64-accurate applies (FP64 or FF)       */
} qams_solve_stats;

void qams_solve_opts_default(qams_solve_opts* opts);

/* Solve (1/2 I + D - i eta S) mu = rhs (Eq. linearsys) for R <= 16
 * right-hand sides, rhs_dev and mu_dev [N][R] complex128 (mu overwritten;
 * the initial guess is zero).  opts may be NULL (defaults); stats may be
 * NULL.  Requires qams_assemble.  Allocates its Krylov workspace
 * ((restart+1) N R complex128) for the duration of the call.  Blocking.
 * Errors: QAMS_EINVAL, QAMS_ENOCONV (mu holds the last iterate, stats
 * filled), QAMS_ENUMERIC, QAMS_EBUDGET, QAMS_ECUDA. */
int qams_solve(qams_ctx* ctx, int R, const void* rhs_dev, void* mu_dev, const qams_solve_opts* opts,
               qams_solve_stats* stats, void* stream);

/* The FP32 inter-body pair sum of qams_pairsum, for callers that cannot
 * allocate device memory: a host framework that reserves all device memory
 * for its own pool up front, or a latency-critical loop that cannot take
 * cudaMalloc's implicit device synchronisation.  It needs no context and
 * allocates nothing: every input and output is a caller-owned buffer, and
 * the call's scratch (launch tables and per-split partial sums) lives in a
 * 32 MiB array of static device memory that every GPU loading the library
 * holds until the process exits.  The paper has no counterpart; this is an
 * interface addition.
 *   body_offsets_host [n_bodies+1]: first node of each body, [0] = 0,
 *                     [n_bodies] = N, strictly increasing (host memory);
 *   centers_host      [n_bodies][3]: body centres c_b (FP64, host memory);
 *   x32_dev           float4 [N]: node position minus its body's centre
 *                     (x, y, z); .w is not read;
 *   n32_dev           float4 [N]: unit normal (x, y, z), .w not read;
 *   sigma_dev, y_dev  complex64 [N][R], y overwritten (as in qams_pairsum):
 *                     sigma must already hold w mu, the quadrature weights
 *                     folded in (Eq. multi2part).
 * Works on the current CUDA device.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it for the
 * life of the process; make that first call before any stream capture, and
 * do not use this call again after a cudaDeviceReset in the same process.
 * All calls on a device share the one array: calls that overlap on the GPU
 * race (serialise them on one stream).  Nothing in the array needs to start
 * at zero.  Blocking (returns after its work on `stream` finished).
 * When the per-split partial sums would not fit in the array, fewer source
 * splits are used (down to one, which needs no partial sums).
 * Errors: QAMS_EINVAL (bad arguments, or `stream` in stream-capture mode:
 * nothing is enqueued then), QAMS_ESCRATCH (more than 4096 bodies or more
 * than 65536 target tiles of 128 nodes), QAMS_ECUDA. */
int qams_pairsum_f32_static(int n_bodies, const long long* body_offsets_host, const double* centers_host,
                            const void* x32_dev, const void* n32_dev, int R, const void* sigma_dev, void* y_dev,
                            double k, double eta, void* stream);

/* Right-hand sides b = -u^inc = -e^{ik d.x} (Sec. 6) for R unit directions
 * dirs_host [R][3]; rhs_dev is [N][R] complex128. */
int qams_incident_plane(qams_ctx* ctx, int R, const double* dirs_host, void* rhs_dev, void* stream);

/* Far-field pattern of densities mu_dev [N][R] complex128 at M unit
 * directions dirs_host [M][3] (Sec. 6, restated for the combined layer):
 *   u_inf(xhat) = (1/4pi) sum_y (-ik xhat.n(y) - i eta) e^{-ik xhat.y} w mu.
 * uinf_dev is [M][R] complex128. */
int qams_farfield(qams_ctx* ctx, int R, const void* mu_dev, int M, const double* dirs_host,
                  void* uinf_dev, void* stream);

/* Scattered field u = (D - i eta S)[mu] at M off-surface points
 * points_host [M][3] (Sec. 6: the field compared with the point-source
 * solution of Eq. artificial point source solution), by the smooth rule on
 * the surface nodes,
 *   u(x) = sum_y [(ik/rho - 1/rho^2) n(y).(y - x) - i eta] e^{ik rho}/(4 pi rho) w mu(y),
 * with a near-field correction: for a point within f node spacings of a
 * body (f = QAMS_OPT_NEAR_FIELD, default 6; the spacing is the body's
 * largest distance between neighbouring nodes) the body's smooth-rule terms
 * on the panels within one of the nearest point's panel are replaced by
 * the self blocks' product integration (Sec. 3) taken at the off-surface
 * target: modal Green's functions of the source rings seen from x, the
 * outer integral graded toward the nearest surface point (found on the host
 * by Levenberg-Marquardt from the nearest node, qams_nearest_surface_point).
 * The result is then the layer potential of the interpolated density on
 * those panels, accurate at any distance off the surface; points on a
 * surface are not supported.  mu_dev
 * [N][R] and u_dev [M][R] are complex128.  Blocking on `stream`.
 * Errors: QAMS_EINVAL (also a near point whose ring bandwidth k (r + d)
 * exceeds the self-block kernel's tables, as qams_assemble), QAMS_EBUDGET,
 * QAMS_ECUDA. */
int qams_field(qams_ctx* ctx, int R, const void* mu_dev, int M, const double* points_host, void* u_dev,
               void* stream);

/* (point, body) pairs the last qams_field corrected in the near field. */
int qams_field_near_pairs(const qams_ctx* ctx, long long* pairs);

/* ------------------------------------------------------------------------
 * Serving: a request loop over independent scattering problems (the
 * paper solves one problem at a time).  Each request is a full solve -- its
 * own bodies, wavenumber and incident directions.  Requests are admitted
 * while their estimated device footprint fits in the server's HBM budget
 * and a slot is free; every admitted request runs on its own CUDA stream
 * with its own library context, so requests that arrive while others are on
 * the GPU start as soon as a slot and memory free up and their kernels
 * overlap on the device (continuous batching).  The kernels are
 * deterministic, so a request's result does not depend on what else runs.
 * ------------------------------------------------------------------------ */
typedef struct qams_server qams_server; /* opaque */

typedef struct {
  int n_bodies;
  const qams_body_desc* bodies; /* copied at submit */
  double k, eta;
  int R;                        /* right-hand sides, 1..16 */
  const double* dirs;           /* [R][3] incident directions, copied */
  int M;                        /* far-field directions (0 = none) */
  const double* far_dirs;       /* [M][3], copied */
  int precision;                /* QAMS_PREC_FP64 or QAMS_PREC_FP32 (refined) */
  double tol;                   /* relative residual target */
  double* mu_host;              /* optional [N][R] complex128 output (caller-owned, valid until done) */
  double* uinf_host;            /* optional [M][R] complex128 output (caller-owned, valid until done) */
} qams_request;

typedef struct {
  int status;           /* QAMS_OK or the request's error code */
  long long n_nodes;
  int iterations, refinements;
  double rel_residual;
  double queue_ms;      /* submit -> admission        */
  double run_ms;        /* admission -> completion    */
  double latency_ms;    /* submit -> completion       */
  size_t footprint;     /* admitted footprint estimate */
} qams_result;

/* Device bytes a solve of these bodies with R right-hand sides and restart m
 * holds: node tables, self blocks (complex128 + complex64), preconditioner
 * (complex64 + complex128), Krylov basis and workspaces.  Host only; the
 * descriptors are validated as by qams_set_bodies (QAMS_EINVAL). */
int qams_footprint(const qams_body_desc* bodies, int n_bodies, int R, int restart, size_t* bytes);

/* Start a server on CUDA device `cuda_device` with `max_slots` concurrent
 * requests and an HBM budget (0 = 90% of the device's free memory now). */
int qams_server_create(qams_server** out, int cuda_device, size_t hbm_budget, int max_slots);
/* Drops queued requests, waits for running ones, frees everything. */
void qams_server_destroy(qams_server* s);
/* Non-blocking.  QAMS_EBUDGET when the request could never fit the budget. */
int qams_submit(qams_server* s, const qams_request* req, uint64_t* ticket);
/* QAMS_EAGAIN while queued or running; otherwise fills *result and forgets
 * the ticket (returns QAMS_OK even when result->status is an error). */
int qams_poll(qams_server* s, uint64_t ticket, qams_result* result);
/* Queued: dropped at once.  Running: stops at the next GMRES restart
 * boundary; the result then has status QAMS_ECANCELLED. */
int qams_cancel(qams_server* s, uint64_t ticket);

#ifdef __cplusplus
}
#endif
#endif /* QAMS_H */
