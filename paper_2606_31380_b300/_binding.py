"""ctypes binding of libqams (argument marshalling only; all arithmetic runs in
the library's CUDA kernels).  Tensors are torch CUDA tensors: complex128
[N, R] for the FP64 path and complex64 [N, R] for the FP32 path."""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
PREC_FP64 = 0
PREC_FP32 = 1
PREC_FF = 2  # float-float pair sum on complex128 data
# launch-timing slots (qams_profile_read)
PROF_PAIRSUM_FP32, PROF_PAIRSUM_FF, PROF_PAIRSUM_FP64, PROF_BLOCK_FP32, PROF_BLOCK_FP64, PROF_ASSEMBLY, \
    PROF_BLOCK_TC, PROF_PAIRSUM_TC, PROF_PAIRSUM_LATTICE, PROF_LATTICE_PRODUCT32, PROF_LATTICE_PRODUCT64 = range(11)
OPT_TC_MIN_RHS, OPT_TC_PAIR_MIN_RHS, OPT_PAIR_TARGETS, OPT_LATTICE, OPT_NEAR_FIELD = 0, 1, 2, 3, 4  # option keys


def lib_path() -> str:
    return os.path.join(HERE, "libqams.so")


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("restart", C.c_int), ("max_iters", C.c_int), ("tol", C.c_double),
                ("inner_tol", C.c_double), ("max_refine", C.c_int), ("precondition", C.c_int),
                ("residual", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("rel_residual", C.c_double),
                ("solve_ms", C.c_double), ("applies_fp32", C.c_int), ("applies_fp64", C.c_int)]


class Tuning(C.Structure):
    _fields_ = [("R", C.c_int), ("pair_tc", C.c_int), ("pair_targets", C.c_int), ("pair_splits", C.c_int),
                ("block_tc", C.c_int),
                ("pair_ms", C.c_double), ("block_ms", C.c_double), ("cached", C.c_int)]


class Request(C.Structure):
    _fields_ = [("n_bodies", C.c_int), ("bodies", C.c_void_p), ("k", C.c_double), ("eta", C.c_double),
                ("R", C.c_int), ("dirs", C.c_void_p), ("M", C.c_int), ("far_dirs", C.c_void_p),
                ("precision", C.c_int), ("tol", C.c_double), ("mu_host", C.c_void_p), ("uinf_host", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("n_nodes", C.c_longlong), ("iterations", C.c_int), ("refinements", C.c_int),
                ("rel_residual", C.c_double), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("latency_ms", C.c_double), ("footprint", C.c_size_t)]


class BodyDesc(C.Structure):
    _fields_ = [("n_panels", C.c_int), ("order", C.c_int), ("n_theta", C.c_int),
                ("base_radius", C.c_double), ("n_modes", C.c_int),
                ("mode_cos", C.POINTER(C.c_double)), ("mode_sin", C.POINTER(C.c_double)),
                ("axis_length", C.c_double), ("curvature", C.c_double),
                ("rotation", C.c_double * 9), ("center", C.c_double * 3),
                ("profile_kind", C.c_int), ("n_terms", C.c_int),
                ("series", C.POINTER(C.c_double)), ("panel_breaks", C.POINTER(C.c_double))]


_LIB = None


def load_library():
    """Load the in-tree libqams.so; raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libqams.so is not built ({path}); run paper_2606_31380_b300/build.py")
    lib = C.CDLL(path)
    vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "qams_strerror": (C.c_char_p, [i]),
        "qams_kernel_launches": (C.c_longlong, []),
        "qams_create": (i, [C.POINTER(vp), i, C.c_size_t]),
        "qams_destroy": (None, [vp]),
        "qams_set_bodies": (i, [vp, i, C.POINTER(BodyDesc), d]),
        "qams_node_count": (i, [vp, C.POINTER(ll)]),
        "qams_body_offsets": (i, [vp, C.POINTER(ll)]),
        "qams_get_nodes": (i, [vp, vp, vp, vp]),
        "qams_set_wavenumber": (i, [vp, d, d]),
        "qams_pairsum": (i, [vp, i, vp, vp, i, vp]),
        "qams_incident_plane": (i, [vp, i, vp, vp, vp]),
        "qams_assemble": (i, [vp, vp]),
        "qams_copy_selfblock": (i, [vp, i, vp, vp]),
        "qams_assembly_counts": (i, [vp, vp]),
        "qams_apply": (i, [vp, i, vp, vp, i, vp]),
        "qams_build_preconditioner": (i, [vp, vp]),
        "qams_footprint": (i, [vp, i, i, i, C.POINTER(C.c_size_t)]),
        "qams_server_create": (i, [C.POINTER(vp), i, C.c_size_t, i]),
        "qams_server_destroy": (None, [vp]),
        "qams_submit": (i, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "qams_poll": (i, [vp, C.c_uint64, C.POINTER(Result)]),
        "qams_cancel": (i, [vp, C.c_uint64]),
        "qams_copy_preconditioner": (i, [vp, i, vp, vp]),
        "qams_solve_opts_default": (None, [C.POINTER(SolveOpts)]),
        "qams_pairsum_f32_static": (i, [i, vp, vp, vp, vp, i, vp, vp, d, d, vp]),
        "qams_solve": (i, [vp, i, vp, vp, C.POINTER(SolveOpts), C.POINTER(SolveStats), vp]),
        "qams_farfield": (i, [vp, i, vp, i, vp, vp, vp]),
        "qams_field": (i, [vp, i, vp, i, vp, vp, vp]),
        "qams_body_nodes": (i, [vp, vp, vp, vp]),
        "qams_selfblock_apply": (i, [vp, i, vp, vp, i, vp]),
        "qams_profile_enable": (i, [vp, i]),
        "qams_set_option": (i, [vp, i, ll]),
        "qams_autotune": (i, [vp, i, C.POINTER(Tuning), vp]),
        "qams_selftest_timeout": (i, [i, ll, vp]),
        "qams_get_option": (i, [vp, i, C.POINTER(ll)]),
        "qams_profile_read": (i, [vp, i, C.POINTER(ll), C.POINTER(d)]),
        "qams_precond_apply": (i, [vp, i, vp, vp, i, vp]),
        "qams_set_lattice": (i, [vp, C.POINTER(BodyDesc), vp, vp, d]),
        "qams_lattice_prepare": (i, [vp, vp]),
        "qams_field_near_pairs": (i, [vp, C.POINTER(ll)]),
        "qams_nearest_surface_point": (i, [vp, vp, C.POINTER(d), C.POINTER(d), C.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


class QamsError(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = load_library()
        super().__init__(f"{what}: {lib.qams_strerror(code).decode()} (code {code})")
        self.code = code


def kernel_launches() -> int:
    """Kernels launched by libqams in this process so far."""
    return int(load_library().qams_kernel_launches())


def _check(code: int, what: str):
    if code != 0:
        raise QamsError(code, what)


def body_desc_array(bodies) -> tuple:
    """Marshal scene bodies (objects with the qams_body_desc fields) into a
    ctypes array; returns (array, keep-alive list)."""
    arr = (BodyDesc * len(bodies))()
    keep = []
    for dst, b in zip(arr, bodies):
        nm = max(len(b.mode_cos), len(b.mode_sin))
        a = np.zeros(nm)
        s = np.zeros(nm)
        a[: len(b.mode_cos)] = b.mode_cos
        s[: len(b.mode_sin)] = b.mode_sin
        ca = (C.c_double * max(nm, 1))(*a)
        cs = (C.c_double * max(nm, 1))(*s)
        keep += [ca, cs]
        dst.n_panels, dst.order, dst.n_theta = b.n_panels, b.order, b.n_theta
        dst.base_radius = b.base_radius
        dst.n_modes = nm
        dst.mode_cos = C.cast(ca, C.POINTER(C.c_double))
        dst.mode_sin = C.cast(cs, C.POINTER(C.c_double))
        dst.axis_length, dst.curvature = b.axis_length, b.curvature
        dst.rotation = (C.c_double * 9)(*[float(v) for v in b.rotation])
        dst.center = (C.c_double * 3)(*[float(v) for v in b.center])
        kind = int(getattr(b, "kind", 0))
        dst.profile_kind = kind
        if kind == 1:
            parts = list(b.series)
            nt = max(1, max(len(p) for p in parts))
            ser = np.zeros((4, nt, 3))
            for q, part in enumerate(parts):
                for j, term in enumerate(part):
                    ser[q, j] = term
            cser = (C.c_double * ser.size)(*ser.reshape(-1))
            keep.append(cser)
            dst.n_terms = nt
            dst.series = C.cast(cser, C.POINTER(C.c_double))
        br = tuple(getattr(b, "panel_breaks", ()) or ())
        if br:
            cbr = (C.c_double * len(br))(*[float(v) for v in br])
            keep.append(cbr)
            dst.panel_breaks = C.cast(cbr, C.POINTER(C.c_double))
    return arr, keep


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _dev(t, dtype, shape, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{what}: expected contiguous {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


class Context:
    """One libqams context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.lib = load_library()
        self._h = C.c_void_p()
        _check(self.lib.qams_create(C.byref(self._h), device, hbm_budget), "qams_create")
        self.device = device
        self.N = 0
        self.R = 0

    def close(self):
        if self._h:
            self.lib.qams_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- setup -------------------------------------------------------------
    def set_bodies(self, bodies, min_gap: float = 0.0):
        arr, keep = body_desc_array(bodies)
        _check(self.lib.qams_set_bodies(self._h, len(bodies), arr, float(min_gap)), "qams_set_bodies")
        n = C.c_longlong()
        _check(self.lib.qams_node_count(self._h, C.byref(n)), "qams_node_count")
        self.N = int(n.value)
        self.n_bodies = len(bodies)

    def set_lattice(self, body, dims, basis, min_gap: float = 0.0):
        """dims[0] x dims[1] x dims[2] copies of ``body`` at body.center + p a0 + q a1 + r a2
        (a_i the rows of the 3x3 ``basis``), body index (p dims[1] + q) dims[2] + r."""
        arr, keep = body_desc_array([body])
        d = (C.c_int * 3)(*[int(v) for v in dims])
        bs = np.ascontiguousarray(np.asarray(basis, dtype=np.float64).reshape(9))
        _check(self.lib.qams_set_lattice(self._h, arr, C.cast(d, C.c_void_p), bs.ctypes.data_as(C.c_void_p),
                                         float(min_gap)), "qams_set_lattice")
        n = C.c_longlong()
        _check(self.lib.qams_node_count(self._h, C.byref(n)), "qams_node_count")
        self.N = int(n.value)
        self.n_bodies = int(dims[0]) * int(dims[1]) * int(dims[2])

    def lattice_prepare(self, stream=None):
        """Build the transformed displacement blocks of a lattice context."""
        _check(self.lib.qams_lattice_prepare(self._h, C.c_void_p(_stream_ptr(stream))), "qams_lattice_prepare")

    def body_offsets(self) -> np.ndarray:
        off = np.zeros(self.n_bodies + 1, np.int64)
        _check(self.lib.qams_body_offsets(self._h, off.ctypes.data_as(C.POINTER(C.c_longlong))),
               "qams_body_offsets")
        return off

    def get_nodes(self):
        x = np.zeros((self.N, 3))
        n = np.zeros((self.N, 3))
        w = np.zeros(self.N)
        _check(self.lib.qams_get_nodes(self._h, x.ctypes.data_as(C.c_void_p), n.ctypes.data_as(C.c_void_p),
                                       w.ctypes.data_as(C.c_void_p)), "qams_get_nodes")
        return x, n, w

    def set_wavenumber(self, k: float, eta: float = 1.0):
        _check(self.lib.qams_set_wavenumber(self._h, float(k), float(eta)), "qams_set_wavenumber")
        self.k, self.eta = float(k), float(eta)

    # --- compute -----------------------------------------------------------
    def pairsum(self, sigma, y, precision: int = PREC_FP64, stream=None):
        import torch
        R = sigma.shape[1]
        dt = torch.complex64 if precision == PREC_FP32 else torch.complex128
        _check(self.lib.qams_pairsum(self._h, R, _dev(sigma, dt, (self.N, R), "sigma"),
                                     _dev(y, dt, (self.N, R), "y"), precision, C.c_void_p(_stream_ptr(stream))),
               "qams_pairsum")

    def autotune(self, R: int, stream=None) -> dict:
        """Time the equivalent FP32 kernel variants for R right-hand sides and
        install the fastest (qams_autotune); returns the choice."""
        t = Tuning()
        _check(self.lib.qams_autotune(self._h, R, C.byref(t), C.c_void_p(_stream_ptr(stream))), "qams_autotune")
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def set_option(self, key: int, value: int):
        _check(self.lib.qams_set_option(self._h, key, int(value)), "qams_set_option")

    def get_option(self, key: int) -> int:
        v = C.c_longlong()
        _check(self.lib.qams_get_option(self._h, key, C.byref(v)), "qams_get_option")
        return int(v.value)

    def profile(self, on: bool):
        """Start (clearing the sums) or stop timing the hot kernels' launches."""
        _check(self.lib.qams_profile_enable(self._h, 1 if on else 0), "qams_profile_enable")

    def profile_read(self, slot: int):
        """(launches, total device ms) of one kernel class since profile(True)."""
        n, ms = C.c_longlong(), C.c_double()
        _check(self.lib.qams_profile_read(self._h, slot, C.byref(n), C.byref(ms)), "qams_profile_read")
        return int(n.value), float(ms.value)

    def assemble(self, stream=None):
        _check(self.lib.qams_assemble(self._h, C.c_void_p(_stream_ptr(stream))), "qams_assemble")

    def assembly_counts(self):
        """(modal outer nodes, far outer nodes) of the last assembly."""
        out = np.zeros(2, np.int64)
        _check(self.lib.qams_assembly_counts(self._h, out.ctypes.data_as(C.c_void_p)), "qams_assembly_counts")
        return int(out[0]), int(out[1])

    def copy_selfblock(self, body: int, dst, stream=None):
        import torch
        n = int(self.body_offsets()[body + 1] - self.body_offsets()[body])
        _check(self.lib.qams_copy_selfblock(self._h, body, _dev(dst, torch.complex128, (n, n), "dst"),
                                            C.c_void_p(_stream_ptr(stream))), "qams_copy_selfblock")

    def build_preconditioner(self, stream=None):
        _check(self.lib.qams_build_preconditioner(self._h, C.c_void_p(_stream_ptr(stream))),
               "qams_build_preconditioner")

    def copy_preconditioner(self, body: int, dst, stream=None):
        import torch
        n = int(self.body_offsets()[body + 1] - self.body_offsets()[body])
        _check(self.lib.qams_copy_preconditioner(self._h, body, _dev(dst, torch.complex128, (n, n), "dst"),
                                                 C.c_void_p(_stream_ptr(stream))), "qams_copy_preconditioner")

    def apply(self, x, y, precision: int = PREC_FP64, stream=None):
        import torch
        R = x.shape[1]
        dt = torch.complex64 if precision == PREC_FP32 else torch.complex128
        _check(self.lib.qams_apply(self._h, R, _dev(x, dt, (self.N, R), "x"), _dev(y, dt, (self.N, R), "y"),
                                   precision, C.c_void_p(_stream_ptr(stream))), "qams_apply")

    def selfblock_apply(self, x, y, precision: int = PREC_FP64, stream=None):
        """y_b = A_b x_b for every body (no inter-body part)."""
        self._diag("qams_selfblock_apply", x, y, precision, stream)

    def precond_apply(self, x, y, precision: int = PREC_FP64, stream=None):
        """y_b = P_b x_b, P_b = A_b^{-1} (after build_preconditioner or a preconditioned solve)."""
        self._diag("qams_precond_apply", x, y, precision, stream)

    def _diag(self, name, x, y, precision, stream):
        import torch
        dt = torch.complex64 if precision == PREC_FP32 else torch.complex128
        R = x.shape[1]
        _check(getattr(self.lib, name)(self._h, R, _dev(x, dt, (self.N, R), "x"), _dev(y, dt, (self.N, R), "y"),
                                       precision, C.c_void_p(_stream_ptr(stream))), name)

    def solve(self, rhs, mu, precision: int = PREC_FP32, tol: float = None, restart: int = None,
              max_iters: int = None, inner_tol: float = None, precondition: bool = True, stream=None,
              check: bool = True, residual: int = None):
        """Solve A mu = rhs; returns a dict of solver statistics."""
        import torch
        R = rhs.shape[1]
        o = SolveOpts()
        self.lib.qams_solve_opts_default(C.byref(o))
        o.precision = precision
        if tol is not None:
            o.tol = tol
        elif precision == PREC_FP64:
            o.tol = 1e-12
        if restart is not None:
            o.restart = restart
        if max_iters is not None:
            o.max_iters = max_iters
        if inner_tol is not None:
            o.inner_tol = inner_tol
        o.precondition = 1 if precondition else 0
        if residual is not None:
            o.residual = residual
        st = SolveStats()
        code = self.lib.qams_solve(self._h, R, _dev(rhs, torch.complex128, (self.N, R), "rhs"),
                                   _dev(mu, torch.complex128, (self.N, R), "mu"), C.byref(o), C.byref(st),
                                   C.c_void_p(_stream_ptr(stream)))
        stats = dict(iterations=st.iterations, refinements=st.refinements, rel_residual=st.rel_residual,
                     solve_ms=st.solve_ms, applies_fp32=st.applies_fp32, applies_fp64=st.applies_fp64,
                     code=code)
        if check:
            _check(code, "qams_solve")
        return stats

    def incident_plane(self, dirs: np.ndarray, rhs, stream=None):
        import torch
        dirs = np.ascontiguousarray(dirs, float)
        R = dirs.shape[0]
        _check(self.lib.qams_incident_plane(self._h, R, dirs.ctypes.data_as(C.c_void_p),
                                            _dev(rhs, torch.complex128, (self.N, R), "rhs"),
                                            C.c_void_p(_stream_ptr(stream))), "qams_incident_plane")

    def farfield(self, mu, dirs: np.ndarray, uinf, stream=None):
        import torch
        dirs = np.ascontiguousarray(dirs, float)
        M = dirs.shape[0]
        R = mu.shape[1]
        _check(self.lib.qams_farfield(self._h, R, _dev(mu, torch.complex128, (self.N, R), "mu"), M,
                                      dirs.ctypes.data_as(C.c_void_p),
                                      _dev(uinf, torch.complex128, (M, R), "uinf"),
                                      C.c_void_p(_stream_ptr(stream))), "qams_farfield")

    def field(self, mu, points: np.ndarray, u, stream=None):
        """Scattered field at off-surface points [M][3] into u [M][R] (complex128)."""
        import torch
        points = np.ascontiguousarray(points, float)
        M = points.shape[0]
        R = mu.shape[1]
        _check(self.lib.qams_field(self._h, R, _dev(mu, torch.complex128, (self.N, R), "mu"), M,
                                   points.ctypes.data_as(C.c_void_p),
                                   _dev(u, torch.complex128, (M, R), "u"),
                                   C.c_void_p(_stream_ptr(stream))), "qams_field")

    def field_near_pairs(self) -> int:
        """(point, body) pairs the last field() call corrected in the near field."""
        v = C.c_longlong()
        _check(self.lib.qams_field_near_pairs(self._h, C.byref(v)), "qams_field_near_pairs")
        return int(v.value)


QAMS_EAGAIN = -10


def body_nodes(body):
    """Host-side Nystrom nodes of one body: world positions (n, 3), unit normals
    (n, 3), weights (n,) -- no device needed."""
    lib = load_library()
    arr, keep = body_desc_array([body])
    n = body.n_panels * body.order * body.n_theta
    x, nn, w = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    _check(lib.qams_body_nodes(C.cast(arr, C.c_void_p), x.ctypes.data_as(C.c_void_p),
                               nn.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p)), "qams_body_nodes")
    return x, nn, w


def nearest_surface_point(body, x):
    """(s, theta, distance) of the nearest surface point of one body to the
    world point x, as the near-field correction finds it -- no device needed."""
    lib = load_library()
    arr, keep = body_desc_array([body])
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))
    s, th, dist = C.c_double(), C.c_double(), C.c_double()
    _check(lib.qams_nearest_surface_point(C.cast(arr, C.c_void_p), xx.ctypes.data_as(C.c_void_p), C.byref(s),
                                          C.byref(th), C.byref(dist)), "qams_nearest_surface_point")
    return s.value, th.value, dist.value


def footprint(bodies, R: int, restart: int = 50) -> int:
    """Device bytes a solve of these bodies holds (host-side estimate)."""
    lib = load_library()
    arr, keep = body_desc_array(bodies)
    out = C.c_size_t()
    _check(lib.qams_footprint(C.cast(arr, C.c_void_p), len(bodies), R, restart, C.byref(out)), "qams_footprint")
    return int(out.value)


class Server:
    """The library's request loop: admission by device footprint, one stream per
    admitted request, requests overlapping on the GPU."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, slots: int = 4):
        self.lib = load_library()
        self._h = C.c_void_p()
        _check(self.lib.qams_server_create(C.byref(self._h), device, hbm_budget, slots), "qams_server_create")
        self._keep = {}

    def close(self):
        if self._h:
            self.lib.qams_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, scene, far_dirs=None, precision: int = PREC_FP32, tol: float = 1e-11, want_mu: bool = True):
        """Queue one scene; returns a ticket.  Outputs land in host arrays returned by poll()."""
        arr, keep = body_desc_array(scene.bodies)
        dirs = np.ascontiguousarray(scene.directions, float)
        R = dirs.shape[0]
        N = scene.n_nodes
        fd = None if far_dirs is None else np.ascontiguousarray(far_dirs, float)
        M = 0 if fd is None else fd.shape[0]
        mu = np.zeros((N, R), complex) if want_mu else None
        uinf = np.zeros((M, R), complex) if M else None
        req = Request(len(scene.bodies), C.cast(arr, C.c_void_p), scene.k, scene.eta, R,
                      dirs.ctypes.data_as(C.c_void_p), M, None if fd is None else fd.ctypes.data_as(C.c_void_p),
                      precision, tol, None if mu is None else mu.ctypes.data_as(C.c_void_p),
                      None if uinf is None else uinf.ctypes.data_as(C.c_void_p))
        t = C.c_uint64()
        _check(self.lib.qams_submit(self._h, C.byref(req), C.byref(t)), "qams_submit")
        self._keep[t.value] = (arr, keep, dirs, fd, mu, uinf)
        return int(t.value)

    def poll(self, ticket: int):
        """None while queued or running; else a dict with status, stats, mu and uinf."""
        res = Result()
        code = self.lib.qams_poll(self._h, C.c_uint64(ticket), C.byref(res))
        if code == QAMS_EAGAIN:
            return None
        _check(code, "qams_poll")
        _, _, _, _, mu, uinf = self._keep.pop(ticket)
        return dict(status=res.status, n_nodes=res.n_nodes, iterations=res.iterations,
                    refinements=res.refinements, rel_residual=res.rel_residual, queue_ms=res.queue_ms,
                    run_ms=res.run_ms, latency_ms=res.latency_ms, footprint=res.footprint, mu=mu, uinf=uinf)

    def wait(self, ticket: int, poll_s: float = 0.005):
        import time
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            time.sleep(poll_s)

    def cancel(self, ticket: int):
        _check(self.lib.qams_cancel(self._h, C.c_uint64(ticket)), "qams_cancel")
