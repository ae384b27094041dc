"""The no-allocation FP32 pair sum (qams_pairsum_f32_static) gives the same
result as qams_pairsum on two calls in a row.

It serves callers that cannot allocate device memory (a host framework that
owns all device memory through its own pool, or a latency-critical loop
that cannot take cudaMalloc's implicit synchronisation): they pass every
buffer, and the call keeps its scratch in static device memory.  This file
is collected last so that a run stopping at the first failure has already
run every other test."""
import ctypes as C

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

FP32_TOL = 3e-5  # the FP32 pair-sum tolerance of the other GPU tests


def _run(sc, Rs):
    import torch

    import paper_2606_31380_b300 as q

    ctx = q.Context(0)
    ctx.set_bodies(sc.bodies)
    ctx.set_wavenumber(sc.k, sc.eta)
    off = ctx.body_offsets()
    x, n, w = ctx.get_nodes()
    cen = np.array([b.center for b in sc.bodies], float)
    owner = np.repeat(np.arange(len(sc.bodies)), np.diff(off))
    x32 = np.zeros((ctx.N, 4), np.float32)
    x32[:, :3] = x - cen[owner]
    x32[:, 3] = w
    n32 = np.zeros((ctx.N, 4), np.float32)
    n32[:, :3] = n
    dx32 = torch.from_numpy(x32).cuda()
    dn32 = torch.from_numpy(n32).cuda()
    lib = q.load_library()
    offs = np.ascontiguousarray(off, np.int64)
    cens = np.ascontiguousarray(cen, np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    for call, R in enumerate(Rs):
        sigma = torch.from_numpy(scenes.rhs_seeded(ctx.N, R, 20 + call)).to(torch.complex64).cuda()
        ref = torch.empty_like(sigma)
        ctx.pairsum(sigma, ref, q.PREC_FP32)
        out = torch.full_like(sigma, float("nan"))
        code = lib.qams_pairsum_f32_static(len(sc.bodies), offs.ctypes.data_as(C.c_void_p),
                                           cens.ctypes.data_as(C.c_void_p), C.c_void_p(dx32.data_ptr()),
                                           C.c_void_p(dn32.data_ptr()), R, C.c_void_p(sigma.data_ptr()),
                                           C.c_void_p(out.data_ptr()), sc.k, sc.eta, C.c_void_p(stream))
        assert code == 0, lib.qams_strerror(code).decode()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < FP32_TOL
    ctx.close()


def test_static_scratch_pairsum_matches_allocating_entry_point():
    """Six 160-node bodies (ragged target tiles), R = 3 then R = 1: several
    source splits whose partial sums sit in the static scratch."""
    _run(scenes.small_scene(6, 1, 8, 20, k=4.0, eta=1.0, seed=13, box=9.0), [3, 1])


def test_static_scratch_pairsum_single_split_at_full_size():
    """1000 bodies x 512 nodes at R = 16: the per-split partial sums (8 N R
    bytes per split) no longer fit the 32 MiB scratch, so the call falls back
    to one source split that writes y directly; then R = 4."""
    _run(scenes.config(3), [16, 4])
