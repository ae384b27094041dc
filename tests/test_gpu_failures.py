"""Failure paths of the C ABI, injected from the host (no device fault):
overlapping bodies (QAMS_EGEOM), an iteration limit (QAMS_ENOCONV with the
statistics filled), a non-finite right-hand side (QAMS_ENUMERIC) and an HBM
budget below the footprint (QAMS_EBUDGET), and a bounded device wait that
runs out (QAMS_ETIMEOUT).  Each leaves the context usable."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx

pytestmark = pytest.mark.gpu

EGEOM, EBUDGET, ENOCONV, ENUMERIC = -3, -2, -4, -5


def test_overlapping_bodies_are_rejected():
    import paper_2606_31380_b300 as q
    b1 = scenes.Body(1, 8, 16, center=(0.0, 0.0, 0.0))
    b2 = scenes.Body(1, 8, 16, center=(0.3, 0.0, 0.0))  # bounding balls overlap
    ctx = q.Context(0)
    with pytest.raises(q.QamsError) as e:
        ctx.set_bodies([b1, b2], min_gap=0.1)
    assert e.value.code == EGEOM
    # the context still accepts a valid configuration
    b2.center = (3.0, 0.0, 0.0)
    ctx.set_bodies([b1, b2], min_gap=0.1)
    assert ctx.N == 2 * 128
    ctx.close()


def test_iteration_limit_reports_enoconv_with_stats():
    import torch

    import paper_2606_31380_b300 as q
    sc = scenes.small_scene(3, 1, 8, 16, k=4.0, seed=3)
    ctx = make_ctx(sc)
    ctx.assemble()
    b = torch.zeros((ctx.N, 1), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    for prec in (q.PREC_FP64, q.PREC_FP32):
        mu = torch.zeros_like(b)
        st = ctx.solve(b, mu, prec, tol=1e-13, max_iters=1, check=False)
        assert st["code"] == ENOCONV
        assert st["iterations"] == 1 and st["rel_residual"] > 1e-13
        assert np.all(np.isfinite(mu.cpu().numpy())) and float(torch.linalg.norm(mu)) > 0
    mu = torch.zeros_like(b)
    assert ctx.solve(b, mu, q.PREC_FP32, tol=1e-11)["code"] == 0
    ctx.close()


def test_nan_right_hand_side_reports_enumeric():
    import torch

    import paper_2606_31380_b300 as q
    sc = scenes.small_scene(2, 1, 8, 16, k=2.0, seed=4)
    ctx = make_ctx(sc)
    ctx.assemble()
    b = torch.zeros((ctx.N, 1), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    bad = b.clone()
    bad[7, 0] = complex(float("nan"), 0.0)
    for prec in (q.PREC_FP64, q.PREC_FP32):
        mu = torch.zeros_like(b)
        assert ctx.solve(bad, mu, prec, check=False)["code"] == ENUMERIC
    mu = torch.zeros_like(b)
    assert ctx.solve(b, mu, q.PREC_FP64, tol=1e-12)["code"] == 0
    ctx.close()


def test_budget_below_footprint_reports_ebudget():
    import paper_2606_31380_b300 as q
    sc = scenes.small_scene(3, 1, 8, 16, k=2.0, seed=5)
    need = q.footprint(sc.bodies, 1)
    # 200 KB: the node tables fit, the self blocks (3 x 128^2 complex128 = 786 KB) do not
    ctx = q.Context(0, hbm_budget=200_000)
    with pytest.raises(q.QamsError) as e:
        ctx.set_bodies(sc.bodies)
        ctx.set_wavenumber(sc.k, sc.eta)
        ctx.assemble()
    assert e.value.code == EBUDGET
    ctx.close()
    ok = q.Context(0, hbm_budget=need * 2)
    ok.set_bodies(sc.bodies)
    ok.set_wavenumber(sc.k, sc.eta)
    ok.assemble()
    ok.close()


def test_bounded_device_wait_reports_etimeout():
    """A CTA waits, the way the tensor-core kernels do, on an mbarrier that
    nothing completes: the wait gives up after ~2^20 cycles, the call returns
    QAMS_ETIMEOUT, and the device keeps working."""
    import torch

    import paper_2606_31380_b300 as q
    lib = q.load_library()
    assert lib.qams_selftest_timeout(0, 1 << 20, None) == -6  # QAMS_ETIMEOUT
    sc = scenes.small_scene(2, 1, 8, 16, k=2.0, seed=6)
    ctx = make_ctx(sc)
    x = torch.from_numpy(scenes.rhs_seeded(ctx.N, 1, 1)).cuda()
    y = torch.empty_like(x)
    ctx.pairsum(x, y, q.PREC_FP64)
    assert bool(torch.isfinite(y).all())
    ctx.close()
