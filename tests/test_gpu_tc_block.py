"""Tensor-core (tcgen05, split-FP16) self-block and preconditioner products
against the FP64 products of the same blocks (the dense diagonal blocks of
Eq. linearsys), and the FP32 operator apply with and without them."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx

pytestmark = pytest.mark.gpu

# split-FP16 keeps ~22 bits per operand: FP32-level, like the CUDA-core product
TC_TOL = 2e-6


def _rand(torch, N, R, seed, dtype):
    return torch.from_numpy(scenes.rhs_seeded(N, R, seed)).to(dtype).cuda()


@pytest.mark.parametrize("R", [4, 7, 16])
def test_tc_block_products_match_fp64(R):
    import torch

    import paper_2606_31380_b300 as q
    # 160-node bodies: two 128-row tiles, the second ragged
    sc = scenes.small_scene(5, 1, 8, 20, k=4.0, eta=1.0, seed=21, box=9.0)
    ctx = make_ctx(sc)
    ctx.assemble()
    ctx.build_preconditioner()
    x = _rand(torch, ctx.N, R, 40 + R, torch.complex64)
    x64 = x.to(torch.complex128)
    for which in ("selfblock_apply", "precond_apply"):
        ref = torch.empty_like(x64)
        getattr(ctx, which)(x64, ref, q.PREC_FP64)
        ctx.set_option(q.OPT_TC_MIN_RHS, 1)
        ctx.profile(True)
        y_tc = torch.full_like(x, float("nan"))
        getattr(ctx, which)(x, y_tc, q.PREC_FP32)
        n_tc, _ = ctx.profile_read(q.PROF_BLOCK_TC)
        ctx.profile(False)
        assert n_tc >= 1  # the tensor-core kernel ran
        ctx.set_option(q.OPT_TC_MIN_RHS, 17)
        y_cc = torch.empty_like(x)
        getattr(ctx, which)(x, y_cc, q.PREC_FP32)
        r = ref.cpu().numpy()
        for y in (y_tc, y_cc):
            a = y.cpu().numpy().astype(np.complex128)
            assert np.all(np.isfinite(a))
            assert np.max(np.abs(a - r)) / np.max(np.abs(r)) < TC_TOL, which
    ctx.close()


def test_tc_apply_matches_cuda_core_apply_and_solve():
    """The full FP32 apply (pair sum plus block products, accumulated) and a
    mixed solve are the same with the tensor-core block products."""
    import torch

    import paper_2606_31380_b300 as q
    sc = scenes.small_scene(4, 1, 8, 16, k=3.0, eta=1.0, n_rhs=4, seed=5, box=8.0)
    ctx = make_ctx(sc)
    ctx.assemble()
    x = _rand(torch, ctx.N, 4, 77, torch.complex64)
    out = {}
    for tc in (1, 17):
        ctx.set_option(q.OPT_TC_MIN_RHS, tc)
        y = torch.empty_like(x)
        ctx.apply(x, y, q.PREC_FP32)
        out[tc] = y.cpu().numpy()
    assert np.max(np.abs(out[1] - out[17])) / np.max(np.abs(out[17])) < TC_TOL
    b = torch.zeros((ctx.N, 4), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    mus = {}
    for tc in (1, 17):
        ctx.set_option(q.OPT_TC_MIN_RHS, tc)
        mu = torch.zeros_like(b)
        ctx.solve(b, mu, q.PREC_FP32, tol=1e-11)
        mus[tc] = mu.cpu().numpy()
    assert np.linalg.norm(mus[1] - mus[17]) / np.linalg.norm(mus[17]) < 1e-9
    ctx.close()
