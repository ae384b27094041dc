"""FP32 inter-body pair sum with its accumulation on the tensor cores
(tcgen05 kind::tf32, split operands) against the FP64 pair sum and the
CUDA-core FP32 kernel (Eq. multi2part), for several right-hand-side counts,
ragged target tiles and several source splits; and through a full solve."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx

pytestmark = pytest.mark.gpu

FP32_TOL = 3e-5  # of the largest entry: the FP32 pair-sum tolerance of the other tests


@pytest.mark.parametrize("R", [2, 4, 5, 16])
def test_tc_pairsum_matches_fp64(R):
    import torch

    import paper_2606_31380_b300 as q
    # 7 bodies of 160 nodes: ragged 128-target tiles, several source splits
    sc = scenes.small_scene(7, 1, 8, 20, k=6.0, eta=1.0, seed=31, box=10.0)
    ctx = make_ctx(sc)
    s64 = torch.from_numpy(scenes.rhs_seeded(ctx.N, R, 50 + R)).cuda()
    s32 = s64.to(torch.complex64)
    ref = torch.empty_like(s64)
    ctx.pairsum(s64, ref, q.PREC_FP64)
    r = ref.cpu().numpy()
    out = {}
    for tc in (1, 17):
        ctx.set_option(q.OPT_TC_PAIR_MIN_RHS, tc)
        ctx.profile(True)
        y = torch.full_like(s32, float("nan"))
        ctx.pairsum(s32, y, q.PREC_FP32)
        n_tc, _ = ctx.profile_read(q.PROF_PAIRSUM_TC)
        ctx.profile(False)
        assert (n_tc > 0) == (tc == 1)
        a = y.cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(a))
        out[tc] = np.max(np.abs(a - r)) / np.max(np.abs(r))
    assert out[1] < FP32_TOL and out[17] < FP32_TOL
    ctx.close()


def test_tc_pairsum_thousand_bodies_sampled_rows_against_oracle():
    """1000 bodies x 512 nodes, k = 3, R = 4 (N = 512,000), one source split:
    sampled rows against the oracle's explicit FP64 pair sum."""
    import torch

    import paper_2606_31380_b300 as q
    from oracle import operator as op
    from oracle.geometry import body_nodes
    sc = scenes.config(3)
    ctx = make_ctx(sc)
    R = sc.n_rhs
    sig = scenes.rhs_seeded(ctx.N, R, 9)
    y = torch.empty((ctx.N, R), dtype=torch.complex64, device="cuda")
    ctx.pairsum(torch.from_numpy(sig).to(torch.complex64).cuda(), y, q.PREC_FP32)
    rows = [5, 512 * 321 + 200, 512 * 777 + 63, ctx.N - 1]
    nodes = [body_nodes(b) for b in sc.bodies]
    ref = op.pair_sum(nodes, sig, sc.k, sc.eta, targets=rows)
    got = y.cpu().numpy()[rows].astype(np.complex128)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < FP32_TOL
    ctx.close()


@pytest.mark.parametrize("R", [1, 4, 16])
def test_two_targets_per_thread_matches_fp64(R):
    """The CUDA-core FP32 pair sum with two targets per thread (tiles of 256
    targets, ragged) against the FP64 pair sum."""
    import torch

    import paper_2606_31380_b300 as q
    sc = scenes.small_scene(5, 1, 8, 40, k=6.0, eta=1.0, seed=33, box=10.0)  # 320-node bodies
    ctx = make_ctx(sc)
    s64 = torch.from_numpy(scenes.rhs_seeded(ctx.N, R, 70 + R)).cuda()
    ref = torch.empty_like(s64)
    ctx.pairsum(s64, ref, q.PREC_FP64)
    ctx.set_option(q.OPT_TC_PAIR_MIN_RHS, 17)
    ctx.set_option(q.OPT_PAIR_TARGETS, 2)
    y = torch.full_like(s64.to(torch.complex64), float("nan"))
    ctx.pairsum(s64.to(torch.complex64), y, q.PREC_FP32)
    r = ref.cpu().numpy()
    a = y.cpu().numpy().astype(np.complex128)
    assert np.all(np.isfinite(a))
    assert np.max(np.abs(a - r)) / np.max(np.abs(r)) < FP32_TOL
    ctx.close()
