"""The launch-shape autotuner (qams_autotune) picks among equivalent FP32
kernels: its choice is cached per shape, and the pair sum and apply it
installs agree with the FP64 ones within the FP32 tolerance."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx

pytestmark = pytest.mark.gpu

FP32_TOL = 3e-5


def test_autotune_choice_cached_and_correct():
    import torch

    import paper_2606_31380_b300 as q
    sc = scenes.small_scene(9, 1, 8, 20, k=5.0, eta=1.0, n_rhs=8, seed=44, box=12.0)
    ctx = make_ctx(sc)
    ctx.assemble()
    t1 = ctx.autotune(8)
    assert t1["cached"] == 0 and 1 <= t1["pair_splits"] <= 9 and t1["block_tc"] in (0, 1)  # timed at R = 8
    assert t1["pair_ms"] > 0 and t1["block_ms"] > 0
    # a second context of the same shape takes the cached choice
    ctx2 = make_ctx(sc)
    t2 = ctx2.autotune(8)
    assert t2["cached"] == 1
    for key in ("pair_tc", "pair_splits"):
        assert t2[key] == t1[key]
    s64 = torch.from_numpy(scenes.rhs_seeded(ctx.N, 8, 3)).cuda()
    ref = torch.empty_like(s64)
    ctx.pairsum(s64, ref, q.PREC_FP64)
    y = torch.empty_like(s64.to(torch.complex64))
    ctx2.pairsum(s64.to(torch.complex64), y, q.PREC_FP32)
    r = ref.cpu().numpy()
    assert np.max(np.abs(y.cpu().numpy() - r)) / np.max(np.abs(r)) < FP32_TOL
    ya = torch.empty_like(y)
    yb = torch.empty_like(s64)
    ctx.apply(s64.to(torch.complex64), ya, q.PREC_FP32)
    ctx.apply(s64, yb, q.PREC_FP64)
    b = yb.cpu().numpy()
    assert np.max(np.abs(ya.cpu().numpy() - b)) / np.max(np.abs(b)) < FP32_TOL
    ctx.close()
    ctx2.close()
