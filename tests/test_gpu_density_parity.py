"""Density- and far-field-level parity with the FP64 oracle on the
discretisation, wavenumber and right-hand sides of each multi-body workload
(Eq. linearsys; Sec. 6 far field), through the C ABI.

The oracle's dense solutions are stored in tests/golden/oracle_solves_*.npz,
written by tests/golden/make_oracle_solves.py (oracle calls only): a full
oracle self block costs minutes to an hour of CPU at these discretisations,
so the scenes are rigid copies of each workload's first seeded body
(scenes.reduced), which share one block."""
import os

import numpy as np
import pytest

import scenes
from gpu_util import make_ctx

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FP64_TOL = 1e-10   # relative L2, FP64 path
MIXED_TOL = 1e-8   # relative L2, FP32 operator + FP64-accurate refinement

CASES = {
    "c1_copies2": lambda: scenes.reduced(1, 2),  # 2 x 2048 nodes (32 x 64), k = 5, 1 RHS
    "c2_copies3": lambda: scenes.reduced(2, 3),  # 3 x 1152 nodes (24 x 48), k = 10, 16 RHS
    "c3_copies4": lambda: scenes.reduced(3, 4),  # 4 x 512 nodes (16 x 32), k = 3, 4 RHS
}


def l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("name", sorted(CASES))
def test_reduced_workload_against_oracle_dense_solve(name):
    import torch

    import paper_2606_31380_b300 as q
    ref = np.load(os.path.join(GOLDEN, f"oracle_solves_{name}.npz"))
    sc = CASES[name]()
    assert np.allclose(ref["directions"], sc.directions) and float(ref["k"]) == sc.k
    ctx = make_ctx(sc)
    ctx.assemble()
    R = sc.n_rhs
    b = torch.zeros((ctx.N, R), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    xh = ref["far_dirs"]
    for prec, tol, stol in [(q.PREC_FP64, FP64_TOL, 1e-13), (q.PREC_FP32, MIXED_TOL, 1e-11)]:
        mu = torch.zeros_like(b)
        st = ctx.solve(b, mu, prec, tol=stol)
        u = torch.zeros((xh.shape[0], R), dtype=torch.complex128, device="cuda")
        ctx.farfield(mu, xh, u)
        assert l2(mu.cpu().numpy(), ref["mu"]) < tol, (prec, st)
        assert l2(u.cpu().numpy(), ref["uinf"]) < tol, (prec, st)
    ctx.close()
