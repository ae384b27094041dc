"""Congruent bodies share one self block and one preconditioner inverse
(the paper computes D_tt once for identical bodies, Sec. 4 and the
cubic-array runs of Sec. 6): the assembly does the work of one body, every
copy sees the same block, and that block equals the one assembled for a
single copy in another orientation (rigid-motion invariance)."""
import numpy as np
import pytest

import scenes
from gpu_util import make_ctx

pytestmark = pytest.mark.gpu


def test_congruent_copies_share_one_block():
    import torch

    import paper_2606_31380_b300 as q
    sc = scenes.reduced(3, 3)  # three rotated copies of a 512-node body, k = 3
    ctx = make_ctx(sc)
    ctx.assemble()
    ctx.build_preconditioner()
    n = sc.bodies[0].n_nodes
    c0 = make_ctx(scenes.Scene("copy 0 alone", [sc.bodies[0]], sc.k, sc.eta, sc.directions))
    c0.assemble()
    assert ctx.assembly_counts() == c0.assembly_counts()  # the work of one body
    c0.close()
    c1 = make_ctx(scenes.Scene("copy 1 alone", [sc.bodies[1]], sc.k, sc.eta, sc.directions))
    c1.assemble()
    blocks = []
    for b in range(3):
        A = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
        ctx.copy_selfblock(b, A)
        blocks.append(A.cpu().numpy())
    assert np.array_equal(blocks[0], blocks[1]) and np.array_equal(blocks[0], blocks[2])
    A1 = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    c1.copy_selfblock(0, A1)
    a1 = A1.cpu().numpy()
    assert np.max(np.abs(blocks[0] - a1)) < 1e-12 * np.max(np.abs(a1))
    P = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    ctx.copy_preconditioner(2, P)
    assert np.max(np.abs(P.cpu().numpy() @ blocks[2] - np.eye(n))) < 1e-3
    ctx.close()
    c1.close()
