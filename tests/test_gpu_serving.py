"""The serving loop (qams_server_*): continuous batching of independent solves.

A request's result is the same alone and in the mix; requests admitted
together overlap in time; admission respects the HBM budget; a queued
request can be cancelled."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

TOL_SAME = 1e-12  # alone vs in the mix (deterministic kernels)


def _reqs():
    return [scenes.serving_request(i, max_bodies=14) for i in range(4)]


def test_result_alone_equals_result_in_the_mix():
    import paper_2606_31380_b300 as q
    reqs = _reqs()
    far = scenes.fibonacci_directions(24)
    srv = q.Server(0, 0, slots=1)
    alone = [srv.wait(srv.submit(r, far)) for r in reqs]
    srv.close()
    srv = q.Server(0, 0, slots=4)
    tickets = [srv.submit(r, far) for r in reqs]
    mix = [srv.wait(t) for t in tickets]
    srv.close()
    for a, m in zip(alone, mix):
        assert a["status"] == 0 and m["status"] == 0
        assert a["rel_residual"] <= 1e-11
        assert np.max(np.abs(a["mu"] - m["mu"])) <= TOL_SAME * np.max(np.abs(a["mu"]))
        assert np.max(np.abs(a["uinf"] - m["uinf"])) <= TOL_SAME * np.max(np.abs(a["uinf"]))
    # all four were submitted together: at least two ran at the same time
    spans = [(m["queue_ms"], m["queue_ms"] + m["run_ms"]) for m in mix]
    overlaps = sum(1 for i in range(4) for j in range(i + 1, 4)
                   if min(spans[i][1], spans[j][1]) > max(spans[i][0], spans[j][0]))
    assert overlaps >= 1


def test_serving_matches_direct_solve():
    import torch
    import paper_2606_31380_b300 as q
    sc = _reqs()[0]
    srv = q.Server(0, 0, slots=2)
    res = srv.wait(srv.submit(sc))
    srv.close()
    ctx = q.Context(0)
    ctx.set_bodies(sc.bodies)
    ctx.set_wavenumber(sc.k, sc.eta)
    ctx.assemble()
    b = torch.zeros((ctx.N, sc.n_rhs), dtype=torch.complex128, device="cuda")
    ctx.incident_plane(sc.directions, b)
    mu = torch.zeros_like(b)
    ctx.solve(b, mu, q.PREC_FP32, tol=1e-11)
    ref = mu.cpu().numpy()
    assert np.max(np.abs(res["mu"] - ref)) <= TOL_SAME * np.max(np.abs(ref))


def test_admission_by_budget_and_cancellation():
    import paper_2606_31380_b300 as q
    reqs = _reqs()
    fps = [q.footprint(r.bodies, r.n_rhs) for r in reqs]
    budget = max(fps) + (1 << 20)  # holds the largest request, never two of them
    srv = q.Server(0, budget, slots=4)
    big = scenes.serving_request(0, max_bodies=14)
    big.bodies = big.bodies * 40  # forty times the bodies: above the budget
    with pytest.raises(q.QamsError):
        srv.submit(big)
    t = [srv.submit(r) for r in reqs]
    srv.cancel(t[3])
    res = [srv.wait(x) for x in t]
    srv.close()
    assert res[3]["status"] == -7  # QAMS_ECANCELLED
    done = [r for r in res[:3] if r["status"] == 0]
    assert len(done) == 3
    spans = sorted((r["queue_ms"], r["queue_ms"] + r["run_ms"]) for r in done)
    for a, b in zip(spans, spans[1:]):
        assert b[0] >= a[1] - 1.0


def test_large_request_in_the_mix_and_oracle_parity():
    """A 446-body request (16 x 32 nodes, k = 6.7, 10 RHS) served together with
    smaller ones: every result is the same alone and in the mix, and request
    12 (10 bodies, k = 2.3, 6 RHS) matches the FP64 oracle's dense solve
    (tests/golden/oracle_solves_serve12.npz) to the mixed-precision tolerance."""
    import os

    import paper_2606_31380_b300 as q
    ids = [51, 12, 3, 6]
    reqs = [scenes.serving_request(i) if i == 51 else scenes.serving_request(i, max_bodies=10) for i in ids]
    assert len(reqs[0].bodies) == 446
    ref = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_solves_serve12.npz"))
    far = ref["far_dirs"]
    srv = q.Server(0, 0, slots=1)
    alone = [srv.wait(srv.submit(r, far)) for r in reqs]
    srv.close()
    srv = q.Server(0, 0, slots=4)
    tickets = [srv.submit(r, far) for r in reqs]
    mix = [srv.wait(t) for t in tickets]
    srv.close()
    for a, m in zip(alone, mix):
        assert a["status"] == 0 and m["status"] == 0
        assert np.max(np.abs(a["mu"] - m["mu"])) <= TOL_SAME * np.max(np.abs(a["mu"]))
        assert np.max(np.abs(a["uinf"] - m["uinf"])) <= TOL_SAME * np.max(np.abs(a["uinf"]))
    m12 = mix[1]
    assert np.linalg.norm(m12["mu"] - ref["mu"]) / np.linalg.norm(ref["mu"]) < 1e-8
    assert np.linalg.norm(m12["uinf"] - ref["uinf"]) / np.linalg.norm(ref["uinf"]) < 1e-8
