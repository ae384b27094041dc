"""Writes tests/golden/oracle_solves_*.npz: the FP64 oracle's dense solutions
(Eq. linearsys, dense LU) and far fields (Sec. 6, 48 Fibonacci directions)
for the reduced scenes of the 16-, 100- and 1000-body workloads
(scenes.reduced: rigid copies of each workload's first seeded body, at its
discretisation, wavenumber and right-hand sides) and for one serving
request.  Calls only oracle/ (and the input generators of scenes/).

    python tests/golden/make_oracle_solves.py [name ...] [--workers W]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import scenes  # noqa: E402
from oracle import operator as op  # noqa: E402
from oracle import solve as osolve  # noqa: E402
from oracle.geometry import body_nodes  # noqa: E402
from oracle.selfblock import self_block  # noqa: E402

CASES = {
    # name: (scene factory, congruent copies share one block)
    "c1_copies2": (lambda: scenes.reduced(1, 2), True),
    "c2_copies3": (lambda: scenes.reduced(2, 3), True),
    "c3_copies4": (lambda: scenes.reduced(3, 4), True),
    "serve12": (lambda: scenes.serving_request(12, max_bodies=10), False),
}
FAR = 48


def run(name, workers):
    make, shared = CASES[name]
    sc = make()
    nodes = [body_nodes(b) for b in sc.bodies]
    t0 = time.time()
    if shared:
        A1 = self_block(nodes[0], sc.k, sc.eta, workers=workers)
        blocks = [A1] * len(nodes)
    else:
        blocks = [self_block(n, sc.k, sc.eta, workers=workers) for n in nodes]
    A = op.dense_matrix(nodes, blocks, sc.k, sc.eta)
    b = op.incident(nodes, sc.directions, sc.k)
    mu = osolve.dense_solve(A, b)
    xh = scenes.fibonacci_directions(FAR)
    uinf = op.farfield(nodes, mu, xh, sc.k, sc.eta)
    path = os.path.join(HERE, f"oracle_solves_{name}.npz")
    np.savez_compressed(path, mu=mu, uinf=uinf, far_dirs=xh, k=sc.k, eta=sc.eta, directions=sc.directions,
                        scene=sc.name)
    print(f"{name}: N={mu.shape[0]} R={mu.shape[1]} k={sc.k:.3f} {time.time() - t0:.0f} s -> {path}", flush=True)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=list(CASES))
    ap.add_argument("--workers", type=int, default=0)
    a = ap.parse_args()
    for nm in a.names:
        run(nm, a.workers)
