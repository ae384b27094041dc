"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def make_ctx(scene):
    import paper_2606_31380_b300 as q
    ctx = q.Context(0)
    ctx.set_bodies(scene.bodies)
    ctx.set_wavenumber(scene.k, scene.eta)
    return ctx
