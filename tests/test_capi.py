"""The C-ABI library loads and exports every entry point include/qams.h declares
(no compute call: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "qams.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qams_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared()
    for must in ["qams_create", "qams_destroy", "qams_set_bodies", "qams_pairsum", "qams_farfield"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2606_31380_b300 as q
    lib = q.load_library()
    for name in declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", q.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(qams_\w+)", out))
    assert set(declared()) <= exported


def test_errors_without_device_are_reported_not_crashing():
    import ctypes as C
    import paper_2606_31380_b300 as q
    lib = q.load_library()
    assert lib.qams_strerror(-3).decode().startswith("bodies overlap")
    assert lib.qams_create(None, 0, 0) == -1  # out == NULL -> QAMS_EINVAL


def test_descriptor_validation_on_host():
    """qams_footprint validates descriptors without a device: the paper's shapes
    and dyadic panels pass; an open profile, a falling axial coordinate and
    breakpoints that do not span [-pi/2, pi/2] are rejected."""
    import math
    import scenes
    import paper_2606_31380_b300 as q
    good = [scenes.conch(), scenes.spiral(), scenes.quasi_wave(), scenes.quasi_ellipsoid(scale=0.3),
            scenes.Body(8, 16, 32, 0.5, (0.1,), (), 1.0, 0.2, panel_breaks=scenes.dyadic_breaks(4, 2)),
            scenes.conch(n_panels=22, breaks=scenes.dyadic_breaks(12, 5))]
    assert q.footprint(good, 1) > 0
    bad = [
        scenes._ring_body((((1.0, 1.0, 0.0),), (), ((1.0, 0.0, 2.0),), ((0.0, 0.5, 0.0),)), 4, 8, 16, 1.0),
        scenes._ring_body(((), (), ((1.0, 0.0, -2.0),), ((1.0, 1.0, 0.0),)), 4, 8, 16, 1.0),
        scenes.Body(3, 8, 16, panel_breaks=(-math.pi / 2, 0.3, 0.2, math.pi / 2)),
        scenes.Body(2, 8, 16, panel_breaks=(-1.5, 0.0, math.pi / 2)),
        scenes.Body(2, 8, 16, 0.5, (0.7, 0.4), ()),
    ]
    for b in bad:
        with pytest.raises(q.QamsError):
            q.footprint([b], 1)


def test_static_pairsum_rejects_oversized_input_before_any_device_work():
    """qams_pairsum_f32_static refuses more bodies than its static scratch
    holds (QAMS_ESCRATCH) before touching the device: no launch, no CUDA call."""
    import ctypes as C
    import numpy as np
    import paper_2606_31380_b300 as q
    lib = q.load_library()
    nb = 4097
    offs = np.arange(nb + 1, dtype=np.int64) * 4
    cens = np.zeros((nb, 3), np.float64)
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    before = q.kernel_launches()
    code = lib.qams_pairsum_f32_static(nb, offs.ctypes.data_as(C.c_void_p), cens.ctypes.data_as(C.c_void_p),
                                       dummy, dummy, 1, dummy, dummy, 2.0, 1.0, None)
    assert code == -9  # QAMS_ESCRATCH
    assert q.kernel_launches() == before
