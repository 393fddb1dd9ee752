"""The C-ABI library loads and exports every entry point of include/dg.h
(no compute calls: these run without a GPU)."""
import ctypes

import pytest
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src)))


def test_header_matches_binding(built_lib):
    assert declared_symbols() == sorted(built_lib.ABI_SYMBOLS)


def test_library_exports_every_symbol(built_lib):
    L = ctypes.CDLL(built_lib.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib.LIB_PATH],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dg_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_last_error_callable_without_gpu(built_lib):
    assert built_lib.lib().dg_last_error() == b""


def test_invalid_mesh_rejected_without_side_effects(built_lib):
    """DG_EINVAL for overlapping boxes, before any device work."""
    import numpy as np
    from paper_2009_01287_gb300.inputs import MeshDesc
    bad = MeshDesc(2, np.array([[0, 0], [0, 0]], dtype=np.int32), np.array([1, 1], dtype=np.int32),
                   np.array([1, 1], dtype=np.int32), (2, 1), 0.5)
    try:
        built_lib.dg_mesh_create(bad)
        raise AssertionError("accepted an invalid mesh")
    except built_lib.DGError as e:
        assert e.code == built_lib.DG_EINVAL


def _desc(dim, lo, size, p, extent, lh=0.25):
    import numpy as np
    from paper_2009_01287_gb300.inputs import MeshDesc
    return MeshDesc(dim, np.asarray(lo, dtype=np.int32).reshape(-1, dim), np.asarray(size, dtype=np.int32),
                    np.asarray(p, dtype=np.int32), tuple(extent), lh)


BAD = {
    "3d-overlap": lambda: _desc(3, [(0, 0, 0), (0, 0, 0)], [1, 1], [1, 1], (2, 1, 1)),
    "3d-gap": lambda: _desc(3, [(0, 0, 0)], [1], [2], (2, 1, 1)),
    "3d-misaligned": lambda: _desc(3, [(1, 0, 0), (0, 0, 0), (0, 2, 0)], [2, 1, 1], [1, 1, 1], (3, 3, 1)),
    "3d-size-not-pow2": lambda: _desc(3, [(0, 0, 0)], [3], [1], (3, 3, 3)),
    "3d-degree-0": lambda: _desc(3, [(0, 0, 0)], [1], [0], (1, 1, 1)),
    "3d-degree-9": lambda: _desc(3, [(0, 0, 0)], [1], [9], (1, 1, 1)),
    "3d-outside": lambda: _desc(3, [(0, 0, 0), (1, 0, 0)], [1, 1], [1, 1], (1, 1, 1)),
    # squares may leave holes, but a side may not border a hole in part only
    "2d-partial-hole": lambda: _desc(2, [(0, 0), (2, 0), (3, 0), (3, 1)], [2, 1, 1, 1], [1, 1, 1, 1], (4, 2)),
    "2d-coeff-zero": lambda: _with_coeff(_desc(2, [(0, 0), (1, 0)], [1, 1], [1, 2], (2, 1)), [1.0, 0.0]),
    "2d-coeff-nan": lambda: _with_coeff(_desc(2, [(0, 0), (1, 0)], [1, 1], [1, 2], (2, 1)), [float("nan"), 1.0]),
    "3d-coeff-negative": lambda: _with_coeff(_desc(3, [(0, 0, 0)], [1], [2], (1, 1, 1)), [-20.0]),
}


def _with_coeff(mesh, a):
    from paper_2009_01287_gb300 import inputs
    return inputs.with_coeff(mesh, a)


@pytest.mark.parametrize("name", list(BAD))
def test_invalid_meshes_rejected(built_lib, name):
    """Invalid 2D and 3D descriptions give DG_EINVAL with a message, before
    any device work (overlap, a gap in a cube mesh or a square's side along
    part of a hole, misaligned or non-dyadic boxes, degrees
    outside 1..8, boxes outside the domain, a coefficient that is not positive
    and finite)."""
    try:
        built_lib.dg_mesh_create(BAD[name]())
        raise AssertionError("accepted an invalid mesh")
    except built_lib.DGError as e:
        assert e.code == built_lib.DG_EINVAL
        assert str(e)
