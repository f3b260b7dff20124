"""C-ABI checks that need no GPU: the library builds and loads, exports every
function that include/mueller.h declares, and rejects bad arguments and bad
meshes on the host before any device work."""

import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads
from paper_2604_21181_gb300 import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pass
    return api.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mueller.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mueller_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_function(lib):
    decl = declared_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(api.EXPORTS) == decl


def test_version_and_status_strings(lib):
    assert lib.mueller_version() >= 1
    assert lib.mueller_status_string(0) == b"ok"
    assert lib.mueller_status_string(2) == b"invalid mesh"


def _load(lib, xyz, tri6):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri6 = np.ascontiguousarray(tri6, dtype=np.int32)
    h = C.c_void_p()
    st = lib.mueller_mesh_load(xyz.ctypes.data_as(C.POINTER(C.c_double)), xyz.shape[0],
                               tri6.ctypes.data_as(C.POINTER(C.c_int32)), tri6.shape[0], 0, None,
                               C.byref(h))
    return st, lib.mueller_last_error().decode()


def test_mesh_validation_rejects_bad_meshes(lib):
    xyz, tri6 = workloads.icosphere_p2(1)
    # null pointers / sizes
    h = C.c_void_p()
    assert lib.mueller_mesh_load(None, 10, None, 10, 0, None, C.byref(h)) == 1
    # open surface: drop one triangle
    st, msg = _load(lib, xyz, tri6[:-1])
    assert st == 2 and "manifold" in msg
    # flipped triangle
    bad = tri6.copy()
    bad[5, [1, 2]] = bad[5, [2, 1]]
    bad[5, [3, 5]] = bad[5, [5, 3]]
    st, msg = _load(lib, xyz, bad)
    assert st == 2 and "orient" in msg
    # NaN coordinate
    x2 = xyz.copy()
    x2[3, 1] = np.nan
    st, msg = _load(lib, x2, tri6)
    assert st == 2 and "finite" in msg
    # node id out of range
    bad = tri6.copy()
    bad[0, 4] = len(xyz) + 5
    st, msg = _load(lib, xyz, bad)
    assert st == 2
    # inconsistent edge node
    bad = tri6.copy()
    bad[0, 3] = bad[1, 3] if bad[1, 3] != bad[0, 3] else bad[2, 3]
    st, msg = _load(lib, xyz, bad)
    assert st == 2


def test_size_queries(lib):
    # 2B x 2B complex128 inverses for ceil((N/2)/B) blocks, plus the sizes
    N, B = 10248, 256
    nb = -(-(N // 2) // B)
    assert lib.mueller_precond_bytes(N, B) >= nb * (2 * B) ** 2 * 16
    assert lib.mueller_precond_bytes(0, B) == 0
