"""The library's host tables, built on the CPU (MUELLER_MESH_HOST_ONLY: the
same mesh load without the device uploads), against the oracle and brute
force:

* the double Morton permutation equals the oracle's, bit for bit;
* the touching pairs (Sec. 4.2) are exactly the element pairs that share a
  corner, found by the oracle's classification over all n_tri^2 pairs, with
  the same class (shared corners) and the same corner relabellings, in the
  order (test element, trial element) ascending;
* the near-block layout: rows ascending without repeats, each row's blocks
  are the nodes of every trial element touching an element that holds the
  row's node, every touching pair's 36 slots point at the block of its node
  pair, and every block is used;
* a host-only handle refuses every call that needs device data.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
import workloads
from paper_2604_21181_gb300 import api

STATE = 9


def _meshes():
    rng = np.random.default_rng(3)
    xyz, tri6 = workloads.icosphere_p2(1)
    perm = rng.permutation(len(xyz))
    inv = np.argsort(perm)
    return {
        "sphere_L1": workloads.icosphere_p2(1),
        "spheroid_L1": workloads.spheroid_p2(1, 1.0, 3.0),
        "sphere_L1_shuffled": (xyz[perm], inv[tri6].astype(np.int32)),
        "sphere_L0": workloads.icosphere_p2(0),
    }


MESHES = _meshes()


def _pack(px, py):
    return sum(int(px[k]) << (2 * k) | int(py[k]) << (8 + 2 * k) for k in range(3))


@pytest.fixture(scope="module", params=sorted(MESHES))
def case(request):
    xyz, tri6 = MESHES[request.param]
    m = api.Mesh(xyz, tri6, host_only=True)
    om = oracle.Mesh(xyz, tri6)
    yield m, om
    m.free()


def test_morton_orders_match_the_oracle(case):
    m, om = case
    npm, epm = m.perm()
    assert np.array_equal(npm, om.node_perm)
    assert np.array_equal(epm, om.elem_perm)


def test_keep_order_flag_gives_identity():
    xyz, tri6 = MESHES["sphere_L1_shuffled"]
    m = api.Mesh(xyz, tri6, morton=False, host_only=True)
    npm, epm = m.perm()
    m.free()
    assert np.array_equal(npm, np.arange(len(xyz)))
    assert np.array_equal(epm, np.arange(len(tri6)))


def test_touching_pairs_match_brute_force_classification(case):
    m, om = case
    t = m.touching()
    expect = []
    for ex in range(om.nt):
        for ey in range(om.nt):
            c, px, py = om.classify(ex, ey)
            if c > 0:
                expect.append((ex, ey, c, _pack(px, py)))
    got = list(zip(t["ex"].tolist(), t["ey"].tolist(), t["cls"].tolist(), t["relabel"].tolist()))
    assert got == expect
    # one coincident pair per element; edge pairs are three per element on a
    # closed surface
    assert np.sum(t["cls"] == 3) == om.nt
    assert np.sum(t["cls"] == 2) == 3 * om.nt


def test_near_layout_is_the_touching_node_pairs(case):
    m, om = case
    T = om.tri6  # Morton order, the same as the library's (checked above)
    t = m.touching()
    rowptr, col, slot = m.near_layout()
    nn = om.nn
    assert rowptr[0] == 0 and rowptr[-1] == len(col) == m.info()["n_near_blocks"]
    rows = [col[rowptr[i]:rowptr[i + 1]] for i in range(nn)]
    for r in rows:
        assert np.all(np.diff(r) > 0)
    # brute force: columns of node i = nodes of every ey touching an ex that holds i
    cols = [set() for _ in range(nn)]
    for ex, ey in zip(t["ex"], t["ey"]):
        for i in T[ex]:
            cols[i].update(T[ey].tolist())
    for i in range(nn):
        assert set(rows[i].tolist()) == cols[i]
    used = np.zeros(len(col), bool)
    for p, (ex, ey) in enumerate(zip(t["ex"], t["ey"])):
        for i in range(6):
            ni = T[ex, i]
            s = slot[p, i]
            assert np.all((s >= rowptr[ni]) & (s < rowptr[ni + 1]))
            assert np.array_equal(col[s], T[ey])
            used[s] = True
    assert used.all()


def test_host_only_handle_refuses_device_work():
    lib = api.load_library()
    xyz, tri6 = MESHES["sphere_L0"]
    m = api.Mesh(xyz, tri6, host_only=True)
    h = m.h
    p = api.CParams(ka=1.0, q_regular=6, ssq_order=4, frame_rule=0)
    p.eps_r[0], p.mu_r[0] = 2.0, 1.0
    assert lib.mueller_tangent_frame(h, 0, None, None) == STATE
    assert "HOST_ONLY" in lib.mueller_last_error().decode()
    buf = C.create_string_buffer(64)
    fake = C.cast(buf, C.c_void_p)
    # no frame: assembly, the operator derivative and the far field need one
    assert lib.mueller_assemble(h, C.byref(p), api.MUELLER_C128, fake, 1 << 20, None, None, None,
                                0, None) == STATE
    assert lib.mueller_dz_matvec(h, C.byref(p), 1, fake, fake, None) == STATE
    inc = np.ascontiguousarray(workloads.plane_wave().reshape(1, 6))
    xs = np.zeros((1, 3))
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    assert lib.mueller_far_field(h, C.byref(p), fake, 1, dp(inc), None, 0, None, dp(xs), 8, 16,
                                 None) == STATE
    # an operator over a host-only mesh
    op = api.COperator()
    op.mesh, op.Z_dev, op.ldz, op.dtype, op.near_dev = h, fake, 1 << 20, api.MUELLER_C64_NEAR64, fake
    assert lib.mueller_precond_build(C.byref(op), 64, fake, None) == STATE
    assert lib.mueller_matvec(C.byref(op), fake, fake, 1, None, 0, None) == STATE
    assert lib.mueller_matvec_mrhs(C.byref(op), fake, fake, 4, fake, 1 << 30, None) == STATE
    o = api.CSolverOpts(mode=api.SOLVE_GMRES_IR, restart=30, maxit=100, tol=1e-8)
    info = api.CSolveInfo()
    assert lib.mueller_solve(C.byref(op), fake, fake, 1, C.byref(o), C.byref(info), None, 0,
                             None) == STATE
    assert m.near_bytes() == 32 * 8 * m.info()["n_near_blocks"]
    m.free()


def test_incident_waves_and_directions_are_checked():
    """Rows (k-hat, p-hat) must be orthonormal and far-field directions unit
    vectors: INVALID_ARG before any device work (here before the missing
    frame of a host-only mesh would give STATE)."""
    lib = api.load_library()
    xyz, tri6 = MESHES["sphere_L0"]
    m = api.Mesh(xyz, tri6, host_only=True)
    p = api.CParams(ka=1.0, q_regular=6, ssq_order=4, frame_rule=0)
    p.eps_r[0], p.mu_r[0] = 2.0, 1.0
    buf = C.create_string_buffer(64)
    fake = C.cast(buf, C.c_void_p)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    good = np.ascontiguousarray(workloads.fibonacci_plane_waves(2))
    xs = np.zeros((4, 3))
    bad_rows = []
    b = good.copy()
    b[0, 3:] = good[0, :3]  # p parallel to k
    bad_rows.append((0, b))
    b = good.copy()
    b[1, :3] *= 1.001  # k not a unit vector
    bad_rows.append((1, b))
    b = good.copy()
    b[2, 3:] = (good[2, 3:] + 0.1 * good[2, :3]) / np.linalg.norm(good[2, 3:] + 0.1 * good[2, :3])
    bad_rows.append((2, b))  # unit p, not orthogonal to k
    b = good.copy()
    b[3, 5] = np.nan
    bad_rows.append((3, b))
    for row, b in bad_rows:
        assert lib.mueller_assemble(m.h, C.byref(p), api.MUELLER_C128, fake, 1 << 20, None, fake,
                                    dp(b), 4, None) == 1
        assert ("incident wave %d" % row) in lib.mueller_last_error().decode()
        for fn in (lib.mueller_far_field, lib.mueller_far_field_noalloc):
            assert fn(m.h, C.byref(p), fake, 4, dp(b), None, 0, None, dp(xs), 8, 16, None) == 1
    # the well-formed waves pass the checks and meet the missing frame
    assert lib.mueller_assemble(m.h, C.byref(p), api.MUELLER_C128, fake, 1 << 20, None, fake,
                                dp(good), 4, None) == STATE
    dirs = np.ascontiguousarray(workloads.fibonacci_directions(5))
    F = fake
    assert lib.mueller_far_field(m.h, C.byref(p), fake, 4, dp(good), dp(dirs), 5, F, dp(xs), 8, 16,
                                 None) == STATE
    dirs[2] *= 1.01
    for fn in (lib.mueller_far_field, lib.mueller_far_field_noalloc):
        assert fn(m.h, C.byref(p), fake, 4, dp(good), dp(dirs), 5, F, dp(xs), 8, 16, None) == 1
        assert "direction 2" in lib.mueller_last_error().decode()
    m.free()
