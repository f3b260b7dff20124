"""The point geometry of the regular rule (Sec. 3.3: P2 position, unit normal,
the continuous tangent frame by Gram-Schmidt of the interpolated nodal frame,
the co-normals, the surface Jacobian) on the GPU, read back with
mueller_point_records, against the oracle's geometry at the same points.

Every regular-pair and far-field integral of the library reads these records,
so this pins them directly (they are otherwise checked only through Z and the
far field).  Both frame rules, both regular rules, a sphere and a spheroid;
the element order is the shared Morton order (checked first)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    ("sphere_L1_paper_q6", lambda: workloads.icosphere_p2(1), 0, 6),
    ("spheroid_L1_polar_q12", lambda: workloads.spheroid_p2(1, 1.0, 1.5), 1, 12),
    ("sphere_L2_polar_q6", lambda: workloads.icosphere_p2(2), 1, 6),
    ("spheroid_L2_paper_q12", lambda: workloads.spheroid_p2(2, 1.3, 1.0), 0, 12),
]


def _library_rule(q):
    import ctypes as C
    lib = mu.load_library()
    a, b, w = np.zeros(16), np.zeros(16), np.zeros(16)
    ptr = lambda v: v.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    assert lib.mueller_quadrature_rule(0, q, ptr(a), ptr(b), ptr(w)) == 0
    return a[:q], b[:q], w[:q]


@pytest.mark.parametrize("name,mk,rule,q", CASES, ids=[c[0] for c in CASES])
def test_point_records_match_the_oracle_geometry(name, mk, rule, q):
    xyz, tri6 = mk()
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(rule, out=False)
    p = mu.Params(ka=1.0, eps_r=(2.0, 0.0), q_regular=q, ssq_order=2, frame_rule=rule)
    mu.assemble(m, p, mu.MUELLER_C128)  # builds the rule's point geometry
    rec = m.point_records(q)
    om = oracle.Mesh(xyz, tri6, frame_rule=rule)
    npm, epm = m.perm()
    assert np.array_equal(npm, om.node_perm) and np.array_equal(epm, om.elem_perm)
    # the oracle's geometry at the library's rule points (the two rules are
    # derived independently: the 12-point ones differ by about 5e-14 in the
    # points and 4e-13 in the weights, within the 1e-11 of the Z parity)
    xi_o, eta_o, w_o = oracle.tri_rule(q)
    xi, eta, w = _library_rule(q)
    assert max(np.abs(xi - xi_o).max(), np.abs(eta - eta_o).max()) <= 1e-13
    assert np.abs(w - w_o).max() <= 1e-12 * w.max()
    ref = np.zeros_like(rec)
    for e in range(m.nt):
        for k in range(q):
            g = om.point_geo(e, xi[k], eta[k])
            ref[e, k, :18] = np.concatenate([g["x"], g["n"], g["t1"], g["t2"], g["s1"], g["s2"]])
            ref[e, k, 18] = g["J"] * w[k]
    vec = np.abs(rec[:, :, :18] - ref[:, :, :18]).max()
    assert vec <= 1e-13, vec
    wt = np.abs(rec[:, :, 18] - ref[:, :, 18]).max() / np.abs(ref[:, :, 18]).max()
    assert wt <= 1e-13, wt
    # unit vectors, orthogonal frame, co-normals as stated
    n, t1, t2 = rec[..., 3:6], rec[..., 6:9], rec[..., 9:12]
    for v in (n, t1, t2):
        assert np.abs(np.linalg.norm(v, axis=-1) - 1).max() <= 1e-13
    assert np.abs((n * t1).sum(-1)).max() <= 1e-13 and np.abs((t1 * t2).sum(-1)).max() <= 1e-13
    assert np.abs(rec[..., 12:15] - np.cross(t1, n)).max() <= 1e-13


def test_point_records_need_the_rule_geometry():
    xyz, tri6 = workloads.icosphere_p2(0)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(0, out=False)
    with pytest.raises(mu.MuellerError) as e:
        m.point_records(6)
    assert e.value.status == 9  # MUELLER_ERR_STATE
