"""Pins of the oracle's mesh handling, frames and singular quadrature on
physical elements (Sec. 3, Sec. 4.2, Sec. 5, Appendix A)."""

import math

import numpy as np
import pytest

import oracle
import workloads


# ------------------------------------------------------------------ Morton
def _spread(v):
    r = np.zeros_like(v, dtype=np.uint64)
    for b in range(21):
        r |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return r


def _keys(p, lo, ext):
    q = np.floor(np.clip((p - lo) / ext * 2097152.0, 0, 2097151)).astype(np.uint64)
    return _spread(q[:, 0]) | (_spread(q[:, 1]) << np.uint64(1)) | (_spread(q[:, 2]) << np.uint64(2))


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_morton_order_is_the_z_curve_definition(level):
    xyz, tri6 = workloads.icosphere_p2(level)
    npm, epm = oracle.morton(xyz, tri6)
    assert sorted(npm.tolist()) == list(range(len(xyz)))
    assert sorted(epm.tolist()) == list(range(len(tri6)))
    lo = xyz.min(0)
    ext = (xyz.max(0) - lo).max()
    kn = _keys(xyz, lo, ext)
    ref = np.lexsort((np.arange(len(xyz)), kn))
    np.testing.assert_array_equal(npm, ref)
    cen = xyz[tri6[:, :3]].mean(1)
    cen = (xyz[tri6[:, 0]] + xyz[tri6[:, 1]] + xyz[tri6[:, 2]]) / 3.0
    ke = _keys(cen, lo, ext)
    np.testing.assert_array_equal(epm, np.lexsort((np.arange(len(tri6)), ke)))


def test_morton_is_local():
    xyz, tri6 = workloads.icosphere_p2(3)
    a = oracle.morton(xyz, tri6)
    # consecutive Morton nodes are much closer than random pairs
    p = xyz[a[0]]
    d_seq = np.linalg.norm(np.diff(p, axis=0), axis=1).mean()
    rng = np.random.default_rng(0)
    d_rand = np.linalg.norm(p[rng.permutation(len(p))] - p, axis=1).mean()
    assert d_seq < 0.2 * d_rand


# ------------------------------------------------------------------ frames
def _normal_error(level, axis=1.0, rule=0):
    if axis == 1.0:
        xyz, tri6 = workloads.icosphere_p2(level)
    else:
        xyz, tri6 = workloads.spheroid_p2(level, 1.0, axis)
    m = oracle.Mesh(xyz, tri6, frame_rule=rule)
    fr = m.frame()
    x = m.xyz
    nex = x / np.array([1.0, 1.0, axis ** 2])
    nex /= np.linalg.norm(nex, axis=1, keepdims=True)
    ang = np.arccos(np.clip(np.einsum("ij,ij->i", fr[:, 0:3], nex), -1, 1))
    return ang.max(), fr


def test_nodal_frame_is_orthonormal_and_right_handed():
    for rule in (0, 1):
        _, fr = _normal_error(2, rule=rule)
        n, t1, t2 = fr[:, 0:3], fr[:, 3:6], fr[:, 6:9]
        for a in (n, t1, t2):
            np.testing.assert_allclose(np.linalg.norm(a, axis=1), 1.0, atol=1e-14)
        assert np.abs(np.einsum("ij,ij->i", n, t1)).max() < 1e-14
        np.testing.assert_allclose(np.cross(n, t1), t2, atol=1e-14)
        # reference-axis rule (Eqs. t1, t2)
        if rule == 0:
            pol = np.abs(n[:, 2]) > 0.9
            ref = np.where(pol[:, None], [1.0, 0, 0], [0, 0, 1.0])
            t1r = np.cross(ref, n)
            t1r /= np.linalg.norm(t1r, axis=1, keepdims=True)
            np.testing.assert_allclose(t1, t1r, atol=1e-14)


def test_metric_weighted_normal_converges_at_paper_rates():
    # Appendix A: O(h^3) on spheres (C_k = 0), O(h^2) in general.
    es = [_normal_error(L)[0] for L in (1, 2, 3, 4)]
    rates = [math.log2(es[i] / es[i + 1]) for i in range(3)]
    assert min(rates[1:]) > 2.6, (es, rates)
    ep = [_normal_error(L, axis=1.5)[0] for L in (2, 3, 4)]
    ratesp = [math.log2(ep[i] / ep[i + 1]) for i in range(2)]
    assert min(ratesp) > 1.7, (ep, ratesp)


def test_quadrature_point_frame_is_tangent_and_orthonormal():
    xyz, tri6 = workloads.spheroid_p2(2, 1.0, 1.5)
    m = oracle.Mesh(xyz, tri6)
    xi, eta, _ = oracle.tri_rule(12)
    worst = 0.0
    for e in range(0, m.nt, 7):
        for a, b in zip(xi, eta):
            g = m.point_geo(e, a, b)
            n, t1, t2 = g["n"], g["t1"], g["t2"]
            worst = max(worst, abs(n @ t1), abs(n @ t2), abs(t1 @ t2),
                        abs(t1 @ t1 - 1), abs(t2 @ t2 - 1))
            np.testing.assert_allclose(g["s1"], np.cross(t1, n), atol=1e-15)
            np.testing.assert_allclose(g["s2"], np.cross(t2, n), atol=1e-15)
    assert worst < 1e-14


def test_mass_matrix_partition_of_unity_gives_area():
    # sum_ij M_ij = area of the P2 surface -> 4 pi, fourth order in h
    errs = []
    for L in (1, 2, 3):
        xyz, tri6 = workloads.icosphere_p2(L)
        m = oracle.Mesh(xyz, tri6)
        M = m.mass(12)
        np.testing.assert_allclose(M, M.T, atol=1e-16)
        errs.append(abs(M.sum() - 4 * math.pi))
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 8


# -------------------------------------------------- singular quadrature
def _pairs_by_class(m, ex=0):
    out = {}
    for ey in range(m.nt):
        c, _, _ = m.classify(ex, ey)
        out.setdefault(c, ey)
    return out


def _subtriangles(level):
    tris = [np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])]
    for _ in range(level):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(t) for t in ([a, ab, ca], [ab, b, bc], [ca, bc, c], [ab, bc, ca])]
        tris = nxt
    return tris


def _elem_integral(m, e, fn, level=3):
    # 12-point rule on 4^level parametric sub-triangles (J is not a polynomial)
    xi, eta, w = oracle.tri_rule(12)
    s = 0.0
    for a, b, c in _subtriangles(level):
        for u, v, ww in zip(xi, eta, w):
            p = a + u * (b - a) + v * (c - a)
            g = m.point_geo(e, p[0], p[1])
            s = s + ww * 0.25 ** level * g["J"] * fn(g["x"])
    return s


def test_ssq_integrates_smooth_integrands_on_curved_pairs():
    xyz, tri6 = workloads.spheroid_p2(1, 1.0, 1.5)
    m = oracle.Mesh(xyz, tri6)
    pairs = _pairs_by_class(m)
    for cls in (3, 2, 1):
        ey = pairs[cls]
        # kappa = 1: product of the two element areas
        Ax = m.ssq_test(0, 0, 10, 0)
        Ay = m.ssq_test(ey, ey, 10, 0)
        got = m.ssq_test(0, ey, 8, 0)
        assert abs(got - math.sqrt(Ax * Ay)) < 1e-13 * got
        # |x - y|^2 = |x|^2 + |y|^2 - 2 x.y separates into single integrals
        ax = _elem_integral(m, 0, lambda x: 1.0)
        ay = _elem_integral(m, ey, lambda x: 1.0)
        ref = (ay * _elem_integral(m, 0, lambda x: x @ x) + ax * _elem_integral(m, ey, lambda x: x @ x)
               - 2 * _elem_integral(m, 0, lambda x: x) @ _elem_integral(m, ey, lambda x: x))
        got = m.ssq_test(0, ey, 8, 2)
        assert abs(got - ref) < 1e-10 * abs(ref), (cls, got, ref)


def _flat_fan():
    # regular hexagon fan in z = 0: vertex 0 at the centre, 6 triangles
    ang = np.arange(6) * np.pi / 3
    V = np.concatenate([[[0.0, 0.0, 0.0]], np.stack([np.cos(ang), np.sin(ang), 0 * ang], 1)])
    V[3] += [0.13, -0.07, 0.0]  # break the symmetry
    tris = [[0, 1 + k, 1 + (k + 1) % 6] for k in range(6)]
    edges = {}
    nodes = [v for v in V]
    tri6 = []
    for t in tris:
        row = list(t)
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            key = (min(a, b), max(a, b))
            if key not in edges:
                edges[key] = len(nodes)
                nodes.append(0.5 * (V[a] + V[b]))
            row.append(edges[key])
        tri6.append(row)
    return np.array(nodes), np.array(tri6, dtype=np.int32)


def _flat_potential(x, T):
    """int_T 1/|x - y| dy for points x (k x 3) in the plane of the flat
    triangle T (3 x 3): signed decomposition into the triangles (x, v_k,
    v_k+1), each h [asinh(t2/h) - asinh(t1/h)]."""
    nT = np.cross(T[1] - T[0], T[2] - T[0])
    nT /= np.linalg.norm(nT)
    out = np.zeros(len(x))
    for k in range(3):
        a, b = T[k], T[(k + 1) % 3]
        e = (b - a) / np.linalg.norm(b - a)
        foot = a + np.outer((x - a) @ e, e)
        hv = x - foot
        h = np.linalg.norm(hv, axis=1)
        t1 = (a - foot) @ e
        t2 = (b - foot) @ e
        sgn = np.sign(np.cross(a - x, b - x) @ nT)
        ok = h > 1e-300
        out[ok] += sgn[ok] * h[ok] * (np.arcsinh(t2[ok] / h[ok]) - np.arcsinh(t1[ok] / h[ok]))
    return out


def _graded_outer(T, fn, n=64):
    t, w = np.polynomial.legendre.leggauss(n)
    p = 0.5 * (t + 1)
    wp = 0.5 * w
    sig = p ** 3 * (10 - 15 * p + 6 * p ** 2)
    dsig = 30 * p ** 2 * (1 - p) ** 2
    S, Tt = np.meshgrid(sig, sig, indexing="ij")
    W = np.outer(wp * dsig, wp * dsig)
    A, B, C = T
    X = A[None, None] + S[..., None] * (B - A) + (S * Tt)[..., None] * (C - B)
    jac = S * np.linalg.norm(np.cross(B - A, C - B))
    return float(np.sum(W * jac * fn(X.reshape(-1, 3)).reshape(S.shape)))


def test_ssq_one_over_r_matches_semi_analytic_flat_integrals():
    nodes, tri6 = _flat_fan()
    m = oracle.Mesh(nodes, tri6, morton=False)
    T = [nodes[tri6[e, :3]] for e in range(6)]
    for ey, cls in ((0, 3), (1, 2), (2, 1)):
        c, _, _ = m.classify(0, ey)
        assert c == cls
        ref = _graded_outer(T[0], lambda X: _flat_potential(X, T[ey]))
        vals = [m.ssq_test(0, ey, ns, 1) for ns in (4, 6, 8, 10)]
        assert abs(vals[-1] - ref) < 1e-9 * ref, (cls, vals, ref)
        # exponential convergence in the order
        errs = [abs(v - ref) for v in vals]
        assert errs[0] > errs[1] > errs[2]


def test_ssq_results_do_not_depend_on_the_relabelling():
    xyz, tri6 = workloads.spheroid_p2(1, 1.0, 1.5)
    m = oracle.Mesh(xyz, tri6)
    pairs = _pairs_by_class(m, ex=5)
    for cls in (2, 1):
        ey = pairs[cls]
        c1, G = m.ssq_singular(5, ey, 10)
        c2, Ga = m.ssq_singular(5, ey, 10, alt=True)
        assert c1 == c2 == cls
        scale = np.abs(G).max()
        assert np.abs(G - Ga).max() < 1e-10 * scale


def test_split_singular_plus_remainder_approaches_full_ssq_on_small_pairs():
    # Sec. 4.1: kappa = kappa^s (by SSQ) + (kappa - kappa^s) (regular rule).
    # On small elements the remainder is tiny, so the split must agree with
    # Sauter-Schwab applied to the whole (cancelled, stable) kernel.  This
    # also confirms that no O(R^-3) term survives: the full kernel integrates
    # to a finite, converged value.
    p = dict(ka=2.0, eps_r=(3.0, 0.2), mu_r=(1.0, 0.0), q_regular=12, ssq_order=8)
    xyz, tri6 = workloads.icosphere_p2(4)
    m = oracle.Mesh(xyz * 0.1, tri6)  # edge length ~ 0.008
    pairs = _pairs_by_class(m, ex=3)
    for cls in (3, 2, 1):
        ey = pairs[cls]
        _, Lsplit = m.pair_block(p, 3, ey)
        _, Lfull = m.ssq_full(p, 3, ey, 10)
        _, Lfull2 = m.ssq_full(p, 3, ey, 12)
        scale = np.abs(Lfull[..., :4]).max()
        assert np.abs(Lfull - Lfull2).max() < 1e-9 * scale  # SSQ converged
        assert np.abs(Lsplit - Lfull).max() < 1e-4 * scale, (cls, np.abs(Lsplit - Lfull).max() / scale)
