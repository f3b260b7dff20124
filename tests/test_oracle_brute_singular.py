"""Pin of the oracle's Sauter-Schwab integrals of the singular kernels
(Sec. 4.2, Eqs. kappa_S and kappa2_S: G1 = int int N_i N_j [s_a.t_b +
(s_a.R^)(R^.t_b)]/R and G2 = int int N_i N_j [(t_a.t_b)(n.R^) -
(t_a.R^)(n.t_b)]/R^2) on curved P2 element pairs of every touching class,
against a brute-force reference that shares no Sauter-Schwab map or
relabelling with it: the trial triangle is placed beside the test triangle in
one parameter plane (identity, folded across the shared edge, or reflected
through the shared corner), the pair integral is taken in relative polar
coordinates q = p + rho e(theta) (the factor rho cancels 1/R), and every
piece between the directions and radii where the overlap polygon changes
shape gets tensor Gauss-Legendre.  Both routes converge exponentially; they
must agree to 1e-9 of the largest entry at Ns = 20 (measured: 1e-14 ..
1e-11; on elements whose interpolated frame turns, Sauter-Schwab needs the
higher order: 4e-8 at Ns = 12, 4e-12 at Ns = 20)."""

import numpy as np
import pytest

import oracle
import workloads


def _pairs(om, e0):
    """One trial element per class (3 coincident, 2 common edge, 1 common
    vertex) for test element e0."""
    T = om.tri6[:, :3]
    found = {}
    for f in range(om.nt):
        c = len(set(T[e0]) & set(T[f]))
        if c and c not in found:
            found[c] = f
    return found


@pytest.mark.parametrize("mesh,frame_rule", [("spheroid_L1", 0), ("spheroid_L1", 1),
                                             ("sphere_L3", 0), ("oblate_L2", 1)])
def test_sauter_schwab_singular_integrals_match_brute_force(mesh, frame_rule):
    xyz, tri6 = {"spheroid_L1": lambda: workloads.spheroid_p2(1, 1.0, 1.5),
                 "sphere_L3": lambda: workloads.icosphere_p2(3),
                 "oblate_L2": lambda: workloads.spheroid_p2(2, 1.8, 1.0)}[mesh]()
    om = oracle.Mesh(xyz, tri6, frame_rule=frame_rule)
    nz = np.abs(om.frame()[:, 2])
    rng = np.random.default_rng(7)
    n_tight = 0
    for e0 in rng.choice(om.nt, 3, replace=False):
        pairs = _pairs(om, int(e0))
        assert sorted(pairs) == [1, 2, 3]
        for cls, f in pairs.items():
            cb, Gb = om.brute_singular(int(e0), f, 22)
            assert cb == cls
            scale = np.abs(Gb).max(axis=(0, 1))  # per component (4 x G1, 4 x G2)
            # the paper's frame rule switches its reference axis at |n.z| =
            # 0.9: a pair with nodes on both sides interpolates unrelated
            # nodal frames, its frame turns by O(1) inside the elements and
            # both routes lose their exponential rate (they still agree)
            nodes = np.concatenate([om.tri6[int(e0)], om.tri6[f]])
            side = nz[nodes] > 0.9
            turning = frame_rule == 0 and side.any() and not side.all()
            cases = ((False, 20, 1e-9), (True, 20, 1e-9), (False, 10, 1e-4))
            if turning:
                cases = ((False, 20, 1e-4), (True, 20, 1e-4))
            else:
                n_tight += 1
            for alt, ns, tol in cases:
                cs, Gs = om.ssq_singular(int(e0), f, ns, alt=alt)
                assert cs == cls
                err = np.abs(Gs - Gb).max(axis=(0, 1)) / scale
                assert err.max() <= tol, (mesh, cls, alt, ns, turning, err)
    assert n_tight >= 3


def test_brute_force_and_sauter_schwab_converge_exponentially():
    """On a smooth pair (level-3 sphere, polar frame rule, element 800: no
    turning frame) the brute-force route's error falls by about two orders
    of magnitude per two extra points per direction, and the Sauter-Schwab
    error against it falls geometrically in Ns (measured at Ns = 4, 6, 8:
    2e-5 .. 4e-5, 4e-8 .. 1.3e-7, 1.4e-10 .. 7e-10)."""
    xyz, tri6 = workloads.icosphere_p2(3)
    om = oracle.Mesh(xyz, tri6, frame_rule=1)
    for cls, f in _pairs(om, 800).items():
        ref = om.brute_singular(800, f, 20)[1]
        scale = np.abs(ref).max()
        d = [np.abs(om.brute_singular(800, f, n)[1] - ref).max() / scale for n in (3, 5, 7, 9)]
        assert all(d[k] > 30 * d[k + 1] for k in range(3)), (cls, d)
        assert d[3] < 1e-9, (cls, d)
        e = [np.abs(om.ssq_singular(800, f, ns)[1] - ref).max() / scale for ns in (2, 4, 6, 8)]
        assert all(e[k] > 30 * e[k + 1] for k in range(3)), (cls, e)
        assert e[3] < 1e-9, (cls, e)


def test_flat_pair_has_no_double_layer_part():
    """On a flat pair n.R^ = 0 and n.t_b = 0, so G2 vanishes identically; the
    brute force returns zeros to rounding for every class (a dropped or
    mis-signed term in the route would not)."""
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [-1, 1, 0]], float)
    # P2 nodes: corners + straight midpoints, three triangles in the plane z = 0
    corners = np.array([[0, 1, 2], [1, 3, 2], [0, 2, 4]])
    mids = {}
    pts = list(map(tuple, xyz))

    def mid(a, b):
        k = (min(a, b), max(a, b))
        if k not in mids:
            mids[k] = len(pts)
            pts.append(tuple((np.array(pts[a]) + np.array(pts[b])) / 2))
        return mids[k]

    tri6 = np.array([[a, b, c, mid(a, b), mid(b, c), mid(c, a)] for a, b, c in corners],
                    dtype=np.int32)
    # an open flat patch is not a closed surface, so build the oracle mesh
    # without the manifold checks the library makes: the oracle takes it
    om = oracle.Mesh(np.array(pts), tri6, morton=False)
    for f in range(3):
        c, G = om.brute_singular(0, f, 12)
        assert c >= 1
        assert np.abs(G[..., 4:]).max() <= 1e-13 * np.abs(G[..., :4]).max()
