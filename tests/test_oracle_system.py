"""System-level pins of the oracle: Mie series, optical theorem, Galerkin
reciprocity, zero contrast, translation invariance, LU vs GMRES + MBJ.
(Sec. 4.3 Eq. global_system, Sec. 5, Sec. 6.2)"""

import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import mie

P1 = dict(ka=1.0, eps_r=(4.0, 0.0), mu_r=(1.0, 0.0), q_regular=6, ssq_order=5)
INC = workloads.plane_wave((0, 0, 1), (1, 0, 0))


# ------------------------------------------------------------------ Mie
@pytest.mark.parametrize("ka,er", [(1.0, 4.0), (5.0, 2.25), (10.0, -10 + 1j), (0.5, 2 + 0.3j),
                                   (3.0, 3 + 0.2j)])
def test_mie_two_independent_evaluations_agree(ka, er):
    a = mie.mie_bh(ka, er)
    b = mie.mie_scipy(ka, er)
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)
    if np.imag(er) == 0 and np.real(er) > 0:
        assert abs(a[2]) < 1e-12 * a[0]  # lossless: C_abs = 0


def test_mie_rayleigh_limit():
    # x << 1: C_sca = (8 pi/3) x^4 |(m^2-1)/(m^2+2)|^2 a^2, C_abs = 4 pi x Im(...) a^2
    for er in (4.0, 2 + 0.5j, -3 + 1j):
        x = 1e-3
        cext, csca, cabs = mie.mie_bh(x, er)
        al = (er - 1) / (er + 2)
        np.testing.assert_allclose(csca, 8 * math.pi / 3 * x ** 4 * abs(al) ** 2, rtol=1e-4)
        if np.imag(er) != 0:
            np.testing.assert_allclose(cabs, 4 * math.pi * x * np.imag(al), rtol=1e-4)


# --------------------------------------------------------- full pipeline
def _solve(level, p, inc=INC, frame_rule=1):
    xyz, tri6 = workloads.icosphere_p2(level)
    m = oracle.Mesh(xyz, tri6, frame_rule=frame_rule)
    Z = m.assemble(p)
    B = m.rhs(p, inc)
    X = np.linalg.solve(Z, B.T).T
    return m, Z, B, X


def test_cross_sections_converge_to_mie():
    """Config-1 physics (eps_r = 4, k_a = 1), polar frame rule, Q = 6,
    Ns = 5: the errors of C_ext, C_sca and C_abs (exactly 0 for this
    lossless sphere) against Mie fall at least as h^1.9 from level 1 to 2
    (measured slopes 2.0, 2.3, 2.2; the GPU table to level 4 gives 2.0-2.4:
    the frame turns by O(1) inside the elements around the poles, so the
    current components there are represented only to O(1) on an O(h^2)
    area), and the energy balance holds to discretisation accuracy."""
    ref = mie.mie_bh(P1["ka"], P1["eps_r"][0])
    errs = []
    for L in (1, 2):
        m, Z, B, X = _solve(L, P1)
        _, xs = m.far_field(P1, X, INC)
        errs.append(np.abs(xs[0] - ref) / ref[0])
        assert abs(xs[0, 0] - xs[0, 1] - xs[0, 2]) / xs[0, 0] < 0.05
    slopes = np.log2(errs[0] / errs[1])  # h halves per level
    assert np.all(slopes >= 1.9), (errs, slopes)
    assert errs[1][0] < 2e-3, errs


def test_zero_contrast_scatters_nothing():
    # eps_r = mu_r = 1: K1 = K2 = 0 and Z is the mass matrix; the radiated
    # field of the projected incident currents vanishes up to discretisation.
    p = dict(P1, eps_r=(1.0, 0.0))
    amps = []
    for L in (2, 3):
        xyz, tri6 = workloads.icosphere_p2(L)
        m = oracle.Mesh(xyz, tri6, frame_rule=1)
        if L == 2:
            Z = m.assemble(p)
            M = m.mass(p["q_regular"])
            H = m.N // 2
            # the operator blocks vanish; only a_chi M remains off-diagonal
            assert np.abs(Z[:H, :H]).max() < 1e-14 and np.abs(Z[H:, H:]).max() < 1e-14
            np.testing.assert_allclose(Z[:H, H:][0::2, 0::2].real, M, atol=1e-14)
        B = m.rhs(p, INC)
        M = m.mass(p["q_regular"])
        H = m.N // 2
        X = np.zeros(m.N, complex)
        X[:H] = np.linalg.solve(M, B[0, H:].reshape(-1, 2)).ravel()
        X[H:] = np.linalg.solve(M, B[0, :H].reshape(-1, 2)).ravel()
        F, xs = m.far_field(p, X, INC, dirs=workloads.fibonacci_directions(16))
        amps.append(np.abs(F).max())
    assert amps[1] < 3e-4 and amps[1] < amps[0] / 3, amps


def test_galerkin_reciprocity_of_K1():
    # With s_1 = -t_2, s_2 = t_1 (t_2 = n x t_1): K1 = S T per node with
    # S = [[0,-1],[1,0]] and T symmetric under (x, i, alpha) <-> (y, j, beta)
    # because S1, S2 depend on R only.  Checked pair by pair: the local
    # block of (ex, ey) against the transposed block of (ey, ex).  Regular,
    # coincident and vertex pairs are symmetric to round-off (their
    # quadratures are symmetric); common-edge Sauter-Schwab is symmetric to
    # quadrature accuracy, checked where the interpolated frame is smooth
    # (all nodal t1 of the pair within 30 degrees of each other).
    xyz, tri6 = workloads.icosphere_p2(2)
    m = oracle.Mesh(xyz, tri6, frame_rule=1)
    p = dict(P1, q_regular=12, ssq_order=10)
    fr = m.frame()
    S = np.array([[0.0, -1.0], [1.0, 0.0]])

    def T_of(L):
        return np.einsum("ga,ijgb->ijab", S, L[:, :, :4].reshape(6, 6, 2, 2))

    seen = {0: 0, 1: 0, 2: 0, 3: 0}
    for ex in range(0, m.nt, 16):
        for ey in range(m.nt):
            c, Lxy = m.pair_block(p, ex, ey)
            _, Lyx = m.pair_block(p, ey, ex)
            A = T_of(Lxy)
            B = T_of(Lyx).transpose(1, 0, 3, 2)
            d = np.abs(A - B).max() / np.abs(A).max()
            if c == 2:
                t1 = fr[np.concatenate([m.tri6[ex], m.tri6[ey]]), 3:6]
                if (t1 @ t1.T).min() < np.cos(np.radians(30)):
                    continue
                assert d < 1e-7, (ex, ey, d)
            else:
                assert d < 1e-12, (ex, ey, c, d)
            seen[c] += 1
    assert min(seen.values()) > 0, seen


def test_z_is_translation_invariant():
    xyz, tri6 = workloads.icosphere_p2(1)
    shift = np.array([0.25, -0.5, 0.125])
    m1 = oracle.Mesh(xyz, tri6, frame_rule=1)
    m2 = oracle.Mesh(xyz + shift, tri6, frame_rule=1)
    Z1, Z2 = m1.assemble(P1), m2.assemble(P1)

    def orig(m, Z):
        # back to the input node order
        idx = np.concatenate([2 * m.node_perm[:, None] + np.arange(2)[None]]).ravel()
        nn = m.nn
        full = np.concatenate([idx, 2 * nn + idx])
        out = np.empty_like(Z)
        out[np.ix_(full, full)] = Z
        return out

    A, B = orig(m1, Z1), orig(m2, Z2)
    assert np.abs(A - B).max() < 1e-12 * np.abs(A).max()


def test_dense_lu_and_gmres_with_block_jacobi_agree():
    m, Z, B, X = _solve(1, P1)
    Xlu = oracle.lu_solve(Z, B)
    np.testing.assert_allclose(Xlu, X, rtol=0, atol=1e-11 * np.abs(X).max())
    for block in (64, 100, 1000):
        x, info = oracle.gmres(Z, B[0], block=block, restart=30, tol=1e-12)
        assert info["converged"]
        assert np.linalg.norm(x - Xlu[0]) < 1e-10 * np.linalg.norm(Xlu[0])
        if block >= m.N // 2:
            assert info["iters"] == 1  # one block = exact inverse
    x0, info0 = oracle.gmres(Z, B[0], block=0, restart=30, tol=1e-10)
    x1, info1 = oracle.gmres(Z, B[0], block=64, restart=30, tol=1e-10)
    assert info1["iters"] < info0["iters"]


def test_mbj_blocks_follow_morton_clusters():
    # Eq. (precond_block): a block is the restriction of Z to I_m in both halves
    m, Z, B, X = _solve(1, P1)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(m.N) + 1j * rng.standard_normal(m.N)
    Bk = 50
    out = oracle.mbj_apply(Z, Bk, v)
    H = m.N // 2
    for b0 in range(0, H, Bk):
        I = np.arange(b0, min(b0 + Bk, H))
        idx = np.concatenate([I, H + I])
        np.testing.assert_allclose(Z[np.ix_(idx, idx)] @ out[idx], v[idx], atol=1e-10)


def test_scattering_amplitude_reciprocity():
    # p2 . F(k2; k1, p1) = p1 . F(-k1; -k2, p2)
    k1 = np.array([0.0, 0.0, 1.0]); p1 = np.array([1.0, 0.0, 0.0])
    k2 = np.array([0.6, 0.0, 0.8]); p2 = np.array([0.8, 0.0, -0.6])
    inc = np.stack([np.concatenate([k1, p1]), np.concatenate([-k2, p2])])
    m, Z, B, X = _solve(2, dict(P1, q_regular=12), inc)
    F1, _ = m.far_field(P1, X[0], inc[0], dirs=k2[None])
    F2, _ = m.far_field(P1, X[1], inc[1], dirs=-k1[None])
    a = p2 @ F1[0, 0]
    b = p1 @ F2[0, 0]
    assert abs(a - b) < 2e-2 * abs(a), (a, b)
