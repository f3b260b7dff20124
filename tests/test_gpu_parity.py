"""GPU parity: the CUDA path through the C ABI against the oracle, element
by element, on seeded synthetic meshes.

Tolerances (FP64 path): max |Z_gpu - Z_oracle| / max |Z_oracle| <= 1e-11 per
2 x 2 quadrant of Z (matrix entries that vanish by symmetry make a pure
entry-wise relative test meaningless).  Mixed path: regular pairs are
computed in FP32, so the complex64 far part is compared at 5e-6 of the
quadrant maximum; the FP64 near part (touching pairs + mass) at 1e-11.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
]

CASES = {
    # name: (mesh builder, physics, q, ns, frame rule)
    "sphere_L1_eps4": (lambda: workloads.icosphere_p2(1),
                       dict(ka=1.0, eps_r=(4.0, 0.0), mu_r=(1.0, 0.0)), 6, 5, 0),
    "spheroid_L2_lossy_q12": (lambda: workloads.spheroid_p2(2, 1.0, 1.5),
                              dict(ka=3.0, eps_r=(3.0, 0.2), mu_r=(1.0, 0.0)), 12, 4, 1),
    "sphere_L1_plasmonic_magnetic": (lambda: workloads.icosphere_p2(1),
                                     dict(ka=10.0, eps_r=(-10.0, 1.0), mu_r=(1.5, 0.1)), 6, 3, 0),
    "icosahedron_L0_ssq1": (lambda: workloads.icosphere_p2(0),
                            dict(ka=2.0, eps_r=(2.25, 0.0), mu_r=(1.0, 0.0)), 6, 1, 1),
    "icosahedron_L0_ssq16": (lambda: workloads.icosphere_p2(0),
                             dict(ka=0.5, eps_r=(6.0, 1.0), mu_r=(1.0, 0.0)), 12, 16, 0),
}

_cache = {}


def case(name):
    if name in _cache:
        return _cache[name]
    mk, phys, q, ns, rule = CASES[name]
    xyz, tri6 = mk()
    pw = dict(phys, q_regular=q, ssq_order=ns)
    om = oracle.Mesh(xyz, tri6, frame_rule=rule)
    Zo = om.assemble(pw)
    p = mu.Params(ka=phys["ka"], eps_r=phys["eps_r"], mu_r=phys["mu_r"], q_regular=q,
                  ssq_order=ns, frame_rule=rule)
    _cache[name] = (xyz, tri6, pw, om, Zo, p)
    return _cache[name]


def quadrant_err(A, B):
    H = A.shape[0] // 2
    out = []
    for r in (slice(0, H), slice(H, None)):
        for c in (slice(0, H), slice(H, None)):
            ref = np.abs(B[r, c]).max()
            out.append(np.abs(A[r, c] - B[r, c]).max() / max(ref, 1e-300))
    return max(out)


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_morton_permutations_are_bit_exact(level):
    xyz, tri6 = workloads.icosphere_p2(level)
    m = mu.Mesh(xyz, tri6)
    npm, epm = m.perm()
    onp, oep = oracle.morton(xyz, tri6)
    np.testing.assert_array_equal(npm, onp)
    np.testing.assert_array_equal(epm, oep)
    info = m.info()
    assert info["n_dof"] == 4 * len(xyz)
    # touching pairs: 1 coincident + 3 edge + (sum over corners of valence - 3) vertex
    assert info["n_touching"] > 4 * len(tri6)


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("level", [1, 3])
def test_tangent_frame_matches_oracle(level, rule):
    xyz, tri6 = workloads.spheroid_p2(level, 1.0, 1.5)
    m = mu.Mesh(xyz, tri6)
    fr = m.tangent_frame(rule).cpu().numpy()
    om = oracle.Mesh(xyz, tri6, frame_rule=rule)
    np.testing.assert_allclose(fr, om.frame(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_assembly_matches_oracle(name):
    xyz, tri6, pw, om, Zo, p = case(name)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule)
    inc = workloads.fibonacci_plane_waves(2)
    Z, _, B = mu.assemble(m, p, mu.MUELLER_C128, inc=inc)
    Zg = Z.cpu().numpy()
    err = quadrant_err(Zg, Zo)
    assert err <= 1e-11, err
    Bo = om.rhs(pw, inc)
    berr = np.abs(B.cpu().numpy() - Bo).max() / np.abs(Bo).max()
    assert berr <= 1e-13, berr


@pytest.mark.parametrize("name", ["sphere_L1_eps4", "spheroid_L2_lossy_q12"])
def test_mixed_operator_matches_oracle(name):
    xyz, tri6, pw, om, Zo, p = case(name)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule)
    Z, near, _ = mu.assemble(m, p, mu.MUELLER_C64_NEAR64)
    Zf = Z.cpu().numpy().astype(np.complex128)
    # the dense operator Z_far + near, column block by column block
    N = m.N
    op = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    E = torch.eye(N, dtype=torch.complex128, device="cuda")
    cols = []
    for k0 in range(0, N, 512):
        Xb = E[k0:k0 + 512].contiguous()
        cols.append(mu.matvec(op, Xb).cpu().numpy())
    Zm = np.concatenate(cols, axis=0).T  # row i of Xb -> column of Z
    err = quadrant_err(Zm, Zo)
    assert err <= 5e-6, err
    # the far part alone carries only FP32 rounding: near part is exact FP64
    near_only = Zm - Zf
    regular_oracle = Zo - near_only
    assert quadrant_err(Zf, regular_oracle) <= 5e-6


def test_fp64_matvec_matches_numpy():
    xyz, tri6, pw, om, Zo, p = case("spheroid_L2_lossy_q12")
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule)
    Z, _, _ = mu.assemble(m, p, mu.MUELLER_C128)
    op = mu.Operator(m, Z, dtype=mu.MUELLER_C128)
    g = torch.Generator(device="cpu").manual_seed(5)
    X = torch.randn((3, m.N), dtype=torch.complex128, generator=g).cuda()
    Y = mu.matvec(op, X).cpu().numpy()
    ref = X.cpu().numpy() @ Z.cpu().numpy().T
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_dense_lu_solve_matches_oracle():
    xyz, tri6, pw, om, Zo, p = case("sphere_L1_eps4")
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule)
    inc = workloads.fibonacci_plane_waves(3)
    Z, _, B = mu.assemble(m, p, mu.MUELLER_C128, inc=inc)
    op = mu.Operator(m, Z, dtype=mu.MUELLER_C128)
    X, info = mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_DENSE_LU, use_precond=0))
    Xo = oracle.lu_solve(Zo, om.rhs(pw, inc))
    err = np.abs(X.cpu().numpy() - Xo).max() / np.abs(Xo).max()
    assert err <= 1e-10, err


@pytest.mark.parametrize("block", [37, 100, 256])
def test_gmres_fp64_with_block_jacobi_matches_oracle(block):
    xyz, tri6, pw, om, Zo, p = case("spheroid_L2_lossy_q12")
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule)
    inc = workloads.plane_wave((0, 0, 1), (1, 0, 0))
    Z, _, B = mu.assemble(m, p, mu.MUELLER_C128, inc=inc)
    op = mu.Operator(m, Z, dtype=mu.MUELLER_C128)
    mu.precond_build(op, block)
    X, info = mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_GMRES, restart=20, tol=1e-10))
    Bo = om.rhs(pw, inc)
    xo, oinfo = oracle.gmres(Zo, Bo[0], block=block, restart=20, tol=1e-10)
    Xd = np.linalg.solve(Zo, Bo[0])
    err = np.linalg.norm(X.cpu().numpy()[0] - Xd) / np.linalg.norm(Xd)
    assert err <= 1e-8, err
    assert info["converged"] == 1 and info["relres"] <= 1e-10
    assert abs(info["iters"] - oinfo["iters"]) <= 1, (info, oinfo)


def test_gmres_ir_mixed_reaches_fp64_accuracy():
    xyz, tri6, pw, om, Zo, p = case("spheroid_L2_lossy_q12")
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule)
    inc = workloads.fibonacci_plane_waves(1)
    Z64, _, B = mu.assemble(m, p, mu.MUELLER_C128, inc=inc)
    op64 = mu.Operator(m, Z64, dtype=mu.MUELLER_C128)
    mu.precond_build(op64, 64)
    X64, _ = mu.solve(op64, B, mu.SolverOpts(mode=mu.SOLVE_GMRES, restart=30, tol=1e-10))
    Z32, near, _ = mu.assemble(m, p, mu.MUELLER_C64_NEAR64)
    op = mu.Operator(m, Z32, near, mu.MUELLER_C64_NEAR64)
    mu.precond_build(op, 64)
    X, info = mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=30, tol=1e-8))
    assert info["converged"] == 2 and info["relres"] <= 1e-8
    # residual against the stored operator, in FP64
    R = B - mu.matvec(op, X)
    rel = (torch.linalg.norm(R, dim=1) / torch.linalg.norm(B, dim=1)).max().item()
    assert rel <= 1e-8, rel
    # solution of the mixed operator vs the FP64 operator
    e = (torch.linalg.norm(X - X64, dim=1) / torch.linalg.norm(X64, dim=1)).max().item()
    assert e <= 1e-5, e


def test_far_field_matches_oracle():
    xyz, tri6, pw, om, Zo, p = case("spheroid_L2_lossy_q12")
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule)
    inc = workloads.fibonacci_plane_waves(1)
    Bo = om.rhs(pw, inc)
    Xo = np.linalg.solve(Zo, Bo.T).T
    X = torch.from_numpy(Xo).cuda()
    dirs = workloads.fibonacci_directions(7)
    F, xs = mu.far_field(m, p, X, inc, dirs=dirs, n_theta=24, n_phi=48)
    Fo, xso = om.far_field(pw, Xo, inc, dirs=dirs, n_theta=24, n_phi=48)
    np.testing.assert_allclose(F.cpu().numpy(), Fo, rtol=0, atol=1e-12 * np.abs(Fo).max())
    np.testing.assert_allclose(xs, xso, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("ka", [0.5, 60.0, 4.0e4])
@pytest.mark.parametrize("r,n_phi", [(1, 16), (1, 15), (3, 16), (3, 15)])
def test_far_field_phase_range_matches_oracle(ka, r, n_phi):
    """Random currents, so that every phase exp(-i k r.y) counts: k a = 60
    spans many periods of the table-driven exp(i th), 4e4 (|th| beyond
    2^20 pi/128) the sincos branch.  One RHS with an even n_phi takes the
    antipodal-pair kernel, an odd n_phi the per-direction one; three RHS
    take the pair kernel two RHS per CTA (a partial group) with an even
    n_phi, the multi-RHS kernel four per CTA with an odd one.  Both sides form th = k r.y in FP64 with its rounding
    of a few ulp(|th|), so the bound is 1e-12 of max |F| or 50 k a eps,
    whichever is larger."""
    xyz, tri6 = workloads.icosphere_p2(1)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(0, out=False)
    mu.assemble(m, mu.Params(ka=1.0, eps_r=(2.0, 0.0), ssq_order=2, frame_rule=0),
                mu.MUELLER_C128)  # point geometry of the rule
    p = mu.Params(ka=ka, eps_r=(2.0, 0.0), ssq_order=2, frame_rule=0)
    inc = workloads.fibonacci_plane_waves(2)[:r]
    rng = np.random.default_rng(11)
    X = rng.standard_normal((r, m.N)) + 1j * rng.standard_normal((r, m.N))
    dirs = workloads.fibonacci_directions(9)
    F, xs = mu.far_field(m, p, torch.from_numpy(X).cuda(), inc, dirs=dirs, n_theta=9, n_phi=n_phi)
    om = oracle.Mesh(xyz, tri6, frame_rule=0)
    pw = dict(ka=ka, eps_r=(2.0, 0.0), mu_r=(1.0, 0.0), q_regular=6, ssq_order=2)
    Fo, xso = om.far_field(pw, X, inc, dirs=dirs, n_theta=9, n_phi=n_phi)
    tol = max(1e-12, 50.0 * ka * np.finfo(float).eps)
    np.testing.assert_allclose(F.cpu().numpy(), Fo, rtol=0, atol=tol * np.abs(Fo).max())
    np.testing.assert_allclose(xs[:, :2], xso[:, :2], rtol=tol, atol=0)
    np.testing.assert_allclose(xs[:, 2], xso[:, 2], rtol=1e-11, atol=1e-14 * np.abs(xso).max())


def test_sampled_rows_at_level3_workload():
    # the benchmark's workload size (level-3 sphere, N = 10248): rows of Z
    # for sampled test nodes, FP64 and mixed storage
    xyz, tri6, inc, w = workloads.workload("sphere_L3_eps2.25_ka5")
    p = mu.Params.from_workload(w)
    pw = dict(ka=w["ka"], eps_r=w["eps_r"], mu_r=w["mu_r"], q_regular=w["q_regular"],
              ssq_order=w["ssq_order"])
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule)
    om = oracle.Mesh(xyz, tri6)
    rng = np.random.default_rng(11)
    nodes = np.sort(rng.choice(m.nn, 6, replace=False))
    nodes[-1] = m.nn - 1  # ragged tail
    rows_o = om.assemble(pw, rows=nodes)
    H = m.N // 2
    idx = np.array([[h * H + 2 * n + a for h in (0, 1) for a in (0, 1)] for n in nodes]).ravel()
    Z, _, _ = mu.assemble(m, p, mu.MUELLER_C128)
    rows_g = Z[torch.from_numpy(idx).cuda()].cpu().numpy()
    del Z
    scale = np.abs(rows_o).max()
    assert np.abs(rows_g - rows_o).max() <= 1e-11 * scale
    # whole rows of the mixed operator: the complex64 far part read from Z
    # plus the FP64 near blocks of those test nodes (near-block layout)
    Z32, near, _ = mu.assemble(m, p, mu.MUELLER_C64_NEAR64)
    far_rows = Z32[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    rowptr, col, _ = m.near_layout()
    blocks = near.cpu().numpy().reshape(-1, 2, 2, 2, 2)
    del Z32, near
    near_rows = np.zeros_like(far_rows)
    for k, n in enumerate(nodes):
        for q in range(rowptr[n], rowptr[n + 1]):
            j = col[q]
            for h in (0, 1):
                for a in (0, 1):
                    for g in (0, 1):
                        for b in (0, 1):
                            near_rows[4 * k + 2 * h + a, g * H + 2 * j + b] = blocks[q, h, a, g, b]
    mixed_rows = far_rows + near_rows
    # the only difference from the oracle is the FP32 rounding of the far
    # part (regular element pairs): within 5e-6 of the largest entry
    # overall, and entry by entry within a few FP32 roundings of the entry
    # (plus 1e-7 of the largest, for entries that cancel)
    d = np.abs(mixed_rows - rows_o)
    assert d.max() <= 5e-6 * scale, d.max() / scale
    assert np.all(d <= 4e-6 * np.abs(rows_o) + 1e-7 * scale)
    # the near blocks carry the singular and mass parts: leaving them out is
    # far outside that bound
    assert np.abs(far_rows - rows_o).max() > 1e-3 * scale


def test_mirrored_inner_products_match_full_read():
    """Z11 = -Z00 bit for bit as assembled, so the inner GMRES's complex64
    product may read three quarters of Z (MUELLER_OP_K1_MIRRORED, set for an
    assembled Z and void once Z changes in place).  The mixed GMRES-IR solve
    with it and with the full read differ only in the order of FP32 sums:
    both reach the FP64 residual 1e-8, with iteration counts within one and
    solutions within 1e-6 of each other."""
    xyz, tri6 = workloads.spheroid_p2(2, 1.0, 1.5)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(0, out=False)
    p = mu.Params(ka=2.0, eps_r=(3.0, 0.1), ssq_order=3, frame_rule=0)
    inc = workloads.fibonacci_plane_waves(1)[:1]
    Z, near, B = mu.assemble(m, p, mu.MUELLER_C64_NEAR64, inc=inc)
    H = m.N // 2
    assert torch.equal(Z[H:, H:], -Z[:H, :H])
    op_m = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    op_f = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64, mirrored=False)
    assert op_m.mirrored and not op_f.mirrored
    assert not mu.Operator(m, Z.clone(), near, mu.MUELLER_C64_NEAR64).mirrored  # untagged copy
    opts = mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=30, tol=1e-8)
    out = []
    for op in (op_m, op_f):
        mu.precond_build(op, 64)
        X, info = mu.solve(op, B, opts)
        assert info["converged"] == 1 and info["relres"] <= 1e-8
        out.append((X, info["iters"]))
    assert abs(out[0][1] - out[1][1]) <= 1
    e = (torch.linalg.norm(out[0][0] - out[1][0]) / torch.linalg.norm(out[1][0])).item()
    assert e <= 1e-6, e
    Z[0, 0] += 1.0  # changed in place: the tag no longer holds
    assert not op_m.mirrored
