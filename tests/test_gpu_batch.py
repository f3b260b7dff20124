"""Batched assembly (mueller_assemble_batch): many bodies with their own k_a,
eps_r and mu_r in one launch of each assembly kernel.

Every body of an FP64 batch is compared with the oracle's assembly of that
body alone (max |Z_gpu - Z_oracle| / max |Z_oracle| <= 1e-11 per quadrant,
right-hand sides <= 1e-13), and a mixed batch of uneven spheroids with the
single-body mixed assembly of each body (the same kernels; only the order of
the atomic additions differs: FP32 far part within 2e-6, FP64 near part
within 1e-12 of the quadrant maximum)."""

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


def quadrant_err(A, B):
    H = A.shape[0] // 2
    out = []
    for r in (slice(0, H), slice(H, None)):
        for c in (slice(0, H), slice(H, None)):
            ref = np.abs(B[r, c]).max()
            out.append(np.abs(A[r, c] - B[r, c]).max() / max(ref, 1e-300))
    return max(out)


BODIES = [
    # mesh, physics: one shared rule (q = 6, Sauter-Schwab order 5)
    (lambda: workloads.icosphere_p2(1), dict(ka=1.0, eps_r=(4.0, 0.0), mu_r=(1.0, 0.0))),
    (lambda: workloads.spheroid_p2(1, 1.0, 1.5), dict(ka=3.0, eps_r=(3.0, 0.2), mu_r=(1.2, 0.05))),
    (lambda: workloads.icosphere_p2(0), dict(ka=2.0, eps_r=(2.25, 0.0), mu_r=(1.0, 0.0))),
    (lambda: workloads.spheroid_p2(1, 1.4, 1.0), dict(ka=0.7, eps_r=(-2.0, 0.5), mu_r=(1.0, 0.0))),
]


def test_fp64_batch_matches_oracle_per_body():
    meshes, params, pws, incs = [], [], [], []
    for k, (mk, phys) in enumerate(BODIES):
        xyz, tri6 = mk()
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(0, out=False)
        meshes.append((m, xyz, tri6))
        params.append(mu.Params(ka=phys["ka"], eps_r=phys["eps_r"], mu_r=phys["mu_r"],
                                q_regular=6, ssq_order=5, frame_rule=0))
        pws.append(dict(phys, q_regular=6, ssq_order=5))
        incs.append(workloads.fibonacci_plane_waves(1 + k))
    out = mu.assemble_batch([m for m, _, _ in meshes], params, mu.MUELLER_C128, incs=incs)
    for (m, xyz, tri6), pw, inc, (Z, _, B) in zip(meshes, pws, incs, out):
        om = oracle.Mesh(xyz, tri6, frame_rule=0)
        err = quadrant_err(Z.cpu().numpy(), om.assemble(pw))
        assert err <= 1e-11, err
        Bo = om.rhs(pw, inc)
        berr = np.abs(B.cpu().numpy() - Bo).max() / np.abs(Bo).max()
        assert berr <= 1e-13, berr


def test_mixed_batch_of_uneven_spheroids_matches_single_body_assembly():
    spec = [b for b in workloads.multibody_spec() if b["level"] <= 2][:8]
    meshes, params, incs = [], [], []
    for b in spec:
        xyz, tri6 = workloads.multibody_mesh(b)
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(0, out=False)
        meshes.append(m)
        params.append(mu.Params(ka=b["ka"], eps_r=b["eps_r"], mu_r=b["mu_r"], q_regular=6,
                                ssq_order=5, frame_rule=0))
        incs.append(workloads.fibonacci_plane_waves(2))
    out = mu.assemble_batch(meshes, params, mu.MUELLER_C64_NEAR64, incs=incs)
    assert {m.nt for m in meshes} == {80, 320}
    for m, p, inc, (Z, near, B) in zip(meshes, params, incs, out):
        Z1, near1, B1 = mu.assemble(m, p, mu.MUELLER_C64_NEAR64, inc=inc)
        zf = quadrant_err(Z.cpu().numpy().astype(np.complex128),
                          Z1.cpu().numpy().astype(np.complex128))
        assert zf <= 2e-6, zf
        n0, n1 = near.cpu().numpy(), near1.cpu().numpy()
        assert np.abs(n0 - n1).max() <= 1e-12 * np.abs(n1).max()
        b0, b1 = B.cpu().numpy(), B1.cpu().numpy()
        assert np.abs(b0 - b1).max() <= 1e-14 * np.abs(b1).max()


def test_batch_rejects_bodies_with_different_rules():
    ms, ps = [], []
    for ns in (5, 4):
        xyz, tri6 = workloads.icosphere_p2(0)
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(0, out=False)
        ms.append(m)
        ps.append(mu.Params(ka=1.0, eps_r=(2.0, 0.0), ssq_order=ns))
    with pytest.raises(mu.MuellerError) as e:
        mu.assemble_batch(ms, ps, mu.MUELLER_C64_NEAR64)
    assert e.value.status == 1 and "body 1" in str(e.value)


@pytest.mark.parametrize("dtype", [mu.MUELLER_C128, mu.MUELLER_C64_NEAR64])
def test_batched_bodies_cross_sections_match_oracle_dense_solve(dtype):
    """The seeded multi-body workload's worst-balanced level-1 bodies (13, 15
    and 44 of multibody_spec: |C_ext - C_sca - C_abs| / C_ext up to 0.44, the
    discretisation error of an 80-triangle mesh at k_a ~ 5) batched with a
    level-2 body, each lit by the workload's 64 incidences, solved per body
    with block-Jacobi GMRES to 1e-10 (FP64 operator) or GMRES-IR to 1e-8
    (mixed operator, the benchmark's path), against the oracle's assembly,
    dense LU solve and far field of each body alone: cross sections within 1e-8
    (FP64) and 1e-6 (mixed) of the oracle's, the balance included."""
    spec = workloads.multibody_spec()
    pick = [13, 15, 44, next(i for i, b in enumerate(spec) if b["level"] == 2)]
    inc = workloads.fibonacci_plane_waves(32)
    meshes, params, raw = [], [], []
    for i in pick:
        b = spec[i]
        xyz, tri6 = workloads.multibody_mesh(b)
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(0, out=False)
        meshes.append(m)
        raw.append((xyz, tri6, b))
        params.append(mu.Params(ka=b["ka"], eps_r=b["eps_r"], mu_r=b["mu_r"], q_regular=6,
                                ssq_order=5, frame_rule=0))
    out = mu.assemble_batch(meshes, params, dtype, incs=[inc] * len(meshes))
    if dtype == mu.MUELLER_C128:
        opts, tol = mu.SolverOpts(mode=mu.SOLVE_GMRES, restart=50, tol=1e-10), 1e-8
    else:
        opts, tol = mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=50, tol=1e-8), 1e-6
    for m, p, (xyz, tri6, b), (Z, near, B) in zip(meshes, params, raw, out):
        op = mu.Operator(m, Z, near, dtype)
        mu.precond_build(op, min(256, m.N // 2))
        X, info = mu.solve(op, B, opts)
        assert info["converged"] == inc.shape[0]
        _, xs = mu.far_field(m, p, X, inc)
        om = oracle.Mesh(xyz, tri6, frame_rule=0)
        pw = dict(ka=b["ka"], eps_r=b["eps_r"], mu_r=b["mu_r"], q_regular=6, ssq_order=5)
        Zo = om.assemble(pw)
        Xo = np.linalg.solve(Zo, om.rhs(pw, inc).T).T  # dense LU (LAPACK)
        xso = om.far_field(pw, Xo, inc)[1]
        scale = np.abs(xso[:, :1])  # per incidence, relative to C_ext
        assert np.abs(xs - xso).max(axis=0).max() <= tol * scale.max(), (np.abs(xs - xso) / scale).max()
        assert np.all(np.abs(xs - xso) <= tol * scale)
        bal = np.abs(xs[:, 0] - xs[:, 1] - xs[:, 2]) / np.abs(xs[:, 0])
        bal_o = np.abs(xso[:, 0] - xso[:, 1] - xso[:, 2]) / np.abs(xso[:, 0])
        np.testing.assert_allclose(bal, bal_o, rtol=0, atol=3 * tol)


@pytest.mark.parametrize("dtype", [mu.MUELLER_C128, mu.MUELLER_C64_NEAR64])
def test_batched_block_jacobi_matches_per_body_builds(dtype):
    """mueller_precond_build_batch factorises the blocks of uneven bodies in
    one batched LU: each body's preconditioner equals the one built for it
    alone (same kernels, block by block: FP64 inverses to 1e-13, complex64
    inverses to FP32 rounding), and a solve with it takes the same number of
    iterations."""
    spec = workloads.multibody_spec()
    pick = [13, 15, next(i for i, b in enumerate(spec) if b["level"] == 2),
            next(i for i, b in enumerate(spec) if b["level"] == 3)]
    ops, Bs, blocks = [], [], []
    inc = workloads.fibonacci_plane_waves(1)
    for i in pick:
        b = spec[i]
        xyz, tri6 = workloads.multibody_mesh(b)
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(0, out=False)
        p = mu.Params(ka=b["ka"], eps_r=b["eps_r"], mu_r=b["mu_r"], ssq_order=3, frame_rule=0)
        Z, near, B = mu.assemble(m, p, dtype, inc=inc)
        ops.append(mu.Operator(m, Z, near, dtype))
        Bs.append(B)
        blocks.append(min(128, m.N // 2))
    batch = [P.clone() for P in mu.precond_build_batch(ops, blocks)]
    elem = 16 if dtype == mu.MUELLER_C128 else 8
    cdt = torch.complex128 if dtype == mu.MUELLER_C128 else torch.complex64
    tol = 1e-13 if dtype == mu.MUELLER_C128 else 1e-5
    opts = mu.SolverOpts(mode=mu.SOLVE_GMRES if dtype == mu.MUELLER_C128 else mu.SOLVE_GMRES_IR,
                         restart=30, tol=1e-8)
    for op, B, blk, Pb in zip(ops, Bs, blocks, batch):
        op.precond = Pb
        Xb, ib = mu.solve(op, B, opts)
        Ps = mu.precond_build(op, blk)
        Xs, is_ = mu.solve(op, B, opts)
        H = op.mesh.N // 2
        nb, d = (H + blk - 1) // blk, 2 * min(blk, H)
        n_inv = nb * d * d  # inverses [nb][d][d], then int32 sizes[nb]
        a = Pb[: n_inv * elem].view(cdt)
        c = Ps[: n_inv * elem].view(cdt)
        assert torch.equal(Pb[n_inv * elem: n_inv * elem + 4 * nb],
                           Ps[n_inv * elem: n_inv * elem + 4 * nb])  # block sizes
        err = ((a - c).abs().max() / c.abs().max()).item()
        assert err <= tol, err
        assert abs(ib["iters"] - is_["iters"]) <= 1 and ib["relres"] <= 1e-8
        e = (torch.linalg.norm(Xb - Xs) / torch.linalg.norm(Xs)).item()
        assert e <= 1e-6, e


def test_batched_block_jacobi_refuses_bad_arguments():
    xyz, tri6 = workloads.icosphere_p2(0)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(0, out=False)
    Z, near, _ = mu.assemble(m, mu.Params(ka=1.0, eps_r=(2.0, 0.0), ssq_order=2),
                             mu.MUELLER_C64_NEAR64)
    ops = [mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64), mu.Operator(m, Z, None, mu.MUELLER_C64_NEAR64)]
    with pytest.raises(mu.MuellerError) as e:
        mu.precond_build_batch(ops, [8, 8])
    assert e.value.status == 1 and "body 1" in str(e.value)
