"""GPU checks at the workload sizes: the level-4 plasmonic sphere with 16
right-hand sides (N = 40968, complex64 Z of 13.4 GB + FP64 near part), the
level-3 spheroid, and the small sphere against Mie."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402
from oracle import mie  # noqa: E402

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
]


def _pw(w):
    return dict(ka=w["ka"], eps_r=w["eps_r"], mu_r=w["mu_r"], q_regular=w["q_regular"],
                ssq_order=w["ssq_order"])


def test_level4_plasmonic_sphere_16_rhs():
    xyz, tri6, inc, w = workloads.workload("sphere_L4_eps-10+1i_ka10")
    assert inc.shape == (16, 6)
    p = mu.Params.from_workload(w)
    m = mu.Mesh(xyz, tri6)
    assert m.N == 40968
    m.tangent_frame(p.frame_rule, out=False)
    # sampled rows of the FP64 operator against the oracle (the last node is
    # the ragged end of the Morton order)
    om = oracle.Mesh(xyz, tri6)
    rng = np.random.default_rng(4)
    nodes = np.sort(rng.choice(m.nn, 4, replace=False))
    nodes[-1] = m.nn - 1
    rows_o = om.assemble(_pw(w), rows=nodes)
    H = m.N // 2
    idx = np.array([[h * H + 2 * n + a for h in (0, 1) for a in (0, 1)] for n in nodes]).ravel()
    Z64, _, _ = mu.assemble(m, p, mu.MUELLER_C128)
    rows_g = Z64[torch.from_numpy(idx).cuda()].cpu().numpy()
    del Z64
    torch.cuda.empty_cache()
    assert np.abs(rows_g - rows_o).max() <= 1e-11 * np.abs(rows_o).max()
    # mixed-precision solve of all 16 right-hand sides
    Z, near, B = mu.assemble(m, p, mu.MUELLER_C64_NEAR64, inc=inc)
    op = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    mu.precond_build(op, int(w["block"]))
    X, info = mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=50, tol=1e-8))
    assert info["converged"] == 16 and info["relres"] <= 1e-8
    R = B - mu.matvec(op, X)
    rel = (torch.linalg.norm(R, dim=1) / torch.linalg.norm(B, dim=1)).max().item()
    assert rel <= 1e-8, rel
    _, xs = mu.far_field(m, p, X, inc)
    # a sphere: every incidence gives the same cross sections, up to the
    # discretisation (the mesh and the frame are not rotation invariant)
    assert np.ptp(xs[:, 0]) <= 2e-2 * xs[0, 0]
    # energy balance and Mie, to discretisation accuracy
    assert np.abs(xs[:, 0] - xs[:, 1] - xs[:, 2]).max() <= 0.05 * xs[0, 0]
    ref = mie.mie_bh(w["ka"], complex(*w["eps_r"]))
    assert abs(xs[:, 0].mean() - ref[0]) <= 0.05 * ref[0], (xs[:, 0].mean(), ref)


def _mie_errors(level, q=6, ns=5, frame_rule=mu.FRAME_POLAR):
    xyz, tri6 = workloads.icosphere_p2(level)
    p = mu.Params(ka=1.0, eps_r=(4.0, 0.0), q_regular=q, ssq_order=ns, frame_rule=frame_rule)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule, out=False)
    inc = workloads.plane_wave()
    Z, near, B = mu.assemble(m, p, mu.MUELLER_C64_NEAR64, inc=inc)
    op = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    mu.precond_build(op, 256)
    X, info = mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, tol=1e-10))
    _, xs = mu.far_field(m, p, X, inc)
    del Z, near, op
    m.free()
    torch.cuda.empty_cache()
    ref = mie.mie_bh(1.0, 4.0)
    return np.abs(xs[0] - ref) / ref[0]  # C_ext, C_sca, C_abs (Mie: 0) errors


def test_small_sphere_converges_to_mie_with_polar_frames():
    """Config-1 physics (eps_r = 4, k_a = 1) on the level-2, 3 and 4 spheres
    (N = 2568, 10248, 40968), polar frame rule, Q = 6, Ns = 5, mixed path to
    a 1e-10 FP64 residual.  Measured errors of C_ext: 1.4e-3, 2.7e-4,
    5.2e-5 (h^2.4 per level); an error of 1e-4 is met at level 4, not
    at level 3 (Q = 12 gives 1.7e-4 there; Ns = 8 changes nothing, so the
    Sauter-Schwab error is not what limits it).  Every error falls at least
    as h^1.9 (C_sca and C_abs measured at h^2.0 .. h^2.3)."""
    errs = [_mie_errors(L) for L in (2, 3, 4)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes >= 1.9), (errs, slopes)
    assert errs[1][0] <= 4e-4 and errs[2][0] <= 1e-4, errs
