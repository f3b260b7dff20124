"""The lockstep mixed-precision solver at small sizes.

The Arnoldi step runs as one thread-block cluster per right-hand side, of
1 to 16 CTAs by the vector length. This file checks that:

* the cluster sizes 1, 2 and 8 solve each right-hand side to the FP64
  residual tolerance against the stored operator (level-0 icosahedron,
  N = 168; level-1 sphere, N = 648; level-2 spheroid, N = 2568);
* several right-hand sides solved together (the last cluster of each step
  decides the stop flag) equal the same right-hand sides solved one by one;
* a zero right-hand side among them gives a zero solution, counts as
  converged and leaves the others untouched.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
]

MESHES = {
    "icosahedron_L0": lambda: workloads.icosphere_p2(0),
    "sphere_L1": lambda: workloads.icosphere_p2(1),
    "spheroid_L2": lambda: workloads.spheroid_p2(2, 1.0, 1.5),
}


def _system(name):
    xyz, tri6 = MESHES[name]()
    p = mu.Params(ka=2.0, eps_r=(3.0, 0.2), q_regular=6, ssq_order=4)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule, out=False)
    inc = workloads.fibonacci_plane_waves(2)[:3]
    Z, near, B = mu.assemble(m, p, mu.MUELLER_C64_NEAR64, inc=inc)
    op = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    mu.precond_build(op, min(64, m.N // 2))
    return m, op, B


def _relres(op, B, X):
    R = B - mu.matvec(op, X)
    nb = torch.linalg.norm(B, dim=1)
    return (torch.linalg.norm(R, dim=1) / torch.where(nb > 0, nb, torch.ones_like(nb))).cpu().numpy()


@pytest.mark.parametrize("name", list(MESHES))
def test_lockstep_matches_single_solves(name):
    m, op, B = _system(name)
    opts = mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=30, tol=1e-8)
    X, info = mu.solve(op, B, opts)
    assert info["converged"] == B.shape[0]
    assert np.all(_relres(op, B, X) <= 1e-8)
    for k in range(B.shape[0]):
        Xk, ik = mu.solve(op, B[k:k + 1].contiguous(), opts)
        assert ik["converged"] == 1
        e = (torch.linalg.norm(X[k] - Xk[0]) / torch.linalg.norm(Xk[0])).item()
        assert e <= 1e-6, (k, e)
    m.free()


def test_zero_right_hand_side_in_the_lockstep():
    m, op, B = _system("sphere_L1")
    B = B.clone()
    B[1] = 0
    X, info = mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=30, tol=1e-8))
    assert info["converged"] == 3
    assert torch.all(X[1] == 0)
    assert torch.isfinite(torch.view_as_real(X)).all()
    rr = _relres(op, B, X)
    assert rr[0] <= 1e-8 and rr[2] <= 1e-8
    m.free()
