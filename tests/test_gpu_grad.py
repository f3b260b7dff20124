"""Gradients of the cross sections with respect to eps_r and mu_r (complex),
FP64 path (grad.material_jacobian):

* against the oracle's gradient (central differences of its own FP64
  pipeline) on the level-1 spheroid of axis ratio 1.5, eps_r = 3 + 0.2i,
  k_a = 3, and a magnetic case (mu_r = 1.5 + 0.1i): within 1e-5 of each
  column's largest entry (the two assemblies
  agree to 1e-11, both solves are direct or converged to 1e-12, and the
  oracle's central differences carry an O(h^2) error of about 1e-8);
* against central differences of the GPU's own cross sections (full solves
  at theta +- h) on the level-2 spheroid, within 1e-5;
* the adjoint form (one solve Z^H lam = conj(dC/dx) for the three outputs,
  then lam^H (dZ/dtheta) x) against the tangent-linear form, within 1e-8,
  and against the oracle, within 1e-5;
* the autograd.Function's backward returns g^T J.
"""

import dataclasses

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

PHYS = dict(ka=3.0, eps_r=(3.0, 0.2), mu_r=(1.0, 0.0))


def _setup(level, ns=4):
    xyz, tri6 = workloads.spheroid_p2(level, 1.0, 1.5)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(0, out=False)
    p = mu.Params(ka=PHYS["ka"], eps_r=PHYS["eps_r"], mu_r=PHYS["mu_r"], q_regular=6,
                  ssq_order=ns, frame_rule=0)
    return xyz, tri6, m, p, workloads.plane_wave((0.0, 0.0, 1.0), (1.0, 0.0, 0.0))


def _colmax_err(A, B):
    return max(np.abs(A[:, k] - B[:, k]).max() / np.abs(B[:, k]).max() for k in range(A.shape[1]))


@pytest.mark.parametrize("phys", [PHYS, dict(ka=2.0, eps_r=(2.0, 0.1), mu_r=(1.5, 0.1))])
def test_material_jacobian_matches_oracle_gradient(phys):
    xyz, tri6, m, p, inc = _setup(1)
    p = dataclasses.replace(p, ka=phys["ka"], eps_r=phys["eps_r"], mu_r=phys["mu_r"])
    xs, state = mu.grad.forward_state(m, p, inc)
    J = mu.grad.material_jacobian(state)
    om = oracle.Mesh(xyz, tri6, frame_rule=0)
    pw = dict(phys, q_regular=6, ssq_order=4)
    xso = oracle.cross_sections(om, pw, inc)[0]
    np.testing.assert_allclose(xs, xso, rtol=1e-10)
    Jo = oracle.cross_section_gradient(om, pw, inc)
    assert _colmax_err(J, Jo) <= 1e-5, (J, Jo)


@pytest.mark.parametrize("phys", [PHYS, dict(ka=2.0, eps_r=(2.0, 0.1), mu_r=(1.5, 0.1))])
def test_adjoint_material_jacobian_matches_tangent_and_oracle(phys):
    xyz, tri6, m, p, inc = _setup(1)
    p = dataclasses.replace(p, ka=phys["ka"], eps_r=phys["eps_r"], mu_r=phys["mu_r"])
    _, state = mu.grad.forward_state(m, p, inc)
    Ja, _ = mu.grad.adjoint_gradients(state, shape=False)
    Jt = mu.grad.material_jacobian(state)
    assert _colmax_err(Ja, Jt) <= 1e-8, (Ja, Jt)
    om = oracle.Mesh(xyz, tri6, frame_rule=0)
    Jo = oracle.cross_section_gradient(om, dict(phys, q_regular=6, ssq_order=4), inc)
    assert _colmax_err(Ja, Jo) <= 1e-5, (Ja, Jo)


def test_material_jacobian_matches_own_central_differences():
    _, _, m, p, inc = _setup(2, ns=3)
    _, state = mu.grad.forward_state(m, p, inc)
    J = mu.grad.material_jacobian(state)
    h = 1e-4
    Jfd = np.zeros((3, 4))
    for k in range(4):
        key, part = ("eps_r", "mu_r")[k // 2], k % 2
        xs = []
        for sgn in (1.0, -1.0):
            v = list(getattr(p, key))
            v[part] += sgn * h
            xs.append(mu.grad.forward_state(m, dataclasses.replace(p, **{key: tuple(v)}), inc)[0])
        Jfd[:, k] = (xs[0] - xs[1]) / (2 * h)
    assert _colmax_err(J, Jfd) <= 1e-5, (J, Jfd)


def test_autograd_backward_is_g_transpose_j():
    _, _, m, p, inc = _setup(1, ns=3)
    eps = torch.tensor(PHYS["eps_r"], dtype=torch.float64, requires_grad=True)
    mur = torch.tensor(PHYS["mu_r"], dtype=torch.float64, requires_grad=True)
    C = mu.grad.cross_sections(eps, mur, m, p, inc)
    g = torch.tensor([1.0, 2.0, -0.5], dtype=torch.float64)
    (C * g).sum().backward()
    _, state = mu.grad.forward_state(m, p, inc)
    J = mu.grad.material_jacobian(state)  # the tangent-linear form; backward uses the adjoint
    want = g.numpy() @ J
    np.testing.assert_allclose(np.r_[eps.grad.numpy(), mur.grad.numpy()], want, rtol=1e-7,
                               atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("which,key", [(1, "eps_r"), (2, "mu_r")])
def test_dz_matvec_matches_central_difference_of_assembled_operator(which, key):
    """mueller_dz_matvec (pair blocks of dZ/dtheta recomputed from the
    derivatives of the radial functions) against the central difference of
    two assembled FP64 operators applied to the same vector: within 1e-8 of
    the largest entry (the difference's own error is O(h^2) with h = 1e-5
    relative, plus rounding over h)."""
    _, _, m, p, _ = _setup(1, ns=3)
    p = dataclasses.replace(p, ka=2.0, eps_r=(2.0, 0.3), mu_r=(1.5, 0.1))
    g = torch.Generator().manual_seed(3)
    X = torch.complex(torch.randn(m.N, generator=g, dtype=torch.float64),
                      torch.randn(m.N, generator=g, dtype=torch.float64)).cuda()
    Y = mu.dz_matvec(m, p, which, X)
    Yfd = mu.grad.dz_matvec_fd(m, p, key, X.reshape(1, -1))[0]
    err = (Y - Yfd).abs().max().item() / Yfd.abs().max().item()
    assert err <= 1e-8, err
