"""Node-coordinate gradients of the cross sections on the GPU (adjoint
method), term by term and whole:

* the adjoint operator (MUELLER_OP_ADJOINT): Z^H x against the conjugate
  transpose in PyTorch, and FP64 GMRES on Z^H with the conjugate-transposed
  block-Jacobi inverse;
* mueller_rhs_shape_vjp against central differences of Re lam^H b over the
  GPU's right-hand sides at displaced nodes;
* mueller_cross_section_partials: the cross sections it returns against
  mueller_far_field, dC/dx (the adjoint right-hand sides) against central
  differences of far_field along a random direction of x, and dC/dX at fixed
  x against central differences of far_field on displaced meshes;
* grad.shape_gradient against the oracle's gradient (central differences of
  its own dense pipeline) on the level-1 spheroid, at sampled nodes away from
  the frame rule's switch, for the paper's and the polar frame rule, and a
  magnetic lossy scatterer (mu_r = 1.4 + 0.1i);
* on the level-3 spheroid of axis ratio 1.5 (eps_r = 3 + 0.2i, k_a = 3,
  the paper's frame rule): adjoint_gradients against central differences
  with step 1e-6 of full FP64 solves at displaced nodes (measured within
  6e-8 of each output's largest entry), its material Jacobian against the
  tangent-linear one, and translation invariance;
* the autograd Function's backward (grad.vjp: one adjoint solve for the
  weighted outputs) returns g^T dC/dX.
Meshes keep the input node order (morton=False) wherever a vector of
unknowns is held fixed while the nodes move."""

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

PHYS = dict(ka=2.0, eps_r=(3.0, 0.2), mu_r=(1.0, 0.0))
INC = workloads.plane_wave((0.0, 0.6, 0.8), (1.0, 0.0, 0.0))


def _params(rule, phys=PHYS, ns=4):
    return mu.Params(ka=phys["ka"], eps_r=phys["eps_r"], mu_r=phys["mu_r"], q_regular=6,
                     ssq_order=ns, frame_rule=rule)


def _mesh(xyz, tri6, rule):
    m = mu.Mesh(xyz, tri6, morton=False)
    m.tangent_frame(rule, out=False)
    return m


def _sample_nodes(xyz, tri6, rule, k, seed):
    """k nodes whose normal is away from the poles and from the paper
    rule's switch at |n_z| = 0.9 (the frame is not differentiable there)."""
    m = mu.Mesh(xyz, tri6, morton=False)
    fr = m.tangent_frame(rule).cpu().numpy()
    m.free()
    nz = np.abs(fr[:, 2])
    ok = np.where((nz < 0.85) | ((nz > 0.95) & (nz < 0.999)))[0] if rule == 0 else \
        np.where(nz < 0.99)[0]
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(ok, k, replace=False))


def _displaced(xyz, k, d, h):
    x = xyz.copy()
    x[k, d] += h
    return x


def test_adjoint_matvec_and_solve():
    xyz, tri6 = workloads.spheroid_p2(2, 1.0, 1.5)
    p = _params(1)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(1, out=False)
    Z, _, _ = mu.assemble(m, p, mu.MUELLER_C128)
    g = torch.Generator().manual_seed(5)
    x = torch.randn(2, m.N, dtype=torch.complex128, generator=g).cuda()
    opa = mu.Operator(m, Z, dtype=mu.MUELLER_C128, adjoint=True)
    y = mu.matvec(opa, x)
    ref = x @ Z.conj()
    assert (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item() <= 1e-13
    op = mu.Operator(m, Z, dtype=mu.MUELLER_C128)
    mu.precond_build(op, 256)
    opa = mu.Operator(m, Z, dtype=mu.MUELLER_C128, precond=op.precond, block=op.block,
                      adjoint=True)
    lam, info = mu.solve(opa, x, mu.SolverOpts(mode=mu.SOLVE_GMRES, tol=1e-12))
    assert info["converged"] == 2
    res = torch.linalg.norm(lam @ Z.conj() - x, dim=1) / torch.linalg.norm(x, dim=1)
    assert res.max().item() <= 1e-11
    # the adjoint flag is refused where it has no meaning
    with pytest.raises(mu.MuellerError):
        mu.solve(opa, x, mu.SolverOpts(mode=mu.SOLVE_DENSE_LU))
    m.free()


def test_rhs_shape_vjp_matches_central_differences():
    xyz, tri6 = workloads.spheroid_p2(1, 1.0, 1.5)
    p = _params(1)
    m = _mesh(xyz, tri6, 1)
    mu.assemble(m, p, mu.MUELLER_C128)
    lam = torch.randn(m.N, dtype=torch.complex128,
                      generator=torch.Generator().manual_seed(9)).cuda()
    G = mu.rhs_shape_vjp(m, p, lam, INC[0])
    m.free()

    def f(x):
        mm = _mesh(x, tri6, 1)
        _, _, B = mu.assemble(mm, p, mu.MUELLER_C128, inc=INC)
        mm.free()
        return torch.vdot(lam, B[0]).real.item()

    nodes = _sample_nodes(xyz, tri6, 1, 6, seed=2)
    h = 1e-5
    fd = np.array([[(f(_displaced(xyz, k, d, h)) - f(_displaced(xyz, k, d, -h))) / (2 * h)
                    for d in range(3)] for k in nodes])
    err = np.abs(G[nodes] - fd).max() / np.abs(fd).max()
    assert err <= 1e-6, (err, G[nodes], fd)


@pytest.fixture(scope="module")
def partials_case():
    xyz, tri6 = workloads.spheroid_p2(1, 1.0, 1.5)
    p = _params(1)
    m = _mesh(xyz, tri6, 1)
    Z, _, B = mu.assemble(m, p, mu.MUELLER_C128, inc=INC)
    op = mu.Operator(m, Z, dtype=mu.MUELLER_C128)
    mu.precond_build(op, 128)
    X, _ = mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_GMRES, tol=1e-13))
    G, gfix, xs = mu.cross_section_partials(m, p, X[0], INC[0], 24, 48)
    _, xs_ff = mu.far_field(m, p, X, INC, n_theta=24, n_phi=48)
    yield dict(xyz=xyz, tri6=tri6, p=p, m=m, X=X, G=G, gfix=gfix, xs=xs, xs_ff=xs_ff[0])
    m.free()


def test_partials_cross_sections_match_far_field(partials_case):
    c = partials_case
    np.testing.assert_allclose(c["xs"], c["xs_ff"], rtol=1e-11)


def test_partials_current_derivative(partials_case):
    c = partials_case
    m, p, X, G = c["m"], c["p"], c["X"], c["G"]
    v = torch.randn(m.N, dtype=torch.complex128,
                    generator=torch.Generator().manual_seed(4)).cuda()
    v *= torch.linalg.norm(X[0]) / torch.linalg.norm(v)
    t = 1e-5
    _, xp = mu.far_field(m, p, (X[0] + t * v).reshape(1, -1), INC, n_theta=24, n_phi=48)
    _, xm = mu.far_field(m, p, (X[0] - t * v).reshape(1, -1), INC, n_theta=24, n_phi=48)
    fd = (xp[0] - xm[0]) / (2 * t)
    lin = np.array([2.0 * torch.vdot(G[o], v).real.item() for o in range(3)])
    assert np.abs(lin - fd).max() <= 1e-7 * np.abs(c["xs"]).max(), (lin, fd)


def test_partials_geometry_derivative_at_fixed_currents(partials_case):
    c = partials_case
    xyz, tri6, p, X = c["xyz"], c["tri6"], c["p"], c["X"]

    def f(x):
        mm = _mesh(x, tri6, 1)
        _, xs = mu.far_field(mm, p, X, INC, n_theta=24, n_phi=48)
        mm.free()
        return xs[0]

    nodes = _sample_nodes(xyz, tri6, 1, 5, seed=11)
    h = 1e-5
    for k in nodes:
        for d in range(3):
            fd = (f(_displaced(xyz, k, d, h)) - f(_displaced(xyz, k, d, -h))) / (2 * h)
            an = c["gfix"][:, k, d]
            assert np.abs(an - fd).max() <= 1e-6 * np.abs(c["gfix"]).max(), (k, d, an, fd)


MAGNETIC = dict(ka=1.5, eps_r=(2.5, 0.3), mu_r=(1.4, 0.1))


@pytest.mark.parametrize("rule,phys", [(0, PHYS), (1, PHYS), (1, MAGNETIC)],
                         ids=["paper_rule", "polar_rule", "polar_rule_magnetic_lossy"])
def test_shape_gradient_matches_oracle(rule, phys):
    xyz, tri6 = workloads.spheroid_p2(1, 1.0, 1.5)
    p = _params(rule, phys)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(rule, out=False)
    xs, state = mu.grad.forward_state(m, p, INC)
    grad = mu.grad.shape_gradient(state)
    assert grad.shape == (3, len(xyz), 3) and np.all(np.isfinite(grad))
    pw = dict(phys, q_regular=6, ssq_order=4)
    nodes = _sample_nodes(xyz, tri6, rule, 5, seed=rule + 20)
    Go = oracle.cross_section_coordinate_gradient(xyz, tri6, pw, INC, nodes=nodes,
                                                  frame_rule=rule)  # (k, 3 coords, 3 outputs)
    Gg = grad[:, nodes, :].transpose(1, 2, 0)
    for o in range(3):
        err = np.abs(Gg[..., o] - Go[..., o]).max() / np.abs(Go[..., o]).max()
        assert err <= 1e-5, (o, err, Gg[..., o], Go[..., o])
    # translation invariance of the whole gradient
    for o in range(3):
        assert np.abs(grad[o].sum(axis=0)).max() <= 1e-8 * np.abs(grad[o]).max()
    m.free()


def test_autograd_backward_is_g_transpose_gradient():
    xyz, tri6 = workloads.spheroid_p2(1, 1.0, 1.5)
    p = _params(1, ns=3)
    X = torch.tensor(xyz, dtype=torch.float64, requires_grad=True)
    C = mu.grad.cross_sections_of_nodes(X, tri6, p, INC)
    w = torch.tensor([0.3, -1.0, 2.0], dtype=torch.float64)
    (C * w).sum().backward()
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(1, out=False)
    _, state = mu.grad.forward_state(m, p, INC)
    G = mu.grad.shape_gradient(state)
    ref = np.einsum("o,onk->nk", w.numpy(), G)
    assert np.abs(X.grad.numpy() - ref).max() <= 1e-8 * np.abs(ref).max()
    m.free()


def test_level3_spheroid_gradient_matches_central_differences():
    xyz, tri6 = workloads.spheroid_p2(3, 1.0, 1.5)
    p = mu.Params(ka=3.0, eps_r=(3.0, 0.2), mu_r=(1.0, 0.0), q_regular=6, ssq_order=5,
                  frame_rule=0)
    inc = workloads.plane_wave((0.0, 0.0, 1.0), (1.0, 0.0, 0.0))

    def fwd(x):
        m = mu.Mesh(x, tri6)
        m.tangent_frame(0, out=False)
        xs, st = mu.grad.forward_state(m, p, inc, tol=1e-13)
        return m, xs, st

    m, xs, st = fwd(xyz)
    J, G = mu.grad.adjoint_gradients(st)
    Jt = mu.grad.material_jacobian(st)
    assert np.abs(J - Jt).max() <= 1e-9 * np.abs(Jt).max()
    gmax = np.abs(G).reshape(3, -1).max(axis=1)
    for o in range(3):
        assert np.abs(G[o].sum(axis=0)).max() <= 1e-8 * gmax[o]
    m.free()
    h = 1e-6
    for k in _sample_nodes(xyz, tri6, 0, 2, seed=1):
        for d in range(3):
            v = []
            for sg in (1.0, -1.0):
                mm, xs_, _ = fwd(_displaced(xyz, k, d, sg * h))
                v.append(xs_)
                mm.free()
            fd = (v[0] - v[1]) / (2 * h)
            assert np.all(np.abs(G[:, k, d] - fd) <= 1e-6 * gmax), (k, d, G[:, k, d], fd)
