"""Gradients with respect to the P2 node coordinates on the GPU.

mueller_zshape_vjp (the gradient of Re lam^H Z(X) x with respect to the node
coordinates, Sec. 3 geometry through Eq. global_system) against central
differences of Re lam^H Z x over FP64 assemblies of the GPU at displaced
nodes (input node order kept, so the unknowns stay put), for sampled
coordinates: a magnetic lossy case, the mass term alone (zero contrast), the
paper's frame rule away from its switch, and a level-2 mesh."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
]


def _s(xyz, tri6, p, lam, x):
    m = mu.Mesh(xyz, tri6, morton=False)
    m.tangent_frame(p.frame_rule, out=False)
    Z, _, _ = mu.assemble(m, p, mu.MUELLER_C128)
    v = torch.vdot(lam, Z @ x).real.item()
    m.free()
    return v


def _sample_nodes(xyz, tri6, rule, k, seed):
    """k nodes whose normal is away from the poles and from the paper
    rule's switch at |n_z| = 0.9 (the frame is not differentiable there)."""
    m = mu.Mesh(xyz, tri6, morton=False)
    fr = m.tangent_frame(rule).cpu().numpy()
    nz = np.abs(fr[:, 2])
    ok = np.where((nz < 0.85) | ((nz > 0.95) & (nz < 0.999)))[0] if rule == 0 else \
        np.where(nz < 0.99)[0]
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(ok, k, replace=False))


CASES = {
    "magnetic_lossy_polar": (lambda: workloads.spheroid_p2(1, 1.0, 1.5),
                             dict(ka=2.0, eps_r=(3.0, 0.2), mu_r=(1.2, 0.05)), 1),
    "mass_only": (lambda: workloads.spheroid_p2(1, 1.0, 1.5),
                  dict(ka=2.0, eps_r=(1.0, 0.0), mu_r=(1.0, 0.0)), 1),
    "paper_rule": (lambda: workloads.spheroid_p2(1, 1.3, 1.0),
                   dict(ka=1.5, eps_r=(4.0, 0.5), mu_r=(1.0, 0.0)), 0),
    "level2": (lambda: workloads.icosphere_p2(2),
               dict(ka=3.0, eps_r=(2.25, 0.1), mu_r=(1.0, 0.0)), 1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_zshape_vjp_matches_central_differences(name):
    mk, phys, rule = CASES[name]
    xyz, tri6 = mk()
    p = mu.Params(ka=phys["ka"], eps_r=phys["eps_r"], mu_r=phys["mu_r"], q_regular=6,
                  ssq_order=4, frame_rule=rule)
    m = mu.Mesh(xyz, tri6, morton=False)
    m.tangent_frame(rule, out=False)
    mu.assemble(m, p, mu.MUELLER_C128)  # point geometry of the rule
    g = torch.Generator().manual_seed(3)
    N = m.N
    lam = torch.randn(N, dtype=torch.complex128, generator=g).cuda()
    x = torch.randn(N, dtype=torch.complex128, generator=g).cuda()
    G = mu.zshape_vjp(m, p, lam, x)
    assert G.shape == (len(xyz), 3) and np.all(np.isfinite(G))
    nodes = _sample_nodes(xyz, tri6, rule, 4 if name == "level2" else 6, seed=7)
    h = 1e-5
    fd = np.zeros((len(nodes), 3))
    for a, k in enumerate(nodes):
        for d in range(3):
            xp = xyz.copy()
            xm = xyz.copy()
            xp[k, d] += h
            xm[k, d] -= h
            fd[a, d] = (_s(xp, tri6, p, lam, x) - _s(xm, tri6, p, lam, x)) / (2 * h)
    err = np.abs(G[nodes] - fd).max() / np.abs(fd).max()
    assert err <= 1e-6, (err, G[nodes], fd)


@pytest.mark.parametrize("r", [2, 3, 5])
def test_zshape_vjp_multi_equals_one_vector_at_a_time(r):
    """mueller_zshape_vjp_multi (several adjoint vectors per pass; the radial
    functions of each point pair shared by up to three of them) gives each
    vector's gradient as mueller_zshape_vjp alone does, to rounding."""
    xyz, tri6 = workloads.spheroid_p2(1, 1.0, 1.5)
    p = mu.Params(ka=2.0, eps_r=(3.0, 0.2), mu_r=(1.2, 0.05), q_regular=6, ssq_order=4,
                  frame_rule=1)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(1, out=False)
    mu.assemble(m, p, mu.MUELLER_C128)
    g = torch.Generator().manual_seed(5)
    lam = torch.randn((r, m.N), dtype=torch.complex128, generator=g).cuda()
    x = torch.randn(m.N, dtype=torch.complex128, generator=g).cuda()
    G = mu.zshape_vjp_multi(m, p, lam, x)
    assert G.shape == (r, len(xyz), 3)
    for o in range(r):
        G1 = mu.zshape_vjp(m, p, lam[o], x)
        err = np.abs(G[o] - G1).max() / np.abs(G1).max()
        assert err <= 1e-12, (o, err)
