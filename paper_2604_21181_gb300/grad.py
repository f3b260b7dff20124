"""Gradients of the cross sections with respect to the material parameters
and to the node coordinates of the P2 mesh.

For the scatterer's relative permittivity eps_r and permeability mu_r (each
complex, i.e. two real parameters) this returns the Jacobian of
(C_ext, C_sca, C_abs) of one incident wave, and a torch.autograd.Function
around it.  For the node coordinates X it returns the three gradients
dC/dX by the adjoint method (shape_gradient, below), and an autograd
Function of the coordinates.

Two forms of the material Jacobian are kept: adjoint_gradients (one adjoint
solve Z^H lam = conj(dC/dx) for the three outputs, then lam^H (dZ/dtheta) x;
the autograd Functions use it, and it serves the node coordinates too) and
material_jacobian, the tangent-linear form below, which checks it:

* Z(theta) x = b with b independent of eps_r, mu_r; Z is holomorphic in
  eps_r and mu_r (through k_i = k_a sqrt(eps_r mu_r), principal branch, and
  the explicit eps_r, mu_r factors of Eq. global_system), so for the real
  part of a parameter  Z x_theta = -(dZ/dtheta) x  and for the imaginary part
  the direction is i x_theta.
* (dZ/dtheta) x comes from mueller_dz_matvec: every element pair's block of
  dZ/dtheta is recomputed from the derivatives of the radial functions and
  multiplied into the result (no dZ is stored).
* C_ext is linear in x and C_sca, C_abs are Hermitian quadratic forms, so
  dC_ext = C_ext(x_theta) and dC_q = C_q(x + x_theta) - C_q(x) - C_q(x_theta),
  all from one far-field call over the combined currents.
Every step runs in the library's CUDA kernels (FP64 assembly, FP64 GMRES
with the block-Jacobi preconditioner, FP64 far field).
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import api


def _fp64_solve(op, B, tol):
    return api.solve(op, B, api.SolverOpts(mode=api.SOLVE_GMRES, restart=50, tol=tol))[0]


def forward_state(mesh, params, inc, block=None, tol=1e-12):
    """Assembly (FP64), block-Jacobi, FP64 GMRES and far field of one incident
    wave.  Returns (xs numpy (3,), state) with state holding Z, the operator
    and the solution for material_jacobian."""
    inc = np.ascontiguousarray(inc, dtype=np.float64).reshape(-1, 6)[:1]
    Z, _, B = api.assemble(mesh, params, api.MUELLER_C128, inc=inc)
    op = api.Operator(mesh, Z, dtype=api.MUELLER_C128)
    api.precond_build(op, block or min(256, mesh.N // 2))
    X = _fp64_solve(op, B, tol)
    _, xs = api.far_field(mesh, params, X, inc)
    return xs[0], dict(mesh=mesh, params=params, inc=inc, op=op, X=X, xs=xs[0], tol=tol)


def dz_matvec_fd(mesh, params, key, X, h_rel=1e-5):
    """(dZ/dtheta) X by the central difference of two assembled operators
    (theta = 'eps_r' or 'mu_r'), for checking mueller_dz_matvec."""
    torch = api._torch()
    val = complex(*getattr(params, key))
    h = h_rel * max(1.0, abs(val))
    Zs = torch.empty((mesh.N, mesh.N), dtype=torch.complex128, device="cuda")
    y = []
    for sgn in (1.0, -1.0):
        v = val + sgn * h
        api.assemble(mesh, dataclasses.replace(params, **{key: (v.real, v.imag)}),
                     api.MUELLER_C128, Z=Zs)
        y.append(api.matvec(api.Operator(mesh, Zs, dtype=api.MUELLER_C128), X))
    return (y[0] - y[1]) / (2.0 * h)


def material_jacobian(state):
    """3 x 4 Jacobian of (C_ext, C_sca, C_abs) with respect to
    (Re eps_r, Im eps_r, Re mu_r, Im mu_r) at the forward state."""
    torch = api._torch()
    mesh, params, inc, op, X = (state[k] for k in ("mesh", "params", "inc", "op", "X"))
    tangents = []
    for which in (1, 2):
        ZtX = api.dz_matvec(mesh, params, which, X[0]).reshape(1, -1)
        tangents.append(_fp64_solve(op, -ZtX, state["tol"]))
    comb = []
    for Xt in tangents:
        comb += [Xt, 1j * Xt, X + Xt, X + 1j * Xt]
    Xall = torch.cat(comb).contiguous()
    _, xs = api.far_field(mesh, params, Xall, np.repeat(inc, Xall.shape[0], axis=0))
    x0 = state["xs"]
    J = np.zeros((3, 4))
    for c in range(2):
        lin_re, lin_im, sum_re, sum_im = xs[4 * c:4 * c + 4]
        J[0, 2 * c] = lin_re[0]
        J[0, 2 * c + 1] = lin_im[0]
        for o in (1, 2):
            J[o, 2 * c] = sum_re[o] - x0[o] - lin_re[o]
            J[o, 2 * c + 1] = sum_im[o] - x0[o] - lin_im[o]
    return J


def _autograd_function():
    torch = api._torch()

    class CrossSections(torch.autograd.Function):
        """(C_ext, C_sca, C_abs) of one incident wave as a function of
        eps = (Re eps_r, Im eps_r) and mu = (Re mu_r, Im mu_r), float64
        tensors of shape (2,); the Jacobian is formed in backward."""

        @staticmethod
        def forward(ctx, eps, mu, mesh, params, inc):
            p = dataclasses.replace(params, eps_r=tuple(float(v) for v in eps.tolist()),
                                    mu_r=tuple(float(v) for v in mu.tolist()))
            xs, state = forward_state(mesh, p, inc)
            ctx.state = state
            return torch.tensor(xs, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            gp = torch.from_numpy(vjp(ctx.state, g.detach().cpu().numpy(), shape=False)[0])
            ctx.state = None
            return gp[:2], gp[2:], None, None, None

    return CrossSections


_cs = None


def cross_sections(eps, mu, mesh, params, inc):
    """Differentiable (C_ext, C_sca, C_abs); see CrossSections."""
    global _cs
    if _cs is None:
        _cs = _autograd_function()
    return _cs.apply(eps, mu, mesh, params, inc)


def adjoint_gradients(state, n_theta=48, n_phi=96, material=True, shape=True, timings=None):
    """Gradients of (C_ext, C_sca, C_abs) at the forward state by one adjoint
    solve: the 3 x 4 Jacobian with respect to (Re eps_r, Im eps_r, Re mu_r,
    Im mu_r) and the (3, n_nodes, 3) gradient with respect to the node
    coordinates (input node order).

    With G_o = conj(dC_o/dx) at fixed geometry and Z^H lam_o = G_o,
        dC_o/dtheta = 2 Re lam_o^H (db/dtheta - (dZ/dtheta) x) + dC_o/dtheta|_x.
    * Material parameters: b and C|_x do not depend on them and Z is
      holomorphic, so with d = lam^H (dZ/dtheta) x (mueller_dz_matvec) the
      real part of theta gives -2 Re d and the imaginary part 2 Im d.
    * Node coordinates: dC/dX|_x from mueller_cross_section_partials,
      2 Re lam^H db/dX from mueller_rhs_shape_vjp, 2 Re lam^H (dZ/dX) x from
      mueller_zshape_vjp (pair blocks recomputed, no dZ stored).  The frame
      depends on X through the nodal normals and frames (Secs. 3.1-3.3), and
      the gradient follows it: it is the derivative of the discrete cross
      sections as the library computes them.
    The three adjoint systems are one FP64 GMRES call on Z^H, right-
    preconditioned by the conjugate transpose of the block-Jacobi inverse.
    material / shape: which of the two to form (the other is returned as
    None).  timings: an optional dict that receives the wall time (ms, device
    synchronised) of each stage."""
    import time

    torch = api._torch()
    mesh, params, inc, op, X = (state[k] for k in ("mesh", "params", "inc", "op", "X"))
    clock = [time.perf_counter()]

    def lap(name):
        if timings is not None:
            torch.cuda.synchronize()
            t = time.perf_counter()
            timings[name] = round((t - clock[0]) * 1e3, 2)
            clock[0] = t

    G, grad, _ = api.cross_section_partials(mesh, params, X[0], inc[0], n_theta, n_phi)
    lap("partials_ms")
    opa = api.Operator(mesh, op.Z, dtype=api.MUELLER_C128, precond=op.precond, block=op.block,
                       adjoint=True)
    lam = _fp64_solve(opa, G, state["tol"])
    lap("adjoint_solve_ms")
    J = None
    if material:
        J = np.zeros((3, 4))
        for c, which in enumerate((1, 2)):
            v = api.dz_matvec(mesh, params, which, X[0])
            d = (lam.conj() @ v).cpu().numpy()
            J[:, 2 * c] = -2.0 * d.real
            J[:, 2 * c + 1] = 2.0 * d.imag
        lap("material_ms")
    if not shape:
        return J, None
    gz = api.zshape_vjp_multi(mesh, params, lam, X[0])  # the three outputs in one pass
    for o in range(3):
        grad[o] += 2.0 * (api.rhs_shape_vjp(mesh, params, lam[o], inc[0]) - gz[o])
    lap("shape_ms")
    return J, grad


def shape_gradient(state, n_theta=48, n_phi=96):
    """The node-coordinate part of adjoint_gradients, numpy (3, n_nodes, 3)."""
    return adjoint_gradients(state, n_theta, n_phi, material=False)[1]


def vjp(state, w, material=True, shape=True, n_theta=48, n_phi=96):
    """w^T of the gradients of (C_ext, C_sca, C_abs) for real weights w (3,):
    (w^T J numpy (4,) or None, w^T dC/dX numpy (n_nodes, 3) or None).

    Everything after the forward solve is real-linear in lam, so the weighted
    sum needs one adjoint solve Z^H lam = sum_o w_o G_o and one pass of each
    derivative kernel, a third of adjoint_gradients' work: this is what a
    reverse-mode backward needs."""
    torch = api._torch()
    mesh, params, inc, op, X = (state[k] for k in ("mesh", "params", "inc", "op", "X"))
    w = np.asarray(w, dtype=np.float64).reshape(3)
    G, gfix, _ = api.cross_section_partials(mesh, params, X[0], inc[0], n_theta, n_phi)
    wt = torch.as_tensor(w, dtype=torch.complex128, device=G.device)
    Gw = (wt @ G).reshape(1, -1)
    opa = api.Operator(mesh, op.Z, dtype=api.MUELLER_C128, precond=op.precond, block=op.block,
                       adjoint=True)
    lam = _fp64_solve(opa, Gw, state["tol"])[0]
    gJ = gX = None
    if material:
        gJ = np.zeros(4)
        for c, which in enumerate((1, 2)):
            d = torch.vdot(lam, api.dz_matvec(mesh, params, which, X[0])).item()
            gJ[2 * c] = -2.0 * d.real
            gJ[2 * c + 1] = 2.0 * d.imag
    if shape:
        gX = np.einsum("o,onk->nk", w, gfix) + 2.0 * (
            api.rhs_shape_vjp(mesh, params, lam, inc[0]) - api.zshape_vjp(mesh, params, lam, X[0]))
    return gJ, gX


def _shape_function():
    torch = api._torch()

    class ShapeCrossSections(torch.autograd.Function):
        """(C_ext, C_sca, C_abs) of one incident wave as a function of the
        node coordinates xyz (float64 tensor (n_nodes, 3)) of a P2 mesh with
        connectivity tri6; the gradient is formed in backward."""

        @staticmethod
        def forward(ctx, xyz, tri6, params, inc, block):
            mesh = api.Mesh(xyz.detach().cpu().numpy(), tri6)
            mesh.tangent_frame(params.frame_rule, out=False)
            xs, state = forward_state(mesh, params, inc, block)
            ctx.state = state
            return torch.tensor(xs, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            gX = torch.from_numpy(vjp(ctx.state, g.detach().cpu().numpy(), material=False)[1])
            ctx.state["mesh"].free()
            ctx.state = None
            return gX, None, None, None, None

    return ShapeCrossSections


_sc = None


def cross_sections_of_nodes(xyz, tri6, params, inc, block=None):
    """Differentiable (C_ext, C_sca, C_abs) of the node coordinates."""
    global _sc
    if _sc is None:
        _sc = _shape_function()
    return _sc.apply(xyz, tri6, params, inc, block)
