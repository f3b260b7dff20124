"""Frequency sweeps and bistatic cuts of one body (through the C ABI only).

spectrum() computes the cross sections of one mesh at many frequencies
(k_a, eps_r, mu_r per frequency, e.g. a dispersive metal over a wavelength
range).  The mesh handle keeps its point geometry, tangent frame and
touching-pair tables, so only the frequency-dependent parts are recomputed:
every chunk of frequencies is assembled by one mueller_assemble_batch call
(one launch of each assembly kernel for the whole chunk), then each
frequency gets its block-Jacobi preconditioner, the mixed-precision GMRES-IR
solve of its right-hand sides and its far field.

bistatic_cut() evaluates the bistatic radar cross section
sigma(r) = 4 pi |F(r)|^2 (unit incident amplitude; F as returned by
mueller_far_field, whose integral of |F|^2 over the sphere is C_sca) along a
great circle of directions.
"""

import numpy as np

from . import api


def spectrum(mesh, ka, eps_r, inc, mu_r=None, q_regular: int = 6, ssq_order: int = 5,
             block: int = 256, tol: float = 1e-8, restart: int = 50, chunk: int = 16,
             n_theta: int = 48, n_phi: int = 96):
    """Cross sections of `mesh` (tangent frame already built) at the
    frequencies ka[i] with permittivities eps_r[i] (complex) and optionally
    permeabilities mu_r[i].  inc: r x 6 incident waves (the same at every
    frequency).  Returns a dict with xs (n_freq x r x 3: C_ext, C_sca,
    C_abs), the lockstep iterations and refinements per frequency, the worst
    final residual and the solutions of the last frequency."""
    torch = api._torch()
    ka = np.atleast_1d(np.asarray(ka, dtype=np.float64))
    eps_r = np.atleast_1d(np.asarray(eps_r, dtype=np.complex128))
    nf = ka.shape[0]
    if eps_r.shape[0] != nf:
        raise ValueError("one eps_r per frequency")
    mu = (np.ones(nf, np.complex128) if mu_r is None
          else np.atleast_1d(np.asarray(mu_r, dtype=np.complex128)))
    if mesh.frame_rule is None:
        raise ValueError("call mesh.tangent_frame first")
    inc = np.ascontiguousarray(inc, dtype=np.float64).reshape(-1, 6)
    params = [api.Params(ka=float(ka[i]), eps_r=(eps_r[i].real, eps_r[i].imag),
                         mu_r=(mu[i].real, mu[i].imag), q_regular=q_regular,
                         ssq_order=ssq_order, frame_rule=mesh.frame_rule) for i in range(nf)]
    opts = api.SolverOpts(mode=api.SOLVE_GMRES_IR, restart=restart, tol=tol)
    blk = min(block, mesh.N // 2)
    xs = np.zeros((nf, inc.shape[0], 3))
    iters = np.zeros(nf, np.int64)
    refinements = np.zeros(nf, np.int64)
    worst = 0.0
    X = None
    for c0 in range(0, nf, chunk):
        sel = list(range(c0, min(nf, c0 + chunk)))
        out = api.assemble_batch([mesh] * len(sel), [params[i] for i in sel],
                                 api.MUELLER_C64_NEAR64, incs=[inc] * len(sel))
        for i, (Z, near, B) in zip(sel, out):
            op = api.Operator(mesh, Z, near, api.MUELLER_C64_NEAR64)
            api.precond_build(op, blk)
            X, info = api.solve(op, B, opts)
            iters[i] = info["iters"] // inc.shape[0]
            refinements[i] = info["refinements"]
            worst = max(worst, info["relres"])
            _, xs[i] = api.far_field(mesh, params[i], X, inc, n_theta=n_theta, n_phi=n_phi)
        del out
        torch.cuda.empty_cache()
    return {"xs": xs, "iters": iters, "refinements": refinements, "worst_relres": worst,
            "X_last": X}


def bistatic_cut(mesh, params, X, inc, n: int = 181, plane: str = "xz"):
    """Bistatic RCS sigma = 4 pi |F|^2 at n directions theta in [0, pi] of the
    great circle in `plane` ("xz": (sin t, 0, cos t); "yz": (0, sin t,
    cos t); "xy": (cos t, sin t, 0) with t in [0, 2 pi)).  Returns (angles,
    sigma r x n)."""
    if plane == "xy":
        t = np.linspace(0.0, 2.0 * np.pi, n, endpoint=False)
        dirs = np.stack([np.cos(t), np.sin(t), np.zeros_like(t)], axis=1)
    else:
        t = np.linspace(0.0, np.pi, n)
        z = np.cos(t)
        if plane == "xz":
            dirs = np.stack([np.sin(t), np.zeros_like(t), z], axis=1)
        elif plane == "yz":
            dirs = np.stack([np.zeros_like(t), np.sin(t), z], axis=1)
        else:
            raise ValueError("plane must be xz, yz or xy")
    F, _ = api.far_field(mesh, params, X, inc, dirs=dirs)
    f2 = (F.abs() ** 2).sum(dim=2).cpu().numpy()
    return t, 4.0 * np.pi * f2
