"""The five synthetic workloads of the solver, with their sizes and physics.

Units: exterior eps = mu = 1, lengths in units of the (transverse) radius, so
omega = k_a and the interior wavenumber is k_a * sqrt(eps_r * mu_r).
"""

from __future__ import annotations

import numpy as np

from .meshes import icosphere_p2, spheroid_p2
from .excitation import plane_wave, fibonacci_plane_waves

WORKLOADS = {
    # small sphere, plain FP64, dense LU
    "sphere_L1_eps4_ka1": dict(
        level=1, shape="sphere", axis=1.0, eps_r=(4.0, 0.0), mu_r=(1.0, 0.0), ka=1.0,
        q_regular=6, ssq_order=5, block=256, restart=50, tol=1e-8, n_rhs=1,
    ),
    # larger sphere: GMRES(50) + Morton block Jacobi (B = 256), mixed vs FP64
    "sphere_L3_eps2.25_ka5": dict(
        level=3, shape="sphere", axis=1.0, eps_r=(2.25, 0.0), mu_r=(1.0, 0.0), ka=5.0,
        q_regular=6, ssq_order=5, block=256, restart=50, tol=1e-8, n_rhs=1,
    ),
    # adjoint-gradient geometry (prolate spheroid, axis ratio 1.5)
    "spheroid_L3_eps3+0.2i_ka3": dict(
        level=3, shape="spheroid", axis=1.5, eps_r=(3.0, 0.2), mu_r=(1.0, 0.0), ka=3.0,
        q_regular=6, ssq_order=5, block=256, restart=50, tol=1e-8, n_rhs=1,
    ),
    # extreme contrast, large mesh, 16 right-hand sides
    "sphere_L4_eps-10+1i_ka10": dict(
        level=4, shape="sphere", axis=1.0, eps_r=(-10.0, 1.0), mu_r=(1.0, 0.0), ka=10.0,
        q_regular=6, ssq_order=5, block=512, restart=50, tol=1e-8, n_rhs=16,
    ),
}


def workload(name: str):
    """Return ``(xyz, tri6, inc, params)`` for a named workload."""
    p = dict(WORKLOADS[name])
    if p["shape"] == "sphere":
        xyz, tri6 = icosphere_p2(p["level"])
    else:
        xyz, tri6 = spheroid_p2(p["level"], 1.0, p["axis"])
    if p["n_rhs"] == 1:
        inc = plane_wave((0, 0, 1), (1, 0, 0))
    else:
        inc = fibonacci_plane_waves(p["n_rhs"] // 2)
    return xyz, tri6, inc, p


def multibody_spec(n_bodies: int = 64, seed: int = 20260421):
    """Seeded list of uneven spheroid bodies (type, axis ratio, level, eps, ka)."""
    rng = np.random.default_rng(seed)
    bodies = []
    for _ in range(n_bodies):
        prolate = bool(rng.random() < 0.5)
        rho = float(rng.uniform(1.0, 2.0))
        level = int(rng.integers(1, 4))
        eps_re = float(rng.uniform(1.5, 6.0))
        eps_im = float(rng.uniform(0.0, 1.0))
        ka = float(rng.uniform(0.5, 5.0))
        bodies.append(dict(prolate=prolate, rho=rho, level=level, eps_r=(eps_re, eps_im),
                           mu_r=(1.0, 0.0), ka=ka))
    return bodies


def multibody_mesh(body: dict):
    """P2 mesh of one multibody_spec entry: prolate (1, 1, rho) or oblate
    (rho, rho, 1) spheroid at the entry's subdivision level."""
    if body["prolate"]:
        return spheroid_p2(body["level"], 1.0, body["rho"])
    return spheroid_p2(body["level"], body["rho"], 1.0)
