"""ORACLE -- test infrastructure only.

Closed-form Mie series for a homogeneous sphere (radius a, exterior medium
eps = mu = 1, interior relative permittivity eps_r, mu_r = 1), time
convention exp(-i omega t).  Pins the cross sections of the solver: the
method's C_ext, C_sca, C_abs must converge to these under mesh refinement.

Two independent evaluations are provided:
* ``mie_bh``: logarithmic-derivative form with a downward recurrence for
  D_n(mx) and upward Riccati-Bessel recurrences (Bohren & Huffman, Ch. 4).
* ``mie_scipy``: the textbook coefficient formulas evaluated with SciPy's
  spherical Bessel functions (a library primitive).
"""

from __future__ import annotations

import numpy as np


def n_terms(x: float) -> int:
    return int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0)) + 10


def mie_coefficients_bh(x: float, m: complex, nmax: int | None = None):
    nstop = n_terms(x) if nmax is None else nmax
    mx = m * x
    nmx = int(max(nstop, abs(mx)) + 16)
    D = np.zeros(nmx + 1, dtype=np.complex128)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    psi_m1, psi_0 = np.cos(x), np.sin(x)
    chi_m1, chi_0 = -np.sin(x), np.cos(x)
    xi_m1 = psi_m1 - 1j * chi_m1
    a = np.zeros(nstop, dtype=np.complex128)
    b = np.zeros(nstop, dtype=np.complex128)
    psi_prev, chi_prev = psi_m1, chi_m1
    psi, chi = psi_0, chi_0
    for n in range(1, nstop + 1):
        psi_n = (2 * n - 1) / x * psi - psi_prev
        chi_n = (2 * n - 1) / x * chi - chi_prev
        xi_n = psi_n - 1j * chi_n
        xi_nm1 = psi - 1j * chi
        da = D[n] / m + n / x
        db = D[n] * m + n / x
        a[n - 1] = (da * psi_n - psi) / (da * xi_n - xi_nm1)
        b[n - 1] = (db * psi_n - psi) / (db * xi_n - xi_nm1)
        psi_prev, psi = psi, psi_n
        chi_prev, chi = chi, chi_n
    return a, b


def mie_coefficients_scipy(x: float, m: complex, nmax: int | None = None):
    from scipy.special import spherical_jn, spherical_yn

    nstop = n_terms(x) if nmax is None else nmax
    n = np.arange(1, nstop + 1)
    mx = m * x
    jx = spherical_jn(n, x)
    djx = spherical_jn(n, x, derivative=True)
    yx = spherical_yn(n, x)
    dyx = spherical_yn(n, x, derivative=True)
    jm = spherical_jn(n, mx)
    djm = spherical_jn(n, mx, derivative=True)
    hx = jx + 1j * yx
    dhx = djx + 1j * dyx
    # [rho z_n(rho)]' = z_n + rho z_n'
    xj_p = jx + x * djx
    xh_p = hx + x * dhx
    mxj_p = jm + mx * djm
    a = (m * m * jm * xj_p - jx * mxj_p) / (m * m * jm * xh_p - hx * mxj_p)
    b = (jm * xj_p - jx * mxj_p) / (jm * xh_p - hx * mxj_p)
    return a, b


def cross_sections(ka: float, eps_r, radius: float = 1.0, method: str = "bh"):
    """Return (C_ext, C_sca, C_abs) for a sphere of the given radius at
    exterior wavenumber ka (so the size parameter is ka * radius)."""
    eps_r = complex(*eps_r) if isinstance(eps_r, (tuple, list)) else complex(eps_r)
    m = np.sqrt(eps_r)
    if m.imag < 0:
        m = -m
    x = ka * radius
    f = mie_coefficients_bh if method == "bh" else mie_coefficients_scipy
    a, b = f(x, m)
    n = np.arange(1, len(a) + 1)
    pre = 2.0 * np.pi / ka ** 2
    cext = pre * np.sum((2 * n + 1) * np.real(a + b))
    csca = pre * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return float(cext), float(csca), float(cext - csca)


def mie_bh(ka, eps_r, radius=1.0):
    return cross_sections(ka, eps_r, radius, "bh")


def mie_scipy(ka, eps_r, radius=1.0):
    return cross_sections(ka, eps_r, radius, "scipy")
