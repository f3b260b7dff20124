"""Dispersive permittivities for wavelength sweeps.

SILVER_JC holds the optical constants of silver (wavelength in nm, refractive
index n, extinction coefficient kappa) that the paper prints for its silver
spheroid benchmark (Benchmark II, table of optical constants after Johnson
and Christy); the relative permittivity is eps_r = (n + i kappa)^2.  Between
the tabulated wavelengths n and kappa are interpolated linearly in the
wavelength (the paper does not state its interpolation; linear interpolation
reproduces the value it quotes at the resonance, eps_r ~ -10.15 + 0.32i at
506 nm).  Outside the table the end values are refused rather than
extrapolated.
"""

import numpy as np

# (lambda [nm], n, kappa)
SILVER_JC = np.array([
    (300.9, 1.34, 0.964), (310.7, 1.13, 0.616), (320.4, 0.81, 0.392), (331.5, 0.17, 0.829),
    (342.5, 0.14, 1.142), (354.2, 0.10, 1.419), (367.9, 0.07, 1.657), (381.5, 0.05, 1.864),
    (397.4, 0.05, 2.070), (413.3, 0.05, 2.275), (430.5, 0.04, 2.462), (450.9, 0.04, 2.657),
    (471.4, 0.05, 2.869), (495.9, 0.05, 3.093), (520.9, 0.05, 3.324), (548.6, 0.06, 3.586),
    (582.1, 0.05, 3.858), (616.8, 0.06, 4.152), (659.5, 0.05, 4.483), (704.5, 0.04, 4.838),
    (756.0, 0.03, 5.242), (821.1, 0.04, 5.727),
])


def eps_silver(lam_nm):
    """Relative permittivity of silver at the wavelengths lam_nm (nm), as a
    complex array (linear interpolation of n and kappa in the wavelength)."""
    lam = np.atleast_1d(np.asarray(lam_nm, dtype=np.float64))
    lo, hi = SILVER_JC[0, 0], SILVER_JC[-1, 0]
    if np.any(lam < lo) or np.any(lam > hi):
        raise ValueError(f"silver table covers {lo} .. {hi} nm")
    n = np.interp(lam, SILVER_JC[:, 0], SILVER_JC[:, 1])
    kappa = np.interp(lam, SILVER_JC[:, 0], SILVER_JC[:, 2])
    return (n + 1j * kappa) ** 2
