"""Plane-wave excitations.

An excitation is a row of six float64 numbers ``(kx, ky, kz, px, py, pz)``:
the unit propagation direction k and the real unit polarisation p (p . k = 0)
of the incident field E_inc(x) = p exp(i k_a k.x).
"""

from __future__ import annotations

import numpy as np


def plane_wave(k=(0.0, 0.0, 1.0), p=(1.0, 0.0, 0.0)) -> np.ndarray:
    k = np.asarray(k, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    k = k / np.linalg.norm(k)
    p = p - k * float(p @ k)
    p = p / np.linalg.norm(p)
    return np.concatenate([k, p])[None, :]


def fibonacci_directions(n: int) -> np.ndarray:
    """n directions on the Fibonacci sphere: z_i = 1-(2i+1)/n,
    phi_i = i*pi*(3-sqrt(5))."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * np.pi * (3.0 - 5.0 ** 0.5)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _theta_phi_hat(k: np.ndarray):
    x, y, z = k
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    phi = np.arctan2(y, x)
    th = np.array([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)])
    ph = np.array([-np.sin(phi), np.cos(phi), 0.0])
    return th, ph


def fibonacci_plane_waves(n_dir: int) -> np.ndarray:
    """2*n_dir excitations: for each Fibonacci direction the theta-hat and the
    phi-hat polarisation.  Rows are ordered (dir0 theta, dir0 phi, dir1 ...)."""
    rows = []
    for k in fibonacci_directions(n_dir):
        th, ph = _theta_phi_hat(k)
        rows.append(np.concatenate([k, th]))
        rows.append(np.concatenate([k, ph]))
    return np.ascontiguousarray(np.array(rows, dtype=np.float64))
