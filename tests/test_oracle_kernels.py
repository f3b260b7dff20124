"""Pins of the oracle's kernel scalars (Sec. 2.3, Eqs. Hessian series,
Hdiff_exact, H_diff_truncated, kappa_S, kappa2_S).

* Closed forms in 50-digit arithmetic (mpmath) fix S1, S2, D and H_diff at
  any R; the oracle's stable series/closed-form switch must agree to ~1e-13.
* The five printed coefficients of the truncated H_diff series must be
  reproduced: the oracle's H_diff minus the printed truncation is O(R^4).
* The O(R^-3) terms cancel: R * |H_diff| stays bounded as R -> 0.
* The remainder limits at R = 0 used on coincident points.
"""

import math

import numpy as np
import pytest

import oracle

CASES = [
    (1.0, 4.0 + 0j, 1.0 + 0j),       # small sphere
    (5.0, 2.25 + 0j, 1.0 + 0j),      # L3 sphere workload
    (3.0, 3.0 + 0.2j, 1.0 + 0j),     # spheroid workload
    (10.0, -10.0 + 1.0j, 1.0 + 0j),  # plasmonic workload
    (2.0, 2.0 + 0.5j, 1.5 + 0.1j),   # magnetic contrast
]


def ki_of(ka, er, mr):
    k = ka * np.sqrt(complex(er) * complex(mr))
    return -k if k.imag < 0 else k


def mp_closed(ka, er, mr, R):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    R = mp.mpf(R)
    ki = ki_of(ka, er, mr)
    kk = {"a": mp.mpf(ka), "i": mp.mpc(ki.real, ki.imag)}
    chi_e = {"a": mp.mpf(1), "i": mp.mpc(er.real, er.imag)}
    chi_m = {"a": mp.mpf(1), "i": mp.mpc(mr.real, mr.imag)}
    pi4 = 4 * mp.pi
    out = {}
    for s, k in kk.items():
        e = mp.exp(1j * k * R)
        out["phi" + s] = e / (pi4 * R)
        out["f" + s] = e * (3 - 3j * k * R - k * k * R * R) / (pi4 * R ** 3)
        out["g" + s] = e * (1 - 1j * k * R) / (pi4 * R ** 3)
        out["dphi" + s] = e * (1j * k * R - 1) / (pi4 * R ** 2)
    S1 = kk["a"] ** 2 * out["phia"] - kk["i"] ** 2 * out["phii"] - (out["ga"] - out["gi"])
    S2 = out["fa"] - out["fi"]
    De = chi_e["a"] * out["dphia"] - chi_e["i"] * out["dphii"]
    Dm = chi_m["a"] * out["dphia"] - chi_m["i"] * out["dphii"]
    Ib = -(out["ga"] - out["gi"])
    return [complex(v) for v in (S1, S2, De, Dm)], complex(Ib)


@pytest.mark.parametrize("ka,er,mr", CASES)
def test_kernel_scalars_match_50_digit_closed_forms(ka, er, mr):
    for R in np.logspace(-8, 1, 31):
        got = oracle.kernel_scalars(ka, er, mr, R)
        ref, Ib = mp_closed(ka, er, mr, R)
        for g, r in zip(got, ref):
            assert abs(g - r) <= 2e-13 * abs(r) + 1e-300, (ka, er, R, g, r)
        A, B = oracle.hdiff(ka, er, mr, R)
        assert abs(A - ref[1]) <= 2e-13 * abs(ref[1])
        assert abs(B - Ib) <= 2e-13 * abs(Ib)


def test_qfuncs_series_and_closed_forms_agree_with_definition():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(3)
    zs = [complex(0, r) for r in np.logspace(-6, 1.5, 25)]
    zs += [complex(-abs(a), b) for a, b in rng.uniform(0, 3, size=(25, 2))]
    for z in zs:
        zz = mp.mpc(z.real, z.imag)
        ez = mp.exp(zz)
        q1 = (zz * zz - zz + 1) * ez - 1 - zz * zz / 2
        q2 = (zz * zz - 3 * zz + 3) * ez - 3 + zz * zz / 2
        q3 = (zz - 1) * ez + 1
        got = oracle.qfuncs(z)
        for g, r in zip(got, (q1, q2, q3)):
            r = complex(r)
            assert abs(g - r) <= 1e-13 * abs(r), (z, g, r)


@pytest.mark.parametrize("ka,er,mr", CASES)
def test_printed_truncated_hdiff_coefficients(ka, er, mr):
    # Eq. (H_diff_truncated): H_diff ~ A R^R^ + B I with
    #  A = (ka^2-ki^2)/(8 pi R) + (ka^4-ki^4) R/(32 pi) + 2i(ka^5-ki^5)R^2/(120 pi)
    #      - 3(ka^6-ki^6) R^3/(576 pi)
    #  B = -(ka^2-ki^2)/(8 pi R) - i(ka^3-ki^3)/(12 pi) + (ka^4-ki^4) R/(32 pi)
    #      + i(ka^5-ki^5) R^2/(120 pi) - (ka^6-ki^6) R^3/(576 pi)
    ki = ki_of(ka, er, mr)
    d = {n: ka ** n - ki ** n for n in range(2, 8)}
    pi = math.pi
    kmax = max(abs(ka), abs(ki))
    for R in (1e-2 / kmax, 3e-3 / kmax, 1e-3 / kmax):
        A = d[2] / (8 * pi * R) + d[4] * R / (32 * pi) + 2j * d[5] * R ** 2 / (120 * pi) \
            - 3 * d[6] * R ** 3 / (576 * pi)
        B = -d[2] / (8 * pi * R) - 1j * d[3] / (12 * pi) + d[4] * R / (32 * pi) \
            + 1j * d[5] * R ** 2 / (120 * pi) - d[6] * R ** 3 / (576 * pi)
        gA, gB = oracle.hdiff(ka, er, mr, R)
        # the first omitted term is O(|k|^7 R^4)
        bound = 0.05 * kmax ** 7 * R ** 4 + 1e-13 * abs(d[2]) / R
        assert abs(gA - A) <= bound, (R, gA, A)
        assert abs(gB - B) <= bound, (R, gB, B)


@pytest.mark.parametrize("ka,er,mr", CASES)
def test_hypersingular_terms_cancel(ka, er, mr):
    # Sec. 2.3: each Hessian is O(R^-3) but the difference is O(R^-1):
    # R * H_diff -> (ka^2 - ki^2)/(8 pi) (R^R^ - I), with a relative
    # correction O(k R).
    ki = ki_of(ka, er, mr)
    kmax = max(abs(ka), abs(ki))
    lim = (ka ** 2 - ki ** 2) / (8 * math.pi)
    for R in np.logspace(-9, -4, 11) / kmax:
        A, B = oracle.hdiff(ka, er, mr, R)
        assert abs(R * A - lim) <= 2 * kmax * R * abs(lim) + 1e-12 * abs(lim)
        assert abs(R * B + lim) <= 2 * kmax * R * abs(lim) + 1e-12 * abs(lim)
        # a single Hessian term grows like R^-3: the difference is far smaller
        assert abs(A) < 1e-3 / (4 * math.pi * R ** 3)


@pytest.mark.parametrize("ka,er,mr", CASES)
def test_singular_parts_and_remainders(ka, er, mr):
    ki = ki_of(ka, er, mr)
    c = 1.0 / (4 * math.pi)
    for R in (1e-6, 1e-3, 0.05, 0.7, 3.0):
        full = oracle.kernel_scalars(ka, er, mr, R, remainder=False)
        rem = oracle.kernel_scalars(ka, er, mr, R, remainder=True)
        s = (ka ** 2 - ki ** 2) / (8 * math.pi * R)  # Eq. (kappa_S)
        de = -(1.0 - complex(er)) / (4 * math.pi * R ** 2)  # Eq. (kappa2_S), chi = eps
        dm = -(1.0 - complex(mr)) / (4 * math.pi * R ** 2)
        np.testing.assert_allclose(full[0] - rem[0], s, rtol=1e-12)
        np.testing.assert_allclose(full[1] - rem[1], s, rtol=1e-12)
        np.testing.assert_allclose(full[2] - rem[2], de, rtol=1e-12)
        np.testing.assert_allclose(full[3] - rem[3], dm, rtol=1e-12)
    # R -> 0 limits of the remainders
    rem = oracle.kernel_scalars(ka, er, mr, 1e-9, remainder=True)
    lim1 = 1j * (ka ** 3 - ki ** 3) / (6 * math.pi)
    assert abs(rem[0] - lim1) < 1e-6 * abs(lim1)
    assert abs(rem[1]) < 1e-6 * abs(lim1)
    lim_e = c * (complex(er) * ki ** 2 - ka ** 2) / 2.0
    assert abs(rem[2] - lim_e) < 1e-6 * max(1.0, abs(lim_e))
