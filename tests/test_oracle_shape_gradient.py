"""The oracle's derivatives of the cross sections with respect to the node
coordinates (central differences of its own pipeline), pinned by geometry and
the physics of a sphere:

* scaling: moving every node of a sphere along its position vector is a
  dilation, C(s xyz) = s^2 C_Mie(k_a s) for the exact sphere, so the
  derivative along V = xyz is 2 C + k_a dC/dk_a of the Mie series, to the
  discretisation accuracy of the level-1 mesh (5 % of the largest entry);
* translation invariance: a rigid shift only multiplies the currents by a
  phase, so the gradient summed over all nodes vanishes along each axis
  (level 0, every coordinate);
* the full gradient contracted with the node positions equals the
  derivative along V = xyz (linearity: a node or axis mix-up fails it).
"""

import numpy as np
import pytest

import oracle
import workloads
from oracle import mie

KA = 1.0
EPS = (3.0, 0.2)
PW = dict(ka=KA, eps_r=EPS, mu_r=(1.0, 0.0), q_regular=6, ssq_order=4)


def test_dilation_matches_mie_size_derivative():
    xyz, tri6 = workloads.icosphere_p2(1)
    d = oracle.cross_section_shape_derivative(xyz, tri6, PW, workloads.plane_wave(), xyz,
                                              frame_rule=1)[0]
    e0 = complex(*EPS)
    h = 1e-5
    c0 = np.array(mie.mie_bh(KA, e0))
    dk = (np.array(mie.mie_bh(KA + h, e0)) - np.array(mie.mie_bh(KA - h, e0))) / (2 * h)
    ref = 2.0 * c0 + KA * dk
    assert np.all(np.abs(d - ref) <= 0.05 * np.abs(ref).max()), (d, ref)


@pytest.fixture(scope="module")
def level0_gradient():
    xyz, tri6 = workloads.icosphere_p2(0)
    inc = workloads.plane_wave()
    G = oracle.cross_section_coordinate_gradient(xyz, tri6, PW, inc, frame_rule=1)
    return xyz, tri6, inc, G


def test_gradient_sums_to_zero_under_translation(level0_gradient):
    xyz, tri6, inc, G = level0_gradient
    scale = np.abs(G).max()
    assert scale > 1e-2
    for ax in range(3):
        assert np.all(np.abs(G[:, ax, :].sum(axis=0)) <= 1e-5 * scale), G[:, ax, :].sum(axis=0)
    # and the directional derivative along a rigid shift vanishes too
    V = np.tile([0.3, -0.5, 0.8], (xyz.shape[0], 1))
    d = oracle.cross_section_shape_derivative(xyz, tri6, PW, inc, V, frame_rule=1)[0]
    assert np.all(np.abs(d) <= 1e-5 * scale), d


def test_gradient_contracted_with_positions_is_the_dilation_derivative(level0_gradient):
    xyz, tri6, inc, G = level0_gradient
    d = oracle.cross_section_shape_derivative(xyz, tri6, PW, inc, xyz, frame_rule=1)[0]
    g = np.einsum("kd,kdc->c", xyz, G)
    assert np.all(np.abs(g - d) <= 1e-5 * np.abs(d).max()), (g, d)
