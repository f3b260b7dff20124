"""The oracle's cross-section gradient (central differences of its own
pipeline) pinned by the physics of a sphere:

* against the derivative of the Mie series (central differences of the
  closed form) with respect to Re and Im of eps_r, at mu_r = 1, to the
  discretisation accuracy of the level-1 mesh (5 % of each column's largest
  entry; the cross sections themselves are within 0.2 % there);
* by duality: for a sphere the Mie coefficients a_n and b_n swap when eps_r
  and mu_r swap, so at eps_r = mu_r the derivatives with respect to eps_r and
  to mu_r are equal; the discrete method keeps this to 1e-3.
A sign error, a dropped factor or a mixed-up parameter fails one of them."""

import numpy as np

import oracle
import workloads
from oracle import mie

KA = 1.0


def _mesh():
    xyz, tri6 = workloads.icosphere_p2(1)
    return oracle.Mesh(xyz, tri6, frame_rule=1)


def test_eps_gradient_matches_mie_derivative():
    om = _mesh()
    er = (3.0, 0.2)
    pw = dict(ka=KA, eps_r=er, mu_r=(1.0, 0.0), q_regular=6, ssq_order=4)
    J = oracle.cross_section_gradient(om, pw, workloads.plane_wave())
    h = 1e-5
    e0 = complex(*er)
    for k, d in ((0, 1.0), (1, 1j)):
        dm = (np.array(mie.mie_bh(KA, e0 + h * d)) - np.array(mie.mie_bh(KA, e0 - h * d))) / (2 * h)
        assert np.all(np.abs(J[:, k] - dm) <= 0.05 * np.abs(dm).max()), (k, J[:, k], dm)


def test_duality_of_eps_and_mu_gradients_on_a_sphere():
    om = _mesh()
    pw = dict(ka=KA, eps_r=(2.0, 0.1), mu_r=(2.0, 0.1), q_regular=6, ssq_order=4)
    J = oracle.cross_section_gradient(om, pw, workloads.plane_wave())
    for k in (0, 1):
        assert np.all(np.abs(J[:, k] - J[:, k + 2]) <= 1e-3 * np.abs(J[:, k]).max()), (J[:, k], J[:, k + 2])
