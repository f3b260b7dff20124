"""The seeded synthetic inputs are what the design notes say they are: P2
icospheres and spheroids (counts, nodes on the surface, closed and outward
oriented), unit plane waves with polarisation orthogonal to the direction,
and the seeded 64-body list (levels, ranges, element pairs)."""

import numpy as np
import pytest

import workloads
from paper_2604_21181_gb300 import api


def _signed_volume(xyz, tri6):
    a, b, c = (xyz[tri6[:, k]] for k in range(3))
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_icosphere_counts_surface_and_orientation(level):
    xyz, tri6 = workloads.icosphere_p2(level)
    assert tri6.shape == (20 * 4 ** level, 6)
    assert xyz.shape == (40 * 4 ** level + 2, 3)  # corners + edge nodes
    assert np.allclose(np.linalg.norm(xyz, axis=1), 1.0, atol=1e-14, rtol=0)
    assert _signed_volume(xyz, tri6) > 0
    m = api.Mesh(xyz, tri6, host_only=True)  # closed, consistently oriented, matching edge nodes
    m.free()


@pytest.mark.parametrize("a,c", [(1.0, 1.5), (1.0, 3.0), (2.0, 1.0)])
def test_spheroid_nodes_on_the_surface(a, c):
    xyz, tri6 = workloads.spheroid_p2(2, a, c)
    q = (xyz[:, 0] ** 2 + xyz[:, 1] ** 2) / a ** 2 + xyz[:, 2] ** 2 / c ** 2
    assert np.allclose(q, 1.0, atol=1e-13, rtol=0)
    assert _signed_volume(xyz, tri6) > 0


def test_plane_waves_are_unit_and_transverse():
    inc = workloads.fibonacci_plane_waves(16)
    assert inc.shape == (32, 6)
    k, p = inc[:, :3], inc[:, 3:]
    assert np.allclose(np.linalg.norm(k, axis=1), 1.0)
    assert np.allclose(np.linalg.norm(p, axis=1), 1.0)
    assert np.allclose(np.einsum("ij,ij->i", k, p), 0.0, atol=1e-15)
    # two polarisations per direction
    assert np.allclose(inc[0::2, :3], inc[1::2, :3])
    assert np.allclose(np.einsum("ij,ij->i", inc[0::2, 3:], inc[1::2, 3:]), 0.0, atol=1e-15)
    d = workloads.fibonacci_directions(50)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    assert np.allclose(np.sort(d[:, 2])[::-1], 1.0 - (2 * np.arange(50) + 1) / 50.0)


def test_multibody_list_is_seeded_and_in_range():
    spec = workloads.multibody_spec()
    assert spec == workloads.multibody_spec()
    assert len(spec) == 64
    levels = [b["level"] for b in spec]
    assert (levels.count(1), levels.count(2), levels.count(3)) == (23, 21, 20)
    for b in spec:
        assert 0.5 <= b["ka"] <= 5.0 and 1.0 <= b["rho"] <= 2.0
        assert 1.5 <= b["eps_r"][0] <= 6.0 and 0.0 <= b["eps_r"][1] <= 1.0
    pairs = sum((20 * 4 ** b["level"]) ** 2 for b in spec)
    assert pairs == 35065600


def test_benchmark_workload_sizes():
    xyz, tri6, inc, w = workloads.workload("sphere_L3_eps2.25_ka5")
    assert tri6.shape[0] == 1280 and 4 * xyz.shape[0] == 10248
    assert inc.shape == (1, 6) and w["ka"] == 5.0
