"""The mesh's host tables (touching pairs, near-block layout; Sec. 4.2, Sec. 5)
built by the library's host thread after mueller_mesh_load returns.

They must equal the tables of a MUELLER_MESH_HOST_ONLY load, which builds
them before returning (that path is checked against the oracle and brute
force on the CPU in test_host_tables.py).  Freeing a mesh right after loading
it, before any call waited for the thread, must be safe, and so must an
assembly issued right after the load, whose regular-pair launch does not wait
for the tables."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("level", [1, 3])
def test_tables_built_beside_the_first_launches_equal_the_host_only_tables(level):
    xyz, tri6 = workloads.icosphere_p2(level)
    for _ in range(4):  # free before anything waited for the table thread
        mu.Mesh(xyz, tri6).free()
    hm = mu.Mesh(xyz, tri6, host_only=True)
    m = mu.Mesh(xyz, tri6)
    info, hinfo = m.info(), hm.info()
    for k in ("n_touching", "n_near_blocks", "n_dof"):
        assert info[k] == hinfo[k], k
    t, ht = m.touching(), hm.touching()
    for k in ("ex", "ey", "cls", "relabel"):
        assert np.array_equal(t[k], ht[k]), k
    for a, b in zip(m.near_layout(), hm.near_layout()):
        assert np.array_equal(a, b)


def test_assembly_issued_right_after_load_matches_a_later_one():
    xyz, tri6 = workloads.icosphere_p2(2)
    p = mu.Params(ka=2.0, eps_r=(2.25, 0.1), ssq_order=3)
    inc = workloads.plane_wave()
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule, out=False)
    near = torch.empty(m.near_bytes() // 16, dtype=torch.complex128, device="cuda")
    Z1, n1, B1 = mu.assemble(m, p, mu.MUELLER_C64_NEAR64, inc=inc, near=near)
    m2 = mu.Mesh(xyz, tri6)
    m2.tangent_frame(p.frame_rule, out=False)
    # near buffer sized from the first mesh: the call below waits for the
    # second mesh's tables only after launching its regular pairs
    Z2, n2, B2 = mu.assemble(m2, p, mu.MUELLER_C64_NEAR64, inc=inc, near=torch.empty_like(near))
    torch.cuda.synchronize()
    # the same kernels on the same mesh; only the order of the atomic additions differs
    assert (Z1 - Z2).abs().max().item() <= 2e-6 * Z1.abs().max().item()
    assert (n1 - n2).abs().max().item() <= 1e-12 * n1.abs().max().item()
    assert (B1 - B2).abs().max().item() <= 1e-13 * B1.abs().max().item()
