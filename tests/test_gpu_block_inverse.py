"""Block-Jacobi inverses of the mixed operator (Sec. 5, Eq. precond_block)
against NumPy's complex128 inverses of the same Morton blocks.

The blocks are taken from the stored operator itself (its FP64 products with
the identity's columns), so the check covers the gather of the blocks, the
FP64 LU with its row swaps and the complex64 inverse formed from the factors,
including ragged last blocks and block sizes that are not multiples of the
32-row tiles."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("level,block", [(1, 37), (1, 128), (2, 300)])
def test_complex64_block_inverses_match_numpy(level, block):
    xyz, tri6 = workloads.icosphere_p2(level)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(0, out=False)
    p = mu.Params(ka=2.0, eps_r=(2.25, 0.1), ssq_order=3)
    Z, near, _ = mu.assemble(m, p, mu.MUELLER_C64_NEAR64)
    op = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    P = mu.precond_build(op, block)
    N = m.N
    H = N // 2
    eye = torch.eye(N, dtype=torch.complex128, device="cuda")
    Zd = mu.matvec(op, eye).cpu().numpy().T  # column j = Z e_j
    nb, d = (H + block - 1) // block, 2 * min(block, H)
    n_inv = nb * d * d
    inv = P[: n_inv * 8].view(torch.complex64).reshape(nb, d, d).cpu().numpy()
    sizes = P[n_inv * 8: n_inv * 8 + 4 * nb].view(torch.int32).cpu().numpy()
    worst = 0.0
    for b in range(nb):
        n = int(sizes[b])
        half, o = n // 2, b * block
        idx = np.r_[o:o + half, H + o:H + o + half]
        ref = np.linalg.inv(Zd[np.ix_(idx, idx)])
        err = np.abs(inv[b, :n, :n] - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
    # complex64 inverse of a well-conditioned block: a few hundred FP32 ulps
    assert worst <= 5e-5, worst
