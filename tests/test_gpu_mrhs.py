"""Tensor-core multi-RHS product (tcgen05, TF32 head/remainder split) against
the FP64 product of the same stored operator.  Sizes span several 128-row
tiles with ragged M and K edges, several right-hand-side counts (padded MMA N;
up to 64 the head meets [B'hi; B'lo] in one MMA, above it in two), and
stream-K ranges that cross row tiles."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
]

_ops = {}


def operator(level):
    if level not in _ops:
        xyz, tri6 = workloads.icosphere_p2(level)
        p = mu.Params(ka=5.0, eps_r=(2.25, 0.0))
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(p.frame_rule, out=False)
        Z, near, _ = mu.assemble(m, p, mu.MUELLER_C64_NEAR64)
        _ops[level] = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    return _ops[level]


@pytest.mark.parametrize("level,r", [(1, 1), (2, 8), (2, 13), (2, 16), (3, 16), (3, 40), (2, 72), (2, 128)])
def test_tensor_core_product_matches_fp64(level, r):
    op = operator(level)
    N = op.mesh.N
    g = torch.Generator().manual_seed(100 + r)
    X = (torch.randn((r, N), generator=g) + 1j * torch.randn((r, N), generator=g)).to(torch.complex64)
    Y = mu.matvec_mrhs(op, X.cuda()).cpu().numpy().astype(np.complex128)
    ref = mu.matvec(op, X.to(torch.complex128).cuda()).cpu().numpy()
    err = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    # FP32 accumulation over K = 2N real terms: 4 u sqrt(2N), u = 2^-24
    tol = 4 * 2.0 ** -24 * np.sqrt(2 * N)
    assert err.max() <= tol, (err.max(), tol)
