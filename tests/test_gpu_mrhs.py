"""Tensor-core multi-RHS product (tcgen05, TF32 head/remainder split) against
NumPy's complex128 product of the same stored operator: the complex64 far
part Z (read as exact values) plus the FP64 near blocks, rebuilt on the host
from the mesh's near-block layout.  Compared element by element.  Sizes span
several 128-row tiles with ragged M and K edges, several right-hand-side
counts (padded MMA N; up to 64 the head meets [B'hi; B'lo] in one MMA, above
it in two), and stream-K ranges that cross row tiles."""

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
    """(operator, host complex128 copy of Z, host near part as (rows, cols, vals))."""
    if level not in _ops:
        _ops.clear()
        xyz, tri6 = workloads.icosphere_p2(level)
        p = mu.Params(ka=5.0, eps_r=(2.25, 0.0))
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(p.frame_rule, out=False)
        Z, near, _ = mu.assemble(m, p, mu.MUELLER_C64_NEAR64)
        op = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
        Zh = Z.cpu().numpy()
        # near part: block q of test node i, trial node col[q], entry
        # [h, alpha, g, beta] at row h*H + 2i + alpha, column g*H + 2j + beta
        rowptr, col, _ = m.near_layout()
        H = m.N // 2
        blocks = near.cpu().numpy().reshape(-1, 2, 2, 2, 2)
        i_of_q = np.repeat(np.arange(m.nn), np.diff(rowptr))
        h, a, g, b = np.meshgrid(*([np.arange(2)] * 4), indexing="ij")
        rows = (h[None] * H + 2 * i_of_q[:, None, None, None, None] + a[None]).ravel()
        cols = (g[None] * H + 2 * col[:, None, None, None, None] + b[None]).ravel()
        _ops[level] = (op, Zh, (rows, cols, blocks.ravel()))
    return _ops[level]


def numpy_product(Zh, near, X):
    """Y = X (Z + near)^T in complex128, and the elementwise scale |X| (|Z| +
    |near|)^T that bounds the rounding of an FP32-accumulated product."""
    rows, cols, vals = near
    Y = X @ Zh.T.astype(np.complex128)
    S = np.abs(X) @ np.abs(Zh).T.astype(np.float64)
    for s in range(X.shape[0]):
        Y[s] += np.bincount(rows, weights=(vals * X[s, cols]).real, minlength=Zh.shape[0]) + \
            1j * np.bincount(rows, weights=(vals * X[s, cols]).imag, minlength=Zh.shape[0])
        S[s] += np.bincount(rows, weights=np.abs(vals) * np.abs(X[s, cols]), minlength=Zh.shape[0])
    return Y, S


@pytest.mark.parametrize("level,r", [(1, 1), (2, 1), (2, 8), (2, 13), (2, 16), (2, 40), (2, 72),
                                     (2, 128), (3, 1), (3, 16), (3, 40), (3, 72)])
def test_tensor_core_product_matches_numpy(level, r):
    op, Zh, near = operator(level)
    N = op.mesh.N
    g = torch.Generator().manual_seed(100 + r)
    X = (torch.randn((r, N), generator=g) + 1j * torch.randn((r, N), generator=g)).to(torch.complex64)
    Y = mu.matvec_mrhs(op, X.cuda()).cpu().numpy().astype(np.complex128)
    ref, scale = numpy_product(Zh, near, X.numpy().astype(np.complex128))
    # FP32 accumulation over K = 2N real terms, each term's operands split
    # into TF32 head + remainder (lo x lo dropped): per element
    # |Y - ref| <= 4 u sqrt(2N) (|X| (|Z| + |near|)^T), u = 2^-24
    tol = 4 * 2.0 ** -24 * np.sqrt(2 * N)
    err = np.abs(Y - ref) / scale
    assert err.max() <= tol, (err.max(), tol)
    # and the norm-wise relative error per right-hand side
    rel = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= tol, (rel.max(), tol)
