"""The FP64 product with a stored complex64 operator (the refinement
residual) widens every float to double exactly, zeros and subnormal floats
included: on an operator whose only nonzero entries are planted special
values, mueller_matvec's FP64 result equals NumPy's complex128 product of the
same entries, element by element (relative 1e-14)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
]

SPECIAL = np.array([1e-40, -1e-40, 1.4e-45, 1.1754944e-38, 0.0, -0.0, 3.0e38, -2.5],
                   dtype=np.float32)


def test_fp64_product_widens_special_floats_exactly():
    xyz, tri6 = workloads.icosphere_p2(1)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(0, out=False)
    Z, near, _ = mu.assemble(m, mu.Params(ka=2.0, eps_r=(3.0, 0.1)), mu.MUELLER_C64_NEAR64)
    near.zero_()
    Zh = np.zeros((m.N, m.N), np.complex64)
    g = np.random.default_rng(5)
    # row i holds special values of one magnitude class only
    for i in range(m.N):
        v = SPECIAL[i % len(SPECIAL)]
        w = SPECIAL[(i // len(SPECIAL)) % len(SPECIAL)]
        if abs(float(v)) > 1e30 or abs(float(w)) > 1e30:
            v, w = np.float32(3.0e38), np.float32(0.0)
        elif abs(float(v)) >= 1e-30 or abs(float(w)) >= 1e-30:
            v, w = np.float32(-2.5), np.float32(1.5)
        for j in g.integers(0, m.N, 3):
            Zh[i, j] = np.complex64(complex(v, w))
    Z.copy_(torch.from_numpy(Zh).cuda())
    op = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    X = g.standard_normal((2, m.N)) + 1j * g.standard_normal((2, m.N))
    Y = mu.matvec(op, torch.tensor(X, dtype=torch.complex128, device="cuda")).cpu().numpy()
    expect = (Zh.astype(np.complex128) @ X.T).T
    assert np.all(np.isfinite(Y))
    err = np.abs(Y - expect)
    assert np.all(err <= 1e-14 * np.abs(expect) + 1e-320), err.max()
    tiny = np.abs(expect) < 1e-30
    assert tiny.any()
