"""Pair-tile shapes of the regular-pair kernel (the autotuner's candidates):
every shape, forced through MUELLER_REGULAR_TILE, gives the oracle's matrix
(FP64 path, max |Z_gpu - Z_oracle| / max |Z_oracle| <= 1e-11 per quadrant)
or, where its staging does not fit in shared memory (in FP64), is refused;
the tuned default gives the same matrix."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
]

SHAPES = 4
_ref = {}


def quadrant_err(A, B):
    H = A.shape[0] // 2
    out = []
    for r in (slice(0, H), slice(H, None)):
        for c in (slice(0, H), slice(H, None)):
            ref = np.abs(B[r, c]).max()
            out.append(np.abs(A[r, c] - B[r, c]).max() / max(ref, 1e-300))
    return max(out)


def reference(q):
    if q not in _ref:
        xyz, tri6 = workloads.spheroid_p2(1, 1.0, 1.3)
        pw = dict(ka=2.0, eps_r=(3.0, 0.3), mu_r=(1.0, 0.0), q_regular=q, ssq_order=3)
        _ref[q] = (xyz, tri6, pw, oracle.Mesh(xyz, tri6, frame_rule=0).assemble(pw))
    return _ref[q]


def assemble(q, shape):
    xyz, tri6, pw, _ = reference(q)
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(0, out=False)
    p = mu.Params(ka=pw["ka"], eps_r=pw["eps_r"], q_regular=q, ssq_order=3, frame_rule=0)
    old = os.environ.get("MUELLER_REGULAR_TILE")
    try:
        if shape is None:
            os.environ.pop("MUELLER_REGULAR_TILE", None)
        else:
            os.environ["MUELLER_REGULAR_TILE"] = str(shape)
        Z, _, _ = mu.assemble(m, p, mu.MUELLER_C128)
    finally:
        if old is None:
            os.environ.pop("MUELLER_REGULAR_TILE", None)
        else:
            os.environ["MUELLER_REGULAR_TILE"] = old
    return Z.cpu().numpy()


@pytest.mark.parametrize("shape", range(SHAPES))
def test_every_tile_shape_matches_oracle_or_is_refused_q6(shape):
    Zo = reference(6)[3]
    try:
        Z = assemble(6, shape)
    except mu.MuellerError as e:  # an FP64 shape whose staging exceeds shared memory
        assert e.status == 1 and "shared memory" in str(e)
        assert shape == 1
        return
    assert quadrant_err(Z, Zo) <= 1e-11


def test_tile_shapes_at_q12_fit_or_are_refused():
    Zo = reference(12)[3]
    ok = 0
    for shape in range(SHAPES):
        try:
            Z = assemble(12, shape)
        except mu.MuellerError as e:
            assert e.status == 1 and "shared memory" in str(e)
            continue
        assert quadrant_err(Z, Zo) <= 1e-11
        ok += 1
    assert ok >= 2


def test_autotuned_shape_matches_oracle():
    Zo = reference(6)[3]
    for _ in range(2):  # tuned on the first call, cached on the second
        assert quadrant_err(assemble(6, None), Zo) <= 1e-11
