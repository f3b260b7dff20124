"""Argument checks of the C ABI that need no GPU: every entry point rejects a
NULL handle or buffer, and invalid parameters, sizes and mode/dtype
combinations, with MUELLER_ERR_INVALID_ARG (1) and a message naming the
problem, before any device work.

Where a check follows the NULL checks, the handles and device buffers are
stand-ins (addresses of a zeroed host buffer): each case below is rejected
by a check that comes before the library's first use of them."""

import ctypes as C

import numpy as np
import pytest

from paper_2604_21181_gb300 import api

INVALID_ARG = 1


@pytest.fixture(scope="module")
def lib():
    return api.load_library()


@pytest.fixture(scope="module")
def fake():
    buf = C.create_string_buffer(1 << 16)
    return buf, C.cast(buf, C.c_void_p)


def _params(**kw):
    p = dict(ka=1.0, eps_r=(2.0, 0.0), mu_r=(1.0, 0.0), q_regular=6, ssq_order=4, frame_rule=0)
    p.update(kw)
    c = api.CParams()
    c.ka = p["ka"]
    c.eps_r[0], c.eps_r[1] = p["eps_r"]
    c.mu_r[0], c.mu_r[1] = p["mu_r"]
    c.q_regular, c.ssq_order, c.frame_rule = p["q_regular"], p["ssq_order"], p["frame_rule"]
    return c


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _err(lib):
    return lib.mueller_last_error().decode()


def test_null_handles_are_rejected(lib):
    p = _params()
    info = api.CMeshInfo()
    assert lib.mueller_mesh_get_info(None, C.byref(info)) == INVALID_ARG
    assert lib.mueller_mesh_perm(None, None, None) == INVALID_ARG
    assert lib.mueller_tangent_frame(None, 0, None, None) == INVALID_ARG
    assert lib.mueller_assemble(None, C.byref(p), api.MUELLER_C128, None, 0, None, None, None,
                                0, None) == INVALID_ARG
    assert lib.mueller_dz_matvec(None, C.byref(p), 1, None, None, None) == INVALID_ARG
    g = np.zeros(3)
    assert lib.mueller_zshape_vjp(None, C.byref(p), None, None, _dp(g), None) == INVALID_ARG
    assert lib.mueller_zshape_vjp_multi(None, C.byref(p), None, 1, None, _dp(g), None) == INVALID_ARG
    assert lib.mueller_point_records(None, 6, _dp(g)) == INVALID_ARG
    inc = np.zeros((1, 6))
    xs = np.zeros((1, 3))
    assert lib.mueller_far_field(None, C.byref(p), None, 1, _dp(inc), None, 0, None, _dp(xs),
                                 8, 16, None) == INVALID_ARG
    assert lib.mueller_far_field_noalloc(None, C.byref(p), None, 1, _dp(inc), None, 0, None,
                                         _dp(xs), 8, 16, None) == INVALID_ARG
    assert lib.mueller_precond_build(None, 16, None, None) == INVALID_ARG
    assert lib.mueller_solve(None, None, None, 1, None, None, None, 0, None) == INVALID_ARG
    assert lib.mueller_matvec(None, None, None, 1, None, 0, None) == INVALID_ARG
    assert lib.mueller_matvec_mrhs(None, None, None, 1, None, 0, None) == INVALID_ARG
    assert lib.mueller_assemble_batch(0, None, None, api.MUELLER_C128, None, None, None, None,
                                      None, None, None) == INVALID_ARG
    # a NULL operator has no workspace; a NULL mesh no near blocks
    assert lib.mueller_solve_workspace_bytes(None, 1, None) == 0
    assert lib.mueller_matvec_workspace_bytes(None, 1) == 0
    assert lib.mueller_near_bytes(None) == 0


@pytest.mark.parametrize("kw,word", [
    (dict(ka=0.0), "ka"), (dict(ka=-1.0), "ka"), (dict(ka=float("inf")), "ka"),
    (dict(ka=float("nan")), "ka"), (dict(q_regular=7), "q_regular"), (dict(ssq_order=0), "ssq_order"),
    (dict(ssq_order=17), "ssq_order"), (dict(eps_r=(0.0, 0.0)), "eps_r"),
    (dict(mu_r=(0.0, 0.0)), "mu_r"), (dict(eps_r=(float("nan"), 0.0)), "material"),
    (dict(mu_r=(1.0, float("inf"))), "material")])
def test_invalid_params_are_rejected(lib, fake, kw, word):
    _, h = fake
    p = _params(**kw)
    inc = np.zeros((1, 6))
    xs = np.zeros((1, 3))
    for fn in (lib.mueller_far_field, lib.mueller_far_field_noalloc):
        assert fn(h, C.byref(p), h, 1, _dp(inc), None, 0, None, _dp(xs), 8, 16, None) == INVALID_ARG
        assert word in _err(lib), _err(lib)
    assert lib.mueller_assemble(h, C.byref(p), api.MUELLER_C128, h, 1 << 20, None, None, None, 0,
                                None) == INVALID_ARG
    assert word in _err(lib)
    assert lib.mueller_dz_matvec(h, C.byref(p), 1, h, h, None) == INVALID_ARG
    assert lib.mueller_assemble(h, None, api.MUELLER_C128, h, 1 << 20, None, None, None, 0,
                                None) == INVALID_ARG  # params NULL
    assert "params" in _err(lib)


@pytest.mark.parametrize("r,ndir,n_theta,n_phi", [
    (0, 0, 8, 16), (1, -1, 8, 16), (1, 3, 8, 16),  # ndir > 0 without dirs / F
    (1, 0, 1, 16), (1, 0, 513, 16), (1, 0, 8, 2), (1, 0, 8, 1025)])
def test_far_field_sizes_are_checked(lib, fake, r, ndir, n_theta, n_phi):
    _, h = fake
    p = _params()
    inc = np.zeros((1, 6))
    xs = np.zeros((1, 3))
    for fn in (lib.mueller_far_field, lib.mueller_far_field_noalloc):
        assert fn(h, C.byref(p), h, r, _dp(inc), None, ndir, None, _dp(xs), n_theta, n_phi,
                  None) == INVALID_ARG


def test_zshape_vjp_multi_needs_a_vector(lib, fake):
    _, h = fake
    p = _params()
    g = np.zeros(3)
    assert lib.mueller_zshape_vjp_multi(h, C.byref(p), h, 0, h, _dp(g), None) == INVALID_ARG


def test_dz_matvec_parameter_index_is_checked(lib, fake):
    _, h = fake
    p = _params()
    for which in (0, 3, -1):
        assert lib.mueller_dz_matvec(h, C.byref(p), which, h, h, None) == INVALID_ARG
        assert "which" in _err(lib)


def _op(h, dtype, near=True, precond=False):
    op = api.COperator()
    op.mesh, op.Z_dev, op.ldz, op.dtype = h, h, 1 << 20, dtype
    op.near_dev = h if near else None
    op.precond_dev = h if precond else None
    return op


def _opts(**kw):
    o = api.CSolverOpts()
    o.mode, o.restart, o.maxit, o.tol = api.SOLVE_GMRES_IR, 30, 100, 1e-8
    o.inner_tol, o.max_refine, o.use_precond = 1e-5, 5, 0
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("dtype,r,kw,word", [
    (api.MUELLER_C64_NEAR64, 0, {}, "r must"),
    (api.MUELLER_C64_NEAR64, 1, dict(mode=3), "mode"),
    (api.MUELLER_C64_NEAR64, 1, dict(mode=-1), "mode"),
    (api.MUELLER_C64_NEAR64, 1, dict(restart=0), "restart"),
    (api.MUELLER_C64_NEAR64, 1, dict(maxit=0), "restart"),
    (api.MUELLER_C64_NEAR64, 1, dict(tol=0.0), "tol"),
    (api.MUELLER_C64_NEAR64, 1, dict(tol=float("nan")), "tol"),
    (api.MUELLER_C64_NEAR64, 1, dict(mode=api.SOLVE_DENSE_LU), "complex128"),
    (api.MUELLER_C128, 1, dict(mode=api.SOLVE_GMRES_IR), "C64_NEAR64"),
    (api.MUELLER_C64_NEAR64, 1, dict(use_precond=1), "precond")])
def test_solve_options_are_checked(lib, fake, dtype, r, kw, word):
    _, h = fake
    op = _op(h, dtype)
    o = _opts(**kw)
    info = api.CSolveInfo()
    assert lib.mueller_solve(C.byref(op), h, h, r, C.byref(o), C.byref(info), None, 0,
                             None) == INVALID_ARG
    assert word in _err(lib), _err(lib)


def test_operator_checks(lib, fake):
    _, h = fake
    # block size, and a mixed operator without its near blocks
    op = _op(h, api.MUELLER_C64_NEAR64)
    assert lib.mueller_precond_build(C.byref(op), 0, h, None) == INVALID_ARG
    assert "block" in _err(lib)
    op = _op(h, api.MUELLER_C64_NEAR64, near=False)
    assert lib.mueller_precond_build(C.byref(op), 64, h, None) == INVALID_ARG
    assert "near" in _err(lib)
    # the tensor-core product is for mixed operators only
    op = _op(h, api.MUELLER_C128)
    assert lib.mueller_matvec_mrhs(C.byref(op), h, h, 4, h, 1 << 20, None) == INVALID_ARG
    assert "C64_NEAR64" in _err(lib)


def test_matvec_checks(lib, fake):
    _, h = fake
    op = _op(h, api.MUELLER_C64_NEAR64)
    assert lib.mueller_matvec(C.byref(op), h, h, 0, None, 0, None) == INVALID_ARG
    assert "r must" in _err(lib)
    op = _op(h, api.MUELLER_C64_NEAR64, near=False)
    assert lib.mueller_matvec(C.byref(op), h, h, 1, None, 0, None) == INVALID_ARG
    assert lib.mueller_matvec_workspace_bytes(C.byref(op), 0) == 0
