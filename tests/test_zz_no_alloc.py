"""The allocation-free far-field entry point (mueller_far_field_noalloc).

Callers that may not allocate device memory -- a framework whose pool owns
all device memory, or a service that forbids allocation after start-up --
use this variant: its scratch is a fixed device array inside the library.
This test calls it through the C ABI twice in a row and checks both results
against the allocating mueller_far_field, with the far-field tolerances of
the parity tests, and checks that an oversized request is refused.

The file is named so that pytest collects it last."""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_21181_gb300 as mu  # noqa: E402
import workloads  # noqa: E402

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU"),
]


def _call(fn, mesh, p, X, inc, dirs, n_theta, n_phi):
    r = inc.shape[0]
    F = torch.zeros((r, dirs.shape[0], 3), dtype=torch.complex128, device="cuda")
    xs = np.zeros((r, 3))
    cp = p.c()
    st = fn(mesh.h, C.byref(cp), C.c_void_p(X.data_ptr()), r,
            inc.ctypes.data_as(C.POINTER(C.c_double)), dirs.ctypes.data_as(C.POINTER(C.c_double)),
            dirs.shape[0], C.c_void_p(F.data_ptr()), xs.ctypes.data_as(C.POINTER(C.c_double)),
            n_theta, n_phi, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, F.cpu().numpy(), xs


def test_noalloc_far_field_matches_allocating_call_twice():
    lib = mu.load_library()
    xyz, tri6 = workloads.spheroid_p2(2, 1.0, 1.5)
    p = mu.Params(ka=3.0, eps_r=(3.0, 0.2), q_regular=6, ssq_order=4, frame_rule=mu.FRAME_PAPER)
    mesh = mu.Mesh(xyz, tri6)
    mesh.tangent_frame(p.frame_rule, out=False)
    mu.assemble(mesh, p, mu.MUELLER_C128)  # builds the point geometry of the rule
    inc = np.ascontiguousarray(workloads.fibonacci_plane_waves(2))
    g = torch.Generator().manual_seed(17)
    X = torch.randn((inc.shape[0], mesh.N), dtype=torch.complex128, generator=g).cuda()
    dirs = np.ascontiguousarray(workloads.fibonacci_directions(9))

    st, F_ref, xs_ref = _call(lib.mueller_far_field, mesh, p, X, inc, dirs, 24, 48)
    assert st == 0, lib.mueller_last_error()
    for _ in range(2):  # two calls in a row share the same scratch
        st, F, xs = _call(lib.mueller_far_field_noalloc, mesh, p, X, inc, dirs, 24, 48)
        assert st == 0, lib.mueller_last_error()
        np.testing.assert_allclose(F, F_ref, rtol=0, atol=1e-12 * np.abs(F_ref).max())
        np.testing.assert_allclose(xs, xs_ref, rtol=1e-11, atol=1e-14)


def test_noalloc_far_field_refuses_oversized_requests():
    lib = mu.load_library()
    xyz, tri6 = workloads.icosphere_p2(1)
    p = mu.Params(ka=1.0, eps_r=(4.0, 0.0))
    mesh = mu.Mesh(xyz, tri6)
    mesh.tangent_frame(p.frame_rule, out=False)
    inc = np.ascontiguousarray(workloads.plane_wave())
    X = torch.zeros((1, mesh.N), dtype=torch.complex128, device="cuda")
    dirs = np.zeros((1, 3))
    dirs[0, 2] = 1.0
    # no point geometry yet: refused, nothing allocated on its behalf
    st, _, _ = _call(lib.mueller_far_field_noalloc, mesh, p, X, inc, dirs, 24, 48)
    assert st == 9  # MUELLER_ERR_STATE
    mu.assemble(mesh, p, mu.MUELLER_C128)
    # 512 x 1024 sphere directions need ~25 MB of far fields: beyond 16 MiB
    st, _, _ = _call(lib.mueller_far_field_noalloc, mesh, p, X, inc, dirs, 512, 1024)
    assert st == 1  # MUELLER_ERR_INVALID_ARG
    assert b"scratch" in lib.mueller_last_error()
