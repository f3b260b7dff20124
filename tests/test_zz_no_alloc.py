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


def _pool_used_high():
    """(used, high-water mark) of the device's default memory pool, through
    the driver API (the pool that cudaMallocAsync draws from)."""
    cu = C.CDLL("libcuda.so.1")
    dev = C.c_int()
    assert cu.cuDeviceGet(C.byref(dev), torch.cuda.current_device()) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    used, high = C.c_uint64(), C.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, 7, C.byref(used)) == 0  # USED_MEM_CURRENT
    assert cu.cuMemPoolGetAttribute(pool, 8, C.byref(high)) == 0  # USED_MEM_HIGH
    return cu, pool, used.value, high.value


def _pool_reset_high():
    cu, pool, _, _ = _pool_used_high()
    zero = C.c_uint64(0)
    assert cu.cuMemPoolSetAttribute(pool, 8, C.byref(zero)) == 0  # high mark := current


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


def test_noalloc_far_field_allocates_no_device_memory():
    """After a first call (which looks up the scratch address), further calls
    leave every allocator's figure where it was: the default memory pool's
    used bytes and high-water mark (cudaMallocAsync), PyTorch's allocator
    and the driver's free memory (cudaMalloc)."""
    lib = mu.load_library()
    xyz, tri6 = workloads.icosphere_p2(2)
    p = mu.Params(ka=2.0, eps_r=(2.25, 0.1), q_regular=6, ssq_order=3)
    mesh = mu.Mesh(xyz, tri6)
    mesh.tangent_frame(p.frame_rule, out=False)
    mu.assemble(mesh, p, mu.MUELLER_C128)
    inc = np.ascontiguousarray(workloads.fibonacci_plane_waves(2))
    X = torch.randn((inc.shape[0], mesh.N), dtype=torch.complex128,
                    generator=torch.Generator().manual_seed(3)).cuda()
    dirs = np.ascontiguousarray(workloads.fibonacci_directions(5))
    F = torch.zeros((inc.shape[0], dirs.shape[0], 3), dtype=torch.complex128, device="cuda")
    xs = np.zeros((inc.shape[0], 3))
    cp = p.c()
    args = (mesh.h, C.byref(cp), C.c_void_p(X.data_ptr()), inc.shape[0],
            inc.ctypes.data_as(C.POINTER(C.c_double)), dirs.ctypes.data_as(C.POINTER(C.c_double)),
            dirs.shape[0], C.c_void_p(F.data_ptr()), xs.ctypes.data_as(C.POINTER(C.c_double)),
            24, 48, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert lib.mueller_far_field_noalloc(*args) == 0, lib.mueller_last_error()
    torch.cuda.synchronize()
    _pool_reset_high()
    _, _, used0, _ = _pool_used_high()
    torch_alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.mueller_far_field_noalloc(*args) == 0, lib.mueller_last_error()
    torch.cuda.synchronize()
    _, _, used1, high1 = _pool_used_high()
    assert used1 == used0 and high1 == used0, (used0, used1, high1)
    assert torch.cuda.memory_allocated() == torch_alloc0
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_far_field_size_limit_at_level3():
    """The documented limit: the level-3 sphere (Q = 6) with the 48 x 96
    sphere rule needs about 0.97 MB per right-hand side, so 17 right-hand
    sides fit in the 16 MiB scratch and 18 are refused."""
    lib = mu.load_library()
    xyz, tri6 = workloads.icosphere_p2(3)
    p = mu.Params(ka=5.0, eps_r=(2.25, 0.0), q_regular=6, ssq_order=2)
    mesh = mu.Mesh(xyz, tri6)
    mesh.tangent_frame(p.frame_rule, out=False)
    mu.assemble(mesh, p, mu.MUELLER_C64_NEAR64)
    dirs = np.zeros((0, 3))
    for r, want in ((17, 0), (18, 1)):
        inc = np.ascontiguousarray(workloads.fibonacci_plane_waves(9)[:r])
        X = torch.zeros((r, mesh.N), dtype=torch.complex128, device="cuda")
        st, _, xs = _call(lib.mueller_far_field_noalloc, mesh, p, X, inc, dirs, 48, 96)
        assert st == want, (r, st, lib.mueller_last_error())
        if want == 0:
            assert np.all(xs == 0.0)  # zero currents radiate nothing


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
