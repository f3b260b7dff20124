"""Thin Python binding of libmueller.so (argument marshalling only).

Every computation of the method runs in the library's CUDA kernels; PyTorch
provides device memory (tensors) and the current CUDA stream.  The names
follow the C ABI in ``include/mueller.h``.  There is no CPU fallback: if the
library or a GPU is missing, the calls raise.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import buildlib as _build

MUELLER_C128 = 0
MUELLER_C64_NEAR64 = 1
MUELLER_OP_K1_MIRRORED = 1
MUELLER_OP_ADJOINT = 2
SOLVE_DENSE_LU = 0
SOLVE_GMRES = 1
SOLVE_GMRES_IR = 2
RULE_TRIANGLE = 0
RULE_GAUSS_LEGENDRE = 1
MESH_KEEP_ORDER = 1
MESH_HOST_ONLY = 2
FRAME_PAPER = 0
FRAME_POLAR = 1

STATUS = {
    0: "ok", 1: "invalid argument", 2: "invalid mesh", 3: "degenerate tangent frame",
    4: "singular preconditioner block", 5: "not converged", 6: "device wait timed out",
    7: "CUDA error", 8: "out of device memory", 9: "call order violated",
    10: "NaN or infinite residual",
}


class MuellerError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CParams(C.Structure):
    _fields_ = [("ka", C.c_double), ("eps_r", C.c_double * 2), ("mu_r", C.c_double * 2),
                ("q_regular", C.c_int32), ("ssq_order", C.c_int32), ("frame_rule", C.c_int32),
                ("reserved", C.c_int32)]


class CMeshInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tri", C.c_int64), ("n_dof", C.c_int64),
                ("n_touching", C.c_int64), ("n_near_blocks", C.c_int64),
                ("min_gs_norm", C.c_double)]


class CSolverOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("restart", C.c_int32), ("maxit", C.c_int32),
                ("warm_start", C.c_int32), ("tol", C.c_double), ("inner_tol", C.c_double),
                ("max_refine", C.c_int32), ("use_precond", C.c_int32)]


class CSolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("refinements", C.c_int32),
                ("converged", C.c_int32), ("relres", C.c_double), ("t_ms", C.c_double)]


class COperator(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("Z_dev", C.c_void_p), ("ldz", C.c_int64),
                ("dtype", C.c_int32), ("flags", C.c_int32), ("near_dev", C.c_void_p),
                ("precond_dev", C.c_void_p), ("block", C.c_int64)]


EXPORTS = [
    "mueller_version", "mueller_last_error", "mueller_status_string", "mueller_mesh_load",
    "mueller_mesh_free", "mueller_mesh_get_info", "mueller_mesh_perm", "mueller_mesh_touching",
    "mueller_mesh_near_layout", "mueller_quadrature_rule", "mueller_tangent_frame",
    "mueller_assemble", "mueller_dz_matvec", "mueller_near_bytes", "mueller_precond_build",
    "mueller_precond_bytes",
    "mueller_solve", "mueller_solve_workspace_bytes", "mueller_matvec",
    "mueller_matvec_workspace_bytes", "mueller_far_field", "mueller_sync",
    "mueller_profile_enable", "mueller_profile_reset", "mueller_launch_count",
    "mueller_profile_get", "mueller_profile_names", "mueller_far_field_noalloc",
    "mueller_matvec_mrhs", "mueller_matvec_mrhs_workspace_bytes", "mueller_assemble_batch",
    "mueller_precond_build_batch", "mueller_zshape_vjp", "mueller_zshape_vjp_multi",
    "mueller_point_records",
    "mueller_rhs_shape_vjp",
    "mueller_cross_section_partials",
]

_lib = None


def load_library(build_if_missing: bool = True):
    """Load libmueller.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libmueller.so not found at {path}; run paper_2604_21181_gb300.build")
    lib = C.CDLL(path)
    vp, i32, i64, d, dp, ip = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    sig = {
        "mueller_version": (i32, []),
        "mueller_last_error": (C.c_char_p, []),
        "mueller_status_string": (C.c_char_p, [C.c_int]),
        "mueller_mesh_load": (C.c_int, [dp, i64, ip, i64, i32, vp, C.POINTER(vp)]),
        "mueller_mesh_free": (None, [vp]),
        "mueller_mesh_get_info": (C.c_int, [vp, C.POINTER(CMeshInfo)]),
        "mueller_mesh_perm": (C.c_int, [vp, ip, ip]),
        "mueller_mesh_touching": (C.c_int, [vp, ip, ip, ip, ip]),
        "mueller_quadrature_rule": (C.c_int, [i32, i32, dp, dp, dp]),
        "mueller_mesh_near_layout": (C.c_int, [vp, ip, ip, ip]),
        "mueller_tangent_frame": (C.c_int, [vp, i32, vp, vp]),
        "mueller_assemble": (C.c_int, [vp, C.POINTER(CParams), i32, vp, i64, vp, vp, dp, i32, vp]),
        "mueller_dz_matvec": (C.c_int, [vp, C.POINTER(CParams), i32, vp, vp, vp]),
        "mueller_zshape_vjp": (C.c_int, [vp, C.POINTER(CParams), vp, vp, dp, vp]),
        "mueller_zshape_vjp_multi": (C.c_int, [vp, C.POINTER(CParams), vp, i32, vp, dp, vp]),
        "mueller_point_records": (C.c_int, [vp, i32, dp]),
        "mueller_rhs_shape_vjp": (C.c_int, [vp, C.POINTER(CParams), vp, dp, dp, vp]),
        "mueller_cross_section_partials": (C.c_int, [vp, C.POINTER(CParams), vp, dp, i32, i32, vp,
                                                     dp, dp, vp]),
        "mueller_near_bytes": (C.c_size_t, [vp]),
        "mueller_precond_build": (C.c_int, [C.POINTER(COperator), i64, vp, vp]),
        "mueller_precond_bytes": (C.c_size_t, [i64, i64]),
        "mueller_precond_build_batch": (C.c_int, [i32, C.POINTER(COperator), C.POINTER(i64),
                                                  C.POINTER(vp), vp]),
        "mueller_solve": (C.c_int, [C.POINTER(COperator), vp, vp, i32, C.POINTER(CSolverOpts),
                                    C.POINTER(CSolveInfo), vp, C.c_size_t, vp]),
        "mueller_solve_workspace_bytes": (C.c_size_t, [C.POINTER(COperator), i32, C.POINTER(CSolverOpts)]),
        "mueller_matvec": (C.c_int, [C.POINTER(COperator), vp, vp, i32, vp, C.c_size_t, vp]),
        "mueller_matvec_workspace_bytes": (C.c_size_t, [C.POINTER(COperator), i32]),
        "mueller_far_field": (C.c_int, [vp, C.POINTER(CParams), vp, i32, dp, dp, i64, vp, dp,
                                        i32, i32, vp]),
        "mueller_sync": (C.c_int, [vp]),
        "mueller_profile_enable": (None, [i32]),
        "mueller_profile_reset": (None, []),
        "mueller_launch_count": (i64, []),
        "mueller_profile_get": (i32, [C.c_char_p, dp, C.POINTER(i64)]),
        "mueller_profile_names": (i32, [C.c_char_p, C.c_size_t]),
        "mueller_far_field_noalloc": (C.c_int, [vp, C.POINTER(CParams), vp, i32, dp, dp, i64, vp,
                                                dp, i32, i32, vp]),
        "mueller_matvec_mrhs": (C.c_int, [C.POINTER(COperator), vp, vp, i32, vp, C.c_size_t, vp]),
        "mueller_matvec_mrhs_workspace_bytes": (C.c_size_t, [C.POINTER(COperator), i32]),
        "mueller_assemble_batch": (C.c_int, [i32, C.POINTER(vp), C.POINTER(CParams), i32,
                                             C.POINTER(vp), C.POINTER(i64), C.POINTER(vp),
                                             C.POINTER(vp), C.POINTER(dp), ip, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def quadrature_rule(kind: int, n: int):
    """(a, b, w) of mueller_quadrature_rule: (xi, eta, w) of a triangle rule,
    (x, None, w) of Gauss-Legendre on [0, 1]."""
    lib = load_library()
    a, b, w = np.zeros(n), np.zeros(n), np.zeros(n)
    _check(lib.mueller_quadrature_rule(int(kind), int(n), _dp(a),
                                       _dp(b) if kind == RULE_TRIANGLE else None, _dp(w)))
    return a, (b if kind == RULE_TRIANGLE else None), w


def _check(status: int):
    if status != 0:
        msg = _lib.mueller_last_error().decode(errors="replace")
        raise MuellerError(status, msg)


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA GPU is required (the library has no CPU path)")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _dev(t, dtype, name):
    """A CUDA tensor of the given dtype, row-major contiguous (the C ABI takes
    plain pointers and assumes dense rows)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device.type != "cuda":
        t = t.cuda()
    return t.contiguous()


@dataclass
class Params:
    ka: float
    eps_r: tuple = (1.0, 0.0)
    mu_r: tuple = (1.0, 0.0)
    q_regular: int = 6
    ssq_order: int = 5
    frame_rule: int = FRAME_PAPER

    def c(self) -> CParams:
        p = CParams()
        p.ka = float(self.ka)
        p.eps_r[0], p.eps_r[1] = float(self.eps_r[0]), float(self.eps_r[1])
        p.mu_r[0], p.mu_r[1] = float(self.mu_r[0]), float(self.mu_r[1])
        p.q_regular = int(self.q_regular)
        p.ssq_order = int(self.ssq_order)
        p.frame_rule = int(self.frame_rule)
        p.reserved = 0
        return p

    @classmethod
    def from_workload(cls, w: dict, frame_rule: int = FRAME_PAPER):
        return cls(ka=w["ka"], eps_r=tuple(w["eps_r"]), mu_r=tuple(w["mu_r"]),
                   q_regular=w["q_regular"], ssq_order=w["ssq_order"], frame_rule=frame_rule)


class Mesh:
    """mueller_mesh_load + mueller_tangent_frame."""

    def __init__(self, xyz, tri6, morton: bool = True, stream=None, host_only: bool = False):
        lib = load_library()
        if not host_only:
            _torch()
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tri6 = np.ascontiguousarray(tri6, dtype=np.int32)
        h = C.c_void_p()
        flags = (0 if morton else MESH_KEEP_ORDER) | (MESH_HOST_ONLY if host_only else 0)
        st = lib.mueller_mesh_load(_dp(self.xyz), self.xyz.shape[0],
                                   self.tri6.ctypes.data_as(C.POINTER(C.c_int32)),
                                   self.tri6.shape[0], flags, None if host_only else _stream(stream),
                                   C.byref(h))
        _check(st)
        self.h = h
        self._lib = lib
        self.frame_rule = None
        # sizes from the arrays: mueller_mesh_get_info would wait for the
        # touching pairs and the near layout, which the library builds on a
        # host thread while the frame and the regular pairs are launched
        self.nn, self.nt = self.xyz.shape[0], self.tri6.shape[0]
        self.N = 4 * self.nn

    def info(self) -> dict:
        i = CMeshInfo()
        _check(self._lib.mueller_mesh_get_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in CMeshInfo._fields_}

    def perm(self):
        npm = np.zeros(self.xyz.shape[0], np.int32)
        epm = np.zeros(self.tri6.shape[0], np.int32)
        _check(self._lib.mueller_mesh_perm(self.h, npm.ctypes.data_as(C.POINTER(C.c_int32)),
                                           epm.ctypes.data_as(C.POINTER(C.c_int32))))
        return npm, epm

    def touching(self) -> dict:
        """The touching element pairs (mueller_mesh_touching): ex, ey, cls,
        relabel, one entry per pair, element ids in the mesh's order."""
        n = int(self.info()["n_touching"])
        out = {k: np.zeros(n, np.int32) for k in ("ex", "ey", "cls", "relabel")}
        _check(self._lib.mueller_mesh_touching(self.h, *(_ip(out[k]) for k in
                                                          ("ex", "ey", "cls", "relabel"))))
        return out

    def near_layout(self):
        """(rowptr, col, slot) of the near-block layout (mueller_mesh_near_layout)."""
        i = self.info()
        rowptr = np.zeros(int(i["n_nodes"]) + 1, np.int32)
        col = np.zeros(int(i["n_near_blocks"]), np.int32)
        slot = np.zeros(36 * int(i["n_touching"]), np.int32)
        _check(self._lib.mueller_mesh_near_layout(self.h, _ip(rowptr), _ip(col), _ip(slot)))
        return rowptr, col, slot.reshape(-1, 6, 6)

    def tangent_frame(self, frame_rule: int = FRAME_PAPER, stream=None, out=True):
        torch = _torch()
        fr = torch.empty((self.nn, 9), dtype=torch.float64, device="cuda") if out else None
        _check(self._lib.mueller_tangent_frame(self.h, int(frame_rule), _ptr(fr), _stream(stream)))
        self.frame_rule = int(frame_rule)
        return fr

    def point_records(self, q_regular: int = 6):
        """mueller_point_records: (n_tri, q_regular, 19) records x, n, t1, t2,
        s1, s2, weight * Jacobian of the regular rule, element order of the mesh."""
        out = np.zeros((self.nt, int(q_regular), 19))
        _check(self._lib.mueller_point_records(self.h, int(q_regular), _dp(out)))
        return out

    def near_bytes(self) -> int:
        return int(self._lib.mueller_near_bytes(self.h))

    def free(self):
        if getattr(self, "h", None):
            self._lib.mueller_mesh_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def assemble(mesh: Mesh, params: Params, dtype: int = MUELLER_C128, inc=None, Z=None, near=None,
             B=None, stream=None):
    """mueller_assemble.  Returns (Z, near, B) as CUDA tensors."""
    torch = _torch()
    N = mesh.N
    if Z is None:
        Z = torch.empty((N, N), dtype=torch.complex128 if dtype == MUELLER_C128 else torch.complex64,
                        device="cuda")
    if dtype == MUELLER_C64_NEAR64 and near is None:
        near = torch.empty(mesh.near_bytes() // 16, dtype=torch.complex128, device="cuda")
    r = 0
    incp = None
    if inc is not None:
        inc = np.ascontiguousarray(inc, dtype=np.float64).reshape(-1, 6)
        r = inc.shape[0]
        if B is None:
            B = torch.empty((r, N), dtype=torch.complex128, device="cuda")
        incp = _dp(inc)
    p = params.c()
    _check(mesh._lib.mueller_assemble(mesh.h, C.byref(p), int(dtype), _ptr(Z), Z.stride(0), _ptr(near),
                                      _ptr(B), incp, r, _stream(stream)))
    Z._mueller_k1_mirrored = Z._version  # Z11 = -Z00 as written; see Operator
    return Z, near, B


def dz_matvec(mesh: Mesh, params: Params, which: int, X, stream=None):
    """mueller_dz_matvec: (dZ/d eps_r) X for which = 1, (dZ/d mu_r) X for 2
    (complex derivatives; X, result complex128 of length N)."""
    torch = _torch()
    X = _dev(X, torch.complex128, "X")
    Y = torch.empty_like(X)
    p = params.c()
    _check(mesh._lib.mueller_dz_matvec(mesh.h, C.byref(p), int(which), _ptr(X), _ptr(Y),
                                       _stream(stream)))
    return Y


def zshape_vjp(mesh: Mesh, params: Params, lam, X, stream=None):
    """mueller_zshape_vjp: gradient of Re lam^H Z(X) x with respect to the
    node coordinates, numpy (n_nodes, 3) in the input node order."""
    torch = _torch()
    lam = _dev(lam, torch.complex128, "lam").reshape(-1)
    X = _dev(X, torch.complex128, "X").reshape(-1)
    if lam.numel() != mesh.N or X.numel() != mesh.N:
        raise ValueError("lam and X must have length N")
    g = np.zeros((mesh.nn, 3))
    p = params.c()
    _check(mesh._lib.mueller_zshape_vjp(mesh.h, C.byref(p), _ptr(lam), _ptr(X), _dp(g),
                                        _stream(stream)))
    return g


def zshape_vjp_multi(mesh: Mesh, params: Params, lam, X, stream=None):
    """mueller_zshape_vjp_multi: the gradients of Re lam_o^H Z(X) x for the
    rows lam_o of lam (r, N), numpy (r, n_nodes, 3) in the input node order."""
    torch = _torch()
    lam = _dev(lam, torch.complex128, "lam")
    if lam.dim() == 1:
        lam = lam.reshape(1, -1)
    X = _dev(X, torch.complex128, "X").reshape(-1)
    r = lam.shape[0]
    if lam.shape[1] != mesh.N or X.numel() != mesh.N:
        raise ValueError("lam must be (r, N) and X of length N")
    g = np.zeros((r, mesh.nn, 3))
    p = params.c()
    _check(mesh._lib.mueller_zshape_vjp_multi(mesh.h, C.byref(p), _ptr(lam), int(r), _ptr(X),
                                              _dp(g), _stream(stream)))
    return g


def rhs_shape_vjp(mesh: Mesh, params: Params, lam, inc, stream=None):
    """mueller_rhs_shape_vjp: gradient of Re lam^H b(X) with respect to the
    node coordinates for one incident wave inc (6,), numpy (n_nodes, 3)."""
    torch = _torch()
    lam = _dev(lam, torch.complex128, "lam").reshape(-1)
    if lam.numel() != mesh.N:
        raise ValueError("lam must have length N")
    inc = np.ascontiguousarray(inc, dtype=np.float64).reshape(6)
    g = np.zeros((mesh.nn, 3))
    p = params.c()
    _check(mesh._lib.mueller_rhs_shape_vjp(mesh.h, C.byref(p), _ptr(lam), _dp(inc), _dp(g),
                                           _stream(stream)))
    return g


def cross_section_partials(mesh: Mesh, params: Params, X, inc, n_theta: int = 48,
                           n_phi: int = 96, stream=None):
    """mueller_cross_section_partials for one solution X and incident wave inc.
    Returns (G complex128 (3, N) CUDA tensor, the adjoint right-hand sides of
    C_ext, C_sca, C_abs; grad numpy (3, n_nodes, 3), dC/dX at fixed X;
    xs numpy (3,))."""
    torch = _torch()
    X = _dev(X, torch.complex128, "X").reshape(-1)
    if X.numel() != mesh.N:
        raise ValueError("X must have length N")
    inc = np.ascontiguousarray(inc, dtype=np.float64).reshape(6)
    G = torch.empty((3, mesh.N), dtype=torch.complex128, device=X.device)
    g = np.zeros((3, mesh.nn, 3))
    xs = np.zeros(3)
    p = params.c()
    _check(mesh._lib.mueller_cross_section_partials(mesh.h, C.byref(p), _ptr(X), _dp(inc),
                                                    int(n_theta), int(n_phi), _ptr(G), _dp(g),
                                                    _dp(xs), _stream(stream)))
    return G, g, xs


def assemble_batch(meshes, params, dtype: int = MUELLER_C64_NEAR64, incs=None, stream=None):
    """mueller_assemble_batch: one launch of each assembly kernel for all bodies.
    Returns a list of (Z, near, B) per body as CUDA tensors."""
    torch = _torch()
    lib = load_library()
    nb = len(meshes)
    if len(params) != nb or (incs is not None and len(incs) != nb):
        raise ValueError("one params (and inc) entry per mesh")
    out, keep = [], []
    for b, m in enumerate(meshes):
        N = m.N
        Z = torch.empty((N, N), dtype=torch.complex128 if dtype == MUELLER_C128 else torch.complex64,
                        device="cuda")
        near = (torch.empty(m.near_bytes() // 16, dtype=torch.complex128, device="cuda")
                if dtype == MUELLER_C64_NEAR64 else None)
        B = None
        if incs is not None:
            inc = np.ascontiguousarray(incs[b], dtype=np.float64).reshape(-1, 6)
            keep.append(inc)
            B = torch.empty((inc.shape[0], N), dtype=torch.complex128, device="cuda")
        out.append((Z, near, B))
    vp = C.c_void_p
    h = (vp * nb)(*[m.h for m in meshes])
    cps = (CParams * nb)(*[p.c() for p in params])
    zs = (vp * nb)(*[o[0].data_ptr() for o in out])
    lds = (C.c_int64 * nb)(*[o[0].stride(0) for o in out])
    ns = (vp * nb)(*[(o[1].data_ptr() if o[1] is not None else None) for o in out])
    bs = incp = rs = None
    if incs is not None:
        bs = (vp * nb)(*[o[2].data_ptr() for o in out])
        incp = (C.POINTER(C.c_double) * nb)(*[_dp(a) for a in keep])
        rs = (C.c_int32 * nb)(*[a.shape[0] for a in keep])
    _check(lib.mueller_assemble_batch(nb, h, cps, int(dtype), zs, lds, ns, bs, incp, rs,
                                      _stream(stream)))
    for o in out:
        o[0]._mueller_k1_mirrored = o[0]._version
    return out


class Operator:
    """The operator struct handed to precond_build / solve / matvec.

    mirrored: Z11 = -Z00 bit for bit (MUELLER_OP_K1_MIRRORED), so that
    products read three quarters of Z.  By default true exactly while Z was
    last written by assemble / assemble_batch (returned or passed in as the
    output) and not changed in place since: the tag holds the tensor's
    version counter and is read at every call.  A copy, a slice or any other
    tensor is not tagged.  A Z written behind PyTorch's back
    (through its raw pointer) keeps its tag: pass False then."""

    def __init__(self, mesh: Mesh, Z, near=None, dtype: int = MUELLER_C128, precond=None, block=0,
                 mirrored=None, adjoint: bool = False):
        self.mesh, self.Z, self.near, self.dtype = mesh, Z, near, dtype
        self.precond, self.block = precond, block
        self._mirrored = mirrored
        self.adjoint = bool(adjoint)  # MUELLER_OP_ADJOINT: Z^H, (P^{-1})^H

    @property
    def mirrored(self) -> bool:
        # evaluated at each call, so an Operator made before its Z is
        # (re)assembled sees the tag
        if self._mirrored is not None:
            return bool(self._mirrored)
        tag = getattr(self.Z, "_mueller_k1_mirrored", None)
        return tag is not None and tag == self.Z._version

    def c(self) -> COperator:
        o = COperator()
        o.mesh = self.mesh.h
        o.Z_dev = self.Z.data_ptr()
        o.ldz = self.Z.stride(0)
        o.dtype = int(self.dtype)
        o.flags = (MUELLER_OP_K1_MIRRORED if self.mirrored else 0) | \
            (MUELLER_OP_ADJOINT if self.adjoint else 0)
        o.near_dev = self.near.data_ptr() if self.near is not None else None
        o.precond_dev = self.precond.data_ptr() if self.precond is not None else None
        o.block = int(self.block)
        return o


def precond_build(op: Operator, block: int, stream=None):
    torch = _torch()
    lib = load_library()
    nbytes = lib.mueller_precond_bytes(op.mesh.N, int(block))
    P = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    o = op.c()
    _check(lib.mueller_precond_build(C.byref(o), int(block), _ptr(P), _stream(stream)))
    op.precond, op.block = P, int(block)
    return P


def precond_build_batch(ops, blocks, stream=None):
    """mueller_precond_build_batch: the block-Jacobi preconditioners of many
    operators (bodies) by one batched LU.  Sets and returns each operator's
    buffer."""
    torch = _torch()
    lib = load_library()
    n = len(ops)
    if len(blocks) != n:
        raise ValueError("one block size per operator")
    bufs = [torch.empty(lib.mueller_precond_bytes(op.mesh.N, int(b)), dtype=torch.uint8,
                        device="cuda") for op, b in zip(ops, blocks)]
    cops = (COperator * n)(*[op.c() for op in ops])
    cblk = (C.c_int64 * n)(*[int(b) for b in blocks])
    cptr = (C.c_void_p * n)(*[b.data_ptr() for b in bufs])
    _check(lib.mueller_precond_build_batch(n, cops, cblk, cptr, _stream(stream)))
    for op, P, b in zip(ops, bufs, blocks):
        op.precond, op.block = P, int(b)
    return bufs


@dataclass
class SolverOpts:
    mode: int = SOLVE_GMRES
    restart: int = 50
    maxit: int = 5000
    warm_start: int = 0
    tol: float = 1e-8
    inner_tol: float = 1e-5
    max_refine: int = 20
    use_precond: int = 1

    def c(self) -> CSolverOpts:
        o = CSolverOpts()
        for k in ("mode", "restart", "maxit", "warm_start", "max_refine", "use_precond"):
            setattr(o, k, int(getattr(self, k)))
        o.tol = float(self.tol)
        o.inner_tol = float(self.inner_tol)
        return o


def solve(op: Operator, B, opts: SolverOpts, X=None, work=None, stream=None, raise_on_nc=True):
    """mueller_solve.  Returns (X, info dict)."""
    torch = _torch()
    lib = load_library()
    B = _dev(B, torch.complex128, "B")
    r = B.shape[0] if B.dim() == 2 else 1
    if X is None:
        X = torch.zeros_like(B)
    elif not (X.is_cuda and X.dtype == torch.complex128 and X.is_contiguous()):
        raise TypeError("X must be a contiguous complex128 CUDA tensor")
    o = op.c()
    so = opts.c()
    info = CSolveInfo()
    wb = 0
    if work is not None:
        wb = work.numel() * work.element_size()
    st = lib.mueller_solve(C.byref(o), _ptr(B), _ptr(X), int(r), C.byref(so), C.byref(info),
                           _ptr(work), wb, _stream(stream))
    d = {k: getattr(info, k) for k, _ in CSolveInfo._fields_}
    if st == 5 and not raise_on_nc:
        return X, d
    _check(st)
    return X, d


def solve_workspace_bytes(op: Operator, r: int, opts: SolverOpts) -> int:
    o = op.c()
    so = opts.c()
    return int(load_library().mueller_solve_workspace_bytes(C.byref(o), int(r), C.byref(so)))


def matvec(op: Operator, X, Y=None, stream=None):
    torch = _torch()
    lib = load_library()
    X = _dev(X, torch.complex128, "X")
    r = X.shape[0] if X.dim() == 2 else 1
    if Y is None:
        Y = torch.empty_like(X)
    o = op.c()
    _check(lib.mueller_matvec(C.byref(o), _ptr(X), _ptr(Y), int(r), None, 0, _stream(stream)))
    return Y


def matvec_mrhs(op: Operator, X, Y=None, work=None, stream=None):
    """mueller_matvec_mrhs: complex64 r x N product on the tensor cores."""
    torch = _torch()
    lib = load_library()
    X = _dev(X, torch.complex64, "X")
    r = X.shape[0] if X.dim() == 2 else 1
    if Y is None:
        Y = torch.empty_like(X)
    o = op.c()
    need = lib.mueller_matvec_mrhs_workspace_bytes(C.byref(o), int(r))
    if work is None or work.numel() * work.element_size() < need:
        work = torch.empty(need, dtype=torch.uint8, device=X.device)
    _check(lib.mueller_matvec_mrhs(C.byref(o), _ptr(X), _ptr(Y), int(r), _ptr(work),
                                   work.numel() * work.element_size(), _stream(stream)))
    return Y


def far_field(mesh: Mesh, params: Params, X, inc, dirs=None, n_theta: int = 48, n_phi: int = 96,
              stream=None):
    """mueller_far_field.  Returns (F tensor r x n_dir x 3 or None, xs numpy r x 3)."""
    torch = _torch()
    X = _dev(X, torch.complex128, "X")
    inc = np.ascontiguousarray(inc, dtype=np.float64).reshape(-1, 6)
    r = inc.shape[0]
    if X.numel() != r * mesh.N:
        raise ValueError("X must hold one solution of length N per incident wave")
    if dirs is None:
        dirs = np.zeros((0, 3))
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    nd = dirs.shape[0]
    F = torch.empty((r, nd, 3), dtype=torch.complex128, device="cuda") if nd else None
    xs = np.zeros((r, 3))
    p = params.c()
    _check(mesh._lib.mueller_far_field(mesh.h, C.byref(p), _ptr(X), r, _dp(inc),
                                       _dp(dirs) if nd else None, nd, _ptr(F), _dp(xs),
                                       int(n_theta), int(n_phi), _stream(stream)))
    return F, xs


def sync(stream=None):
    _check(load_library().mueller_sync(_stream(stream)))


def profile_enable(on: bool = True):
    """Per-kernel CUDA-event timing on the launching stream (serialising)."""
    load_library().mueller_profile_enable(1 if on else 0)


def profile_reset():
    load_library().mueller_profile_reset()


def launch_count() -> int:
    """Kernel launches made by the library since load (or the last reset)."""
    return int(load_library().mueller_launch_count())


def profile_report() -> dict:
    """{kernel name: (total ms, launches)} of the timed launches."""
    lib = load_library()
    buf = C.create_string_buffer(1 << 16)
    lib.mueller_profile_names(buf, len(buf))
    out = {}
    for name in buf.value.decode().split("\n"):
        if not name:
            continue
        ms = C.c_double()
        n = C.c_int64()
        lib.mueller_profile_get(name.encode(), C.byref(ms), C.byref(n))
        out[name] = (ms.value, n.value)
    return out
