"""ORACLE -- test infrastructure only.

A plain FP64 CPU implementation of the nodal P2 Mueller method (arXiv
2604.21181), written from the paper and sharing no code with the CUDA library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does.

The C++ core (``mueller_oracle.cpp``) is compiled on first use (or by
``build()``) into ``liboracle.so`` next to this file and driven through
ctypes.  ``mie.py`` holds the closed-form Mie series that pins the oracle's
cross sections.

Parity status of each function: see the header of ``mueller_oracle.cpp``;
every function is pinned by a test under ``tests/test_oracle_*.py``.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mueller_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            D = C.c_double
            I = C.c_int
            I64 = C.c_int64
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            sig = {
                "oracle_tri_rule": (I, [I, dp, dp, dp]),
                "oracle_gauss_legendre01": (None, [I, dp, dp]),
                "oracle_morton": (None, [dp, I64, ip, I64, ip, ip]),
                "oracle_mesh_new": (P, [dp, I64, ip, I64, C.c_int32]),
                "oracle_mesh_free": (None, [P]),
                "oracle_mesh_perm": (None, [P, ip, ip]),
                "oracle_frame": (None, [P, dp]),
                "oracle_point_geo": (D, [P, I64, D, D, dp]),
                "oracle_kernel_scalars": (None, [D, D, D, D, D, D, I, dp]),
                "oracle_qfuncs": (None, [D, D, dp]),
                "oracle_hdiff": (None, [D, D, D, D, D, D, dp]),
                "oracle_ss_points": (I64, [I, I, dp]),
                "oracle_classify": (I, [P, I64, I64, I, ip, ip]),
                "oracle_ssq_singular": (I, [P, I64, I64, I, I, dp]),
                "oracle_ssq_test": (D, [P, I64, I64, I, I, I]),
                "oracle_brute_singular": (I, [P, I64, I64, I, dp]),
                "oracle_pair_block": (I, [P, D, D, D, D, D, I, I, I64, I64, dp]),
                "oracle_ssq_full": (I, [P, D, D, D, D, D, I64, I64, I, dp]),
                "oracle_assemble": (None, [P, D, D, D, D, D, I, I, I, dp, ip, I64]),
                "oracle_rhs": (None, [P, D, D, D, D, D, I, dp, I, dp]),
                "oracle_mass": (None, [P, I, dp]),
                "oracle_lu_solve": (I, [I64, dp, dp, I, dp]),
                "oracle_gmres": (I, [I64, dp, dp, dp, I64, I, D, I, dp]),
                "oracle_mbj_apply": (I, [I64, dp, I64, dp, dp]),
                "oracle_far_field": (None, [P, D, I, dp, I, dp, dp, I64, dp, dp, I, I]),
                "oracle_num_threads": (I, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def tri_rule(q: int):
    xi = np.zeros(16)
    eta = np.zeros(16)
    w = np.zeros(16)
    n = _load().oracle_tri_rule(q, _d(xi), _d(eta), _d(w))
    if n < 0:
        raise ValueError(f"no {q}-point rule")
    return xi[:n].copy(), eta[:n].copy(), w[:n].copy()


def gauss_legendre01(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _load().oracle_gauss_legendre01(n, _d(x), _d(w))
    return x, w


def morton(xyz, tri6):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri6 = np.ascontiguousarray(tri6, dtype=np.int32)
    npm = np.zeros(xyz.shape[0], np.int32)
    epm = np.zeros(tri6.shape[0], np.int32)
    _load().oracle_morton(_d(xyz), xyz.shape[0], _i(tri6), tri6.shape[0], _i(npm), _i(epm))
    return npm, epm


def qfuncs(z: complex):
    o = np.zeros(6)
    _load().oracle_qfuncs(float(np.real(z)), float(np.imag(z)), _d(o))
    return complex(o[0], o[1]), complex(o[2], o[3]), complex(o[4], o[5])


def kernel_scalars(ka, eps_r, mu_r, R, remainder=False):
    o = np.zeros(8)
    eps_r = complex(*eps_r) if isinstance(eps_r, (tuple, list)) else complex(eps_r)
    mu_r = complex(*mu_r) if isinstance(mu_r, (tuple, list)) else complex(mu_r)
    _load().oracle_kernel_scalars(ka, eps_r.real, eps_r.imag, mu_r.real, mu_r.imag, R,
                                  int(remainder), _d(o))
    return o[0::2] + 1j * o[1::2]


def hdiff(ka, eps_r, mu_r, R):
    """Coefficients (A, B) of H_diff = A R^R^ + B I at distance R."""
    o = np.zeros(4)
    eps_r = complex(*eps_r) if isinstance(eps_r, (tuple, list)) else complex(eps_r)
    mu_r = complex(*mu_r) if isinstance(mu_r, (tuple, list)) else complex(mu_r)
    _load().oracle_hdiff(ka, eps_r.real, eps_r.imag, mu_r.real, mu_r.imag, R, _d(o))
    return complex(o[0], o[1]), complex(o[2], o[3])


def ss_points(cls: int, ns: int):
    lib = _load()
    n = lib.oracle_ss_points(cls, ns, None)
    out = np.zeros((n, 5))
    lib.oracle_ss_points(cls, ns, _d(out))
    return out


class Mesh:
    """Oracle mesh: Morton-permuted P2 mesh with its nodal frame."""

    def __init__(self, xyz, tri6, morton: bool = True, frame_rule: int = 0):
        self._lib = _load()
        self.xyz_in = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tri6_in = np.ascontiguousarray(tri6, dtype=np.int32)
        self.nn = self.xyz_in.shape[0]
        self.nt = self.tri6_in.shape[0]
        self.N = 4 * self.nn
        self.h = self._lib.oracle_mesh_new(_d(self.xyz_in), self.nn, _i(self.tri6_in), self.nt,
                                           (0 if morton else 1) | (int(frame_rule) << 1))
        self.node_perm = np.zeros(self.nn, np.int32)
        self.elem_perm = np.zeros(self.nt, np.int32)
        self._lib.oracle_mesh_perm(self.h, _i(self.node_perm), _i(self.elem_perm))
        inv = np.empty_like(self.node_perm)
        inv[self.node_perm] = np.arange(self.nn, dtype=np.int32)
        self.xyz = self.xyz_in[self.node_perm]
        self.tri6 = inv[self.tri6_in[self.elem_perm]]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.oracle_mesh_free(h)
            self.h = None

    def frame(self):
        out = np.zeros((self.nn, 9))
        self._lib.oracle_frame(self.h, _d(out))
        return out

    def point_geo(self, e, xi, eta):
        out = np.zeros(22)
        self._lib.oracle_point_geo(self.h, e, xi, eta, _d(out))
        return dict(x=out[0:3], n=out[3:6], t1=out[6:9], t2=out[9:12], s1=out[12:15],
                    s2=out[15:18], J=out[18], gs_min=out[19])

    def classify(self, ex, ey, alt=False):
        px = np.zeros(3, np.int32)
        py = np.zeros(3, np.int32)
        c = self._lib.oracle_classify(self.h, ex, ey, int(alt), _i(px), _i(py))
        return c, px, py

    def ssq_singular(self, ex, ey, ns, alt=False):
        out = np.zeros((6, 6, 8))
        c = self._lib.oracle_ssq_singular(self.h, ex, ey, ns, int(alt), _d(out))
        return c, out

    def brute_singular(self, ex, ey, n):
        """G1, G2 of a touching pair by the brute-force route (relative polar
        coordinates over the unfolded pair, no Sauter-Schwab map): (class,
        array 6 x 6 x 8) like ssq_singular."""
        out = np.zeros((6, 6, 8))
        c = self._lib.oracle_brute_singular(self.h, ex, ey, n, _d(out))
        return c, out

    def ssq_test(self, ex, ey, ns, which, alt=False):
        return self._lib.oracle_ssq_test(self.h, ex, ey, ns, int(alt), which)

    def pair_block(self, p, ex, ey):
        out = np.zeros((6, 6, 12, 2))
        c = self._lib.oracle_pair_block(self.h, p["ka"], p["eps_r"][0], p["eps_r"][1],
                                        p["mu_r"][0], p["mu_r"][1], p["q_regular"],
                                        p["ssq_order"], ex, ey, _d(out))
        return c, out[..., 0] + 1j * out[..., 1]

    def ssq_full(self, p, ex, ey, ns):
        out = np.zeros((6, 6, 12, 2))
        c = self._lib.oracle_ssq_full(self.h, p["ka"], p["eps_r"][0], p["eps_r"][1],
                                      p["mu_r"][0], p["mu_r"][1], ex, ey, ns, _d(out))
        return c, out[..., 0] + 1j * out[..., 1]

    def assemble(self, p, alt=False, rows=None):
        """Dense Z (N x N complex128).  If ``rows`` (test node ids) is given,
        returns only their 4*len(rows) rows ordered (node, h, alpha)."""
        if rows is None:
            Z = np.zeros((self.N, self.N), np.complex128)
            sel = None
            nsel = 0
        else:
            rows = np.asarray(rows, dtype=np.int64)
            sel = np.full(self.nn, -1, np.int32)
            sel[rows] = np.arange(len(rows), dtype=np.int32)
            Z = np.zeros((4 * len(rows), self.N), np.complex128)
            nsel = len(rows)
        Zr = Z.view(np.float64)
        self._lib.oracle_assemble(self.h, p["ka"], p["eps_r"][0], p["eps_r"][1], p["mu_r"][0],
                                  p["mu_r"][1], p["q_regular"], p["ssq_order"], int(alt),
                                  _d(Zr), None if sel is None else _i(sel), nsel)
        return Z

    def rhs(self, p, inc):
        inc = np.ascontiguousarray(inc, dtype=np.float64).reshape(-1, 6)
        r = inc.shape[0]
        B = np.zeros((r, self.N), np.complex128)
        self._lib.oracle_rhs(self.h, p["ka"], p["eps_r"][0], p["eps_r"][1], p["mu_r"][0],
                             p["mu_r"][1], p["q_regular"], _d(inc), r, _d(B.view(np.float64)))
        return B

    def mass(self, q_regular=6):
        M = np.zeros((self.nn, self.nn))
        self._lib.oracle_mass(self.h, q_regular, _d(M))
        return M

    def far_field(self, p, X, inc, dirs=None, n_theta=48, n_phi=96):
        X = np.ascontiguousarray(X, dtype=np.complex128).reshape(-1, self.N)
        inc = np.ascontiguousarray(inc, dtype=np.float64).reshape(-1, 6)
        r = X.shape[0]
        if dirs is None:
            dirs = np.zeros((0, 3))
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        F = np.zeros((r, dirs.shape[0], 3), np.complex128)
        xs = np.zeros((r, 3))
        self._lib.oracle_far_field(self.h, p["ka"], p["q_regular"], _d(X.view(np.float64)), r,
                                   _d(inc), _d(dirs) if dirs.size else None, dirs.shape[0],
                                   _d(F.view(np.float64)) if F.size else None, _d(xs),
                                   n_theta, n_phi)
        return F, xs


def lu_solve(Z, B):
    Z = np.array(Z, dtype=np.complex128, order="C", copy=True)
    B = np.ascontiguousarray(B, dtype=np.complex128).reshape(-1, Z.shape[0])
    X = np.zeros_like(B)
    st = _load().oracle_lu_solve(Z.shape[0], _d(Z.view(np.float64)), _d(B.view(np.float64)),
                                 B.shape[0], _d(X.view(np.float64)))
    if st:
        raise np.linalg.LinAlgError(f"zero pivot at step {st}")
    return X


def gmres(Z, b, block=256, restart=50, tol=1e-8, maxit=5000, x0=None):
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    info = np.zeros(4)
    st = _load().oracle_gmres(Z.shape[0], _d(Z.view(np.float64)), _d(b.view(np.float64)),
                              _d(x.view(np.float64)), block, restart, tol, maxit, _d(info))
    if st:
        raise np.linalg.LinAlgError("singular preconditioner block")
    return x, dict(iters=int(info[0]), restarts=int(info[1]), converged=bool(info[2]),
                   relres=float(info[3]))


def mbj_apply(Z, block, v):
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    v = np.ascontiguousarray(v, dtype=np.complex128).ravel()
    out = np.zeros_like(v)
    st = _load().oracle_mbj_apply(Z.shape[0], _d(Z.view(np.float64)), block,
                                  _d(v.view(np.float64)), _d(out.view(np.float64)))
    if st:
        raise np.linalg.LinAlgError("singular preconditioner block")
    return out


def cross_sections(mesh: Mesh, p, inc):
    """C_ext, C_sca, C_abs (one row per incident wave) of the oracle's
    pipeline: assembly (Sec. 4), dense LU solve, far field and cross
    sections (the formulas of the far-field step)."""
    Z = mesh.assemble(p)
    B = mesh.rhs(p, inc)
    X = lu_solve(Z, B)
    return np.asarray(mesh.far_field(p, X, inc)[1])


def cross_section_shape_derivative(xyz, tri6, p, inc, V, h: float = 1e-6, frame_rule: int = 0):
    """Derivative of (C_ext, C_sca, C_abs), one row per incident wave, along
    the node displacement field V (n_nodes x 3): d/dt C(xyz + t V) at t = 0,
    by central differences of cross_sections on the meshes with nodes
    xyz +- h V and the same connectivity (truncation O(h^2)).  The paper
    defines no shape derivative; this is the plain derivative of the
    oracle's own results."""
    xyz = np.asarray(xyz, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    xs = []
    for sgn in (1.0, -1.0):
        m = Mesh(xyz + sgn * h * V, tri6, frame_rule=frame_rule)
        xs.append(cross_sections(m, p, inc))
    return (xs[0] - xs[1]) / (2.0 * h)


def cross_section_coordinate_gradient(xyz, tri6, p, inc, nodes=None, h: float = 1e-6,
                                      frame_rule: int = 0):
    """Gradient of (C_ext, C_sca, C_abs) of the first incident wave with
    respect to the coordinates of the listed nodes (all nodes by default;
    node ids of the caller's xyz): array (len(nodes), 3 coordinates,
    3 cross sections), each entry cross_section_shape_derivative along one
    unit coordinate displacement."""
    xyz = np.asarray(xyz, dtype=np.float64)
    nodes = range(xyz.shape[0]) if nodes is None else nodes
    G = np.zeros((len(nodes), 3, 3))
    for a, k in enumerate(nodes):
        for d in range(3):
            V = np.zeros_like(xyz)
            V[k, d] = 1.0
            G[a, d] = cross_section_shape_derivative(xyz, tri6, p, inc, V, h, frame_rule)[0]
    return G


def cross_section_gradient(mesh: Mesh, p, inc, h: float = 1e-4):
    """Jacobian of (C_ext, C_sca, C_abs) of the first incident wave with
    respect to (Re eps_r, Im eps_r, Re mu_r, Im mu_r), by central differences
    of cross_sections with step h on each real parameter (truncation
    O(h^2)).  The paper defines no gradient; this is the plain derivative of
    the oracle's own results, a 3 x 4 array."""
    J = np.zeros((3, 4))
    for k in range(4):
        key, part = ("eps_r", "mu_r")[k // 2], k % 2
        val = list(p[key])
        xs = []
        for sgn in (1.0, -1.0):
            q = dict(p)
            v = list(val)
            v[part] += sgn * h
            q[key] = tuple(v)
            xs.append(cross_sections(mesh, q, inc)[0])
        J[:, k] = (xs[0] - xs[1]) / (2.0 * h)
    return J
