"""Curved P2 surface meshes: subdivided icosahedra projected onto a sphere,
optionally stretched into a spheroid.

Layout of a mesh (the input format of ``mueller_mesh_load`` and of the oracle):

* ``xyz``  float64 ``[n_nodes, 3]``: corner vertices first, then one node per
  edge.  Every node lies on the exact surface (edge nodes are the projected
  midpoints of the straight chord).
* ``tri6`` int32 ``[n_tri, 6]``: ``(v0, v1, v2, m01, m12, m20)`` -- three
  corners in counter-clockwise order seen from outside, then the edge nodes of
  the edges v0v1, v1v2, v2v0.  The parametric map of a triangle therefore has
  its normal ``d_xi x  d_eta x`` pointing outwards.

A level-L icosphere has F = 20*4^L triangles, V = 10*4^L + 2 corners and
E = 30*4^L edges, so n_nodes = V + E.
"""

from __future__ import annotations

import numpy as np

_T = (1.0 + 5.0 ** 0.5) / 2.0

_ICO_V = np.array(
    [
        [-1, _T, 0], [1, _T, 0], [-1, -_T, 0], [1, -_T, 0],
        [0, -1, _T], [0, 1, _T], [0, -1, -_T], [0, 1, -_T],
        [_T, 0, -1], [_T, 0, 1], [-_T, 0, -1], [-_T, 0, 1],
    ],
    dtype=np.float64,
)

_ICO_F = np.array(
    [
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ],
    dtype=np.int64,
)


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _orient_outward(verts: np.ndarray, faces: np.ndarray) -> np.ndarray:
    a, b, c = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    s = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c)
    faces = faces.copy()
    flip = s < 0
    faces[flip, 1], faces[flip, 2] = faces[flip, 2].copy(), faces[flip, 1].copy()
    return faces


def _edge_table(faces: np.ndarray, n_verts: int):
    """Unique undirected edges of a triangle list and, per face, the edge ids of
    (v0v1, v1v2, v2v0)."""
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]], axis=0)
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    key = lo * n_verts + hi
    uniq, inv = np.unique(key, return_inverse=True)
    n_f = faces.shape[0]
    face_edges = inv.reshape(3, n_f).T
    edges = np.stack([uniq // n_verts, uniq % n_verts], axis=1)
    return edges, face_edges


def _subdivide(verts: np.ndarray, faces: np.ndarray):
    edges, fe = _edge_table(faces, verts.shape[0])
    mids = _unit(0.5 * (verts[edges[:, 0]] + verts[edges[:, 1]]))
    nv = verts.shape[0]
    verts = np.concatenate([verts, mids], axis=0)
    a, b, c = faces[:, 0], faces[:, 1], faces[:, 2]
    ab, bc, ca = nv + fe[:, 0], nv + fe[:, 1], nv + fe[:, 2]
    new = np.concatenate(
        [
            np.stack([a, ab, ca], 1),
            np.stack([ab, b, bc], 1),
            np.stack([ca, bc, c], 1),
            np.stack([ab, bc, ca], 1),
        ],
        axis=0,
    )
    return verts, new


def mesh_counts(level: int) -> dict:
    """Closed-form sizes of a level-``level`` icosphere P2 mesh."""
    f = 20 * 4 ** level
    v = 10 * 4 ** level + 2
    e = 30 * 4 ** level
    return {"n_tri": f, "n_vertices": v, "n_edges": e, "n_nodes": v + e, "n_dof": 4 * (v + e)}


def icosphere_p2(level: int, radius: float = 1.0):
    """Level-``level`` icosphere of the given radius with curved P2 triangles.

    Returns ``(xyz float64 [n_nodes,3], tri6 int32 [n_tri,6])``.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    verts = _unit(_ICO_V)
    faces = _orient_outward(verts, _ICO_F)
    for _ in range(level):
        verts, faces = _subdivide(verts, faces)
    faces = _orient_outward(verts, faces)
    edges, fe = _edge_table(faces, verts.shape[0])
    mids = _unit(0.5 * (verts[edges[:, 0]] + verts[edges[:, 1]]))
    nv = verts.shape[0]
    xyz = np.concatenate([verts, mids], axis=0) * radius
    tri6 = np.concatenate([faces, nv + fe], axis=1).astype(np.int32)
    return np.ascontiguousarray(xyz, dtype=np.float64), np.ascontiguousarray(tri6)


def spheroid_p2(level: int, a: float = 1.0, c: float = 1.5):
    """Spheroid with semi-axes (a, a, c): the unit icosphere stretched axially.
    Every node of the sphere mesh maps onto the spheroid surface."""
    xyz, tri6 = icosphere_p2(level, 1.0)
    xyz = xyz * np.array([a, a, c], dtype=np.float64)
    return np.ascontiguousarray(xyz), tri6
