"""Oracle: automatic selection of the collision region from the rest geometry.

Test infrastructure only (see the package docstring).

The paper takes the collision-aware region x2 and its proxy surface from the
user (Sec. 3.1, Fig. 2a) and names their automatic selection as future work
(Sec. 5).  The rule restated here (the same one the library's
fsim_select_region implements, in code of its own):

* boundary triangles: faces of the tets that belong to exactly one tet;
* surface graph: the edges of the boundary triangles;
* a boundary vertex v can take part in contact when some other boundary
  vertex u is closer than `radius` at rest, ((dx dx + dy dy) + dz dz) <
  radius^2 in float64, while u is more than `rings` surface edges from v;
* the proxy is every boundary triangle whose three vertices can take part in
  contact and are not all pinned; its vertices (W = selection) give x2.

Written plainly: a k-d tree proposes the close pairs (with a slightly larger
radius), the strict float64 test decides them, and "within `rings` edges" is
the sparsity pattern of (A + I)^rings for the surface adjacency A.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree


def boundary_triangles(tets: np.ndarray) -> np.ndarray:
    """Sorted vertex triples of the faces that belong to exactly one tet,
    in lexicographic order."""
    tets = np.asarray(tets, dtype=np.int64)
    f = np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]], tets[:, [0, 2, 3]],
                        tets[:, [1, 2, 3]]], axis=0)
    key = np.sort(f, axis=1)
    uniq, cnt = np.unique(key, axis=0, return_counts=True)
    return uniq[cnt == 1]


def select_region(rest, tets, pinned, radius: float, rings: int):
    """(proxy triangles in proxy-vertex numbering, proxy vertex ids)."""
    rest = np.asarray(rest, dtype=np.float64)
    n = rest.shape[0]
    bf = boundary_triangles(tets)
    e = np.concatenate([bf[:, [0, 1]], bf[:, [1, 2]], bf[:, [0, 2]]], axis=0)
    A = sp.coo_matrix((np.ones(2 * len(e)), (np.concatenate([e[:, 0], e[:, 1]]),
                                              np.concatenate([e[:, 1], e[:, 0]]))),
                      shape=(n, n)).tocsr()
    A.data[:] = 1.0
    reach = sp.identity(n, format="csr")
    step = (A + sp.identity(n, format="csr")).tocsr()
    step.data[:] = 1.0
    for _ in range(rings):
        reach = (reach @ step).tocsr()
        reach.data[:] = 1.0
    onb = np.unique(bf.ravel())
    tree = cKDTree(rest[onb])
    pairs = tree.query_pairs(radius * (1.0 + 1e-9), output_type="ndarray")
    capable = np.zeros(n, dtype=bool)
    if len(pairs):
        u, v = onb[pairs[:, 0]], onb[pairs[:, 1]]
        d = rest[u] - rest[v]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        near = np.asarray(reach[u, v]).ravel() > 0
        keep = (d2 < radius * radius) & ~near
        capable[u[keep]] = True
        capable[v[keep]] = True
    pinned = np.asarray(pinned).astype(bool)
    ok = capable[bf].all(axis=1) & ~pinned[bf].all(axis=1)
    faces = bf[ok]
    verts = np.unique(faces.ravel())
    local = -np.ones(n, dtype=np.int64)
    local[verts] = np.arange(len(verts))
    return local[faces].astype(np.int32), verts.astype(np.int32)
