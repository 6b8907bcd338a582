"""Automatic collision-region selection (the paper's Sec. 5 future work).

The library's fsim_select_region (host code, no GPU needed) against the
oracle's restatement of the same rule (oracle/region.py), bit-exact; the
oracle pinned by brute force on a small mesh and by geometry whose answer is
known: two slabs across a gap select exactly their two facing faces, one
body alone selects nothing, and on the face only the two lips across the
mouth slit are selected.
"""
import collections

import numpy as np
import pytest

from oracle import region as R
from paper_2312_02999_gb300 import inputs as I


def _lib():
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim
    return fsim


@pytest.mark.parametrize("case", ["slabs", "face5k", "face10k"])
def test_native_selection_equals_oracle(case):
    fsim = _lib()
    mesh, radius, rings = {
        "slabs": (I.two_slabs(4, 4, 2, gap=0.004), 0.01, 3),
        "face5k": (I.face_shell(n_target=5000), 0.002, 4),
        "face10k": (I.face_shell(n_target=10000), 0.003, 3),
    }[case]
    to, vo = R.select_region(mesh.rest, mesh.tets, mesh.pinned, radius, rings)
    tg, vg = fsim.select_region(mesh.rest, mesh.tets, mesh.pinned, radius, rings)
    assert len(to) > 0
    assert np.array_equal(to, tg) and np.array_equal(vo, vg)


@pytest.mark.parametrize("nx,nz", [(3, 2), (4, 2), (5, 3)])
def test_two_slabs_select_their_facing_faces(nx, nz):
    # the generator's proxy of two slabs is exactly their two facing faces
    mesh = I.two_slabs(nx, nx, nz, gap=0.004)
    tris, verts = R.select_region(mesh.rest, mesh.tets, mesh.pinned, 0.01, 3)
    assert np.array_equal(verts, np.sort(mesh.W_col))
    want = {tuple(sorted(mesh.W_col[t])) for t in mesh.proxy_tris}
    got = {tuple(sorted(verts[t])) for t in tris}
    assert got == want


def test_one_body_alone_selects_nothing():
    mesh = I.two_slabs(4, 4, 2, gap=0.004)
    bottom = mesh.rest[:, 2] < mesh.rest[:, 2].mean()
    keep = bottom[mesh.tets].all(axis=1)
    tris, verts = R.select_region(mesh.rest, mesh.tets[keep], mesh.pinned, 0.01, 3)
    assert len(tris) == 0 and len(verts) == 0


def test_face_selects_the_two_lips():
    mesh = I.face_shell(n_target=10000)
    tris, verts = R.select_region(mesh.rest, mesh.tets, mesh.pinned, 0.003, 3)
    assert len(verts) > 0
    assert np.isin(verts, mesh.W_col).all()               # inside the mouth region
    g = mesh.grid
    jm = g["jm"]
    # vertices on both sides of the removed row of cells (rows jm and jm + 1)
    rows = g["gj"][verts]
    assert (rows <= jm).any() and (rows >= jm + 1).any()
    assert (mesh.pinned[verts] == 0).all()


def test_oracle_rule_by_brute_force():
    # every pair of boundary vertices and breadth-first surface distances, by hand
    mesh = I.two_slabs(3, 3, 2, gap=0.004)
    rest, tets = mesh.rest, mesh.tets
    radius, rings = 0.0045, 2
    faces = collections.Counter()
    for t in tets:
        for f in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
            faces[tuple(sorted(int(t[i]) for i in f))] += 1
    bf = sorted(k for k, c in faces.items() if c == 1)
    adj = collections.defaultdict(set)
    for a, b, c in bf:
        adj[a] |= {b, c}; adj[b] |= {a, c}; adj[c] |= {a, b}
    onb = sorted(adj)

    def within(v):
        seen, front = {v}, [v]
        for _ in range(rings):
            front = [w for u in front for w in adj[u] if w not in seen]
            seen |= set(front)
        return seen

    capable = set()
    for v in onb:
        near = within(v)
        for u in onb:
            d = rest[u] - rest[v]
            if u != v and u not in near and (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] < radius ** 2:
                capable.add(v)
                break
    want = [f for f in bf if all(v in capable for v in f) and not all(mesh.pinned[v] for v in f)]
    tris, verts = R.select_region(rest, tets, mesh.pinned, radius, rings)
    assert sorted(tuple(int(x) for x in verts[t]) for t in tris) == want
