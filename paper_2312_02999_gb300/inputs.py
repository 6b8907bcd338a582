"""Seeded synthetic workloads for the actuated face simulator.

This module only *builds inputs*: tetrahedral meshes (rest positions and
connectivity), Dirichlet masks, the contact proxy surface with its embedding
rows ``s = W x``, and per-tet actuation fields (fibre direction and stretch).
It holds none of the solver's arithmetic -- no energies, derivatives,
distances or linear algebra of the method -- so that the CPU oracle and the
CUDA path can be fed the very same arrays without sharing any solver code.

Workloads (shapes follow the paper's setting of Sec. 4: a face-like soft body
whose collision proxy is the mouth region, n2 about a tenth of n1 or less):

* ``two_slabs``   -- two stacked hex-grid slabs split 6 tets/hex with a small
                     gap between them; the proxy is the pair of facing faces.
* ``face_shell``  -- an ellipsoidal soft-tissue shell (front half of a head)
                     3 cm thick, inner surface pinned as the skull, with a thin
                     mouth slit that separates two lip lobes; the proxy is the
                     boundary surface around the mouth.
* ``embed_finer_surface`` -- turns a selection proxy into a finer surface
                     embedded in the tets (barycentric rows of W).
* ``bump_actuation`` -- stretch field from a sum of seeded Gaussian bumps.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

# The six tetrahedra of the Kuhn (Freudenthal) split of a unit cube: each one
# follows a monotone lattice path 000 -> e_a -> e_a+e_b -> 111 for an ordering
# (a, b, c) of the three axes.  Every cube uses the same main diagonal, so the
# split is conforming across neighbouring cubes.
_KUHN_ORDERS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


@dataclass
class MeshInput:
    """One simulation mesh plus its collision proxy and solver constants."""
    name: str
    rest: np.ndarray          # (n, 3) float64 rest positions
    tets: np.ndarray          # (T, 4) int32 vertex ids, positively oriented
    pinned: np.ndarray        # (n,) uint8, 1 = Dirichlet vertex (kept at rest)
    proxy_tris: np.ndarray    # (Nt, 3) int32 ids into the proxy vertices
    W_rowptr: np.ndarray      # (Ns+1,) int64 CSR row pointer of W
    W_col: np.ndarray         # (nnz,) int32 simulation-vertex ids
    W_val: np.ndarray         # (nnz,) float64 interpolation weights
    region: np.ndarray | None  # (n,) uint8 marks the collision-aware set, or None
    dhat: float               # barrier activation distance d0
    weight_scale: float       # w_i = weight_scale * rest volume
    tol_abs: float            # stop when ||g|| <= max(tol_abs, tol_rel*||g(x_t)||)
    tol_rel: float
    grid: dict | None = None  # generator metadata (grid indices etc.)

    @property
    def n(self) -> int:
        return int(self.rest.shape[0])

    @property
    def T(self) -> int:
        return int(self.tets.shape[0])

    @property
    def Ns(self) -> int:
        return int(self.W_rowptr.shape[0] - 1)


@dataclass
class Actuation:
    """Per-tet actuation: unit fibre direction and stretch along it."""
    fiber: np.ndarray    # (T, 3) float64 unit vectors
    stretch: np.ndarray  # (T,) float64


# ----------------------------------------------------------------------------
# generic hex-grid helpers
# ----------------------------------------------------------------------------
def _kuhn_tets(vid: np.ndarray, cell_mask: np.ndarray) -> np.ndarray:
    """Tets of all masked cells of a structured grid with vertex-id array vid."""
    I, J, K = np.nonzero(cell_mask)
    out = []
    for order in _KUHN_ORDERS:
        path = [np.zeros(3, dtype=np.int64)]
        for ax in order:
            step = path[-1].copy()
            step[ax] += 1
            path.append(step)
        tet = [vid[I + p[0], J + p[1], K + p[2]] for p in path]
        out.append(np.stack(tet, axis=1))
    tets = np.stack(out, axis=1).reshape(-1, 4)
    return tets.astype(np.int64)


def _orient(rest: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Swap two vertices of negatively oriented tets (input normalisation)."""
    a = rest[tets[:, 1]] - rest[tets[:, 0]]
    b = rest[tets[:, 2]] - rest[tets[:, 0]]
    c = rest[tets[:, 3]] - rest[tets[:, 0]]
    neg = np.einsum("ij,ij->i", np.cross(a, b), c) < 0
    tets = tets.copy()
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def _compact(rest: np.ndarray, tets: np.ndarray):
    """Drop vertices no tet references; returns (rest, tets, old->new map)."""
    used = np.zeros(rest.shape[0], dtype=bool)
    used[tets.ravel()] = True
    remap = -np.ones(rest.shape[0], dtype=np.int64)
    remap[used] = np.arange(int(used.sum()))
    return rest[used], remap[tets], remap


def boundary_faces(tets: np.ndarray) -> np.ndarray:
    """Triangles that belong to exactly one tet (the mesh boundary)."""
    f = np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]],
                        tets[:, [0, 2, 3]], tets[:, [1, 2, 3]]], axis=0)
    key = np.sort(f, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    once = cnt[inv.ravel()] == 1
    return f[once]


def _proxy_from_faces(n: int, faces: np.ndarray):
    """Selection embedding (one weight 1.0 per proxy vertex) for given faces."""
    pv = np.unique(faces.ravel())
    local = -np.ones(n, dtype=np.int64)
    local[pv] = np.arange(pv.size)
    tris = local[faces].astype(np.int32)
    rowptr = np.arange(pv.size + 1, dtype=np.int64)
    col = pv.astype(np.int32)
    val = np.ones(pv.size, dtype=np.float64)
    return tris, rowptr, col, val


# ----------------------------------------------------------------------------
# two stacked slabs (the small lip-contact case)
# ----------------------------------------------------------------------------
def two_slabs(nx: int = 10, ny: int = 10, nz: int = 3, h: float = 0.1,
              gap: float = 0.005, dhat: float = 1e-3,
              weight_scale: float = 1e3, tol_abs: float = 1e-8) -> MeshInput:
    """Two nx*ny*nz hex slabs (edge h), 6 tets per hex, stacked with a gap.

    The lower face of the bottom slab and the upper face of the top slab are
    pinned; the proxy is the upper face of the bottom slab plus the lower face
    of the top slab (selection embedding, so the proxy vertices are mesh
    vertices).
    """
    rests, tets_all, pins, zs = [], [], [], []
    base = 0
    for slab in range(2):
        z0 = 0.0 if slab == 0 else nz * h + gap
        gx, gy, gz = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1),
                                 np.arange(nz + 1), indexing="ij")
        vid = (gx * (ny + 1) + gy) * (nz + 1) + gz
        rest = np.stack([gx * h, gy * h, z0 + gz * h], axis=-1).reshape(-1, 3)
        tets = _kuhn_tets(vid, np.ones((nx, ny, nz), dtype=bool))
        pin = (gz.ravel() == 0) if slab == 0 else (gz.ravel() == nz)
        rests.append(rest)
        tets_all.append(tets + base)
        pins.append(pin)
        zs.append((gz.ravel(), slab))
        base += rest.shape[0]
    rest = np.concatenate(rests).astype(np.float64)
    tets = _orient(rest, np.concatenate(tets_all))
    pinned = np.concatenate(pins).astype(np.uint8)
    # facing faces: top of slab 0 (gz == nz), bottom of slab 1 (gz == 0)
    n0 = rests[0].shape[0]
    facing = np.zeros(rest.shape[0], dtype=bool)
    facing[:n0] = zs[0][0] == nz
    facing[n0:] = zs[1][0] == 0
    bf = boundary_faces(tets)
    faces = bf[facing[bf].all(axis=1)]
    tris, rowptr, col, val = _proxy_from_faces(rest.shape[0], faces)
    return MeshInput(name=f"two_slabs_{nx}x{ny}x{nz}", rest=rest,
                     tets=tets.astype(np.int32), pinned=pinned, proxy_tris=tris,
                     W_rowptr=rowptr, W_col=col, W_val=val, region=None,
                     dhat=dhat, weight_scale=weight_scale, tol_abs=tol_abs,
                     tol_rel=0.0, grid={"nx": nx, "ny": ny, "nz": nz, "h": h})


def slab_actuation(mesh: MeshInput, seed: int = 1, lo: float = 0.7,
                   hi: float = 1.0) -> Actuation:
    """Fibre along +x for every tet, stretch ~ U[lo, hi] per tet."""
    rng = np.random.default_rng(seed)
    T = mesh.T
    fiber = np.zeros((T, 3), dtype=np.float64)
    fiber[:, 0] = 1.0
    stretch = rng.uniform(lo, hi, size=T).astype(np.float64)
    return Actuation(fiber=fiber, stretch=stretch)


# ----------------------------------------------------------------------------
# face-like ellipsoidal shell with a mouth slit
# ----------------------------------------------------------------------------
def face_shell(n_target: int = 30000, nr: int = 7, thickness: float = 0.03,
               semi=(0.08, 0.11, 0.09), slit: float = 5e-4,
               slit_layers: int = 4, mouth_half_angle: float = 32.0,
               theta_range=(-55.0, 65.0), phi_range=(-80.0, 80.0),
               theta_mouth: float = -20.0, proxy_phi: float = 60.0,
               proxy_theta: float = 22.0, dhat_rel: float = 1e-4,
               weight_scale: float = 1e3, tol_abs: float = 1e-10,
               tol_rel: float = 1e-7) -> MeshInput:
    """Front half of an ellipsoidal head, ``thickness`` thick, nr vertex layers.

    Vertex (i, j, k) sits at the outer ellipsoid point for azimuth phi_i and
    elevation theta_j, moved inward along the ellipsoid normal by
    ``k/(nr-1) * thickness`` (k = 0 outer skin, k = nr-1 skull, pinned).  The
    theta row that holds the mouth is made ``slit`` metres tall and its cells
    are removed in the outer ``slit_layers`` layers over |phi| <=
    mouth_half_angle, leaving an upper and a lower lip lobe that face each
    other across the slit.  The proxy is every non-skull boundary triangle
    whose vertices lie within |phi| <= proxy_phi and |theta - theta_mouth| <=
    proxy_theta (the mouth region).
    """
    ax, ay, az = semi
    ntheta = max(8, int(round(math.sqrt(n_target / nr * 54.0 / 80.0))))
    nphi = max(8, int(round(n_target / (nr * ntheta))))
    phi = np.deg2rad(np.linspace(phi_range[0], phi_range[1], nphi))
    # theta grid: uniform rows except one thin row at the mouth
    t0, t1 = np.deg2rad(theta_range[0]), np.deg2rad(theta_range[1])
    tm = np.deg2rad(theta_mouth)
    r_mouth = math.hypot(ay * math.cos(tm), az * math.sin(tm))
    dslit = slit / r_mouth
    nrow = ntheta - 1
    drow = (t1 - t0 - dslit) / (nrow - 1)
    jm = int(round((tm - t0) / drow))
    jm = min(max(jm, 2), nrow - 3)
    steps = np.full(nrow, drow)
    steps[jm] = dslit
    theta = t0 + np.concatenate([[0.0], np.cumsum(steps)])

    P, T_, K = np.meshgrid(phi, theta, np.arange(nr), indexing="ij")
    outer = np.stack([ax * np.sin(P) * np.cos(T_), ay * np.sin(T_),
                      az * np.cos(P) * np.cos(T_)], axis=-1)
    nrm = outer / np.array([ax * ax, ay * ay, az * az])
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    depth = (K / (nr - 1) * thickness)[..., None]
    pos = outer - depth * nrm
    gi, gj, gk = np.meshgrid(np.arange(nphi), np.arange(ntheta), np.arange(nr),
                             indexing="ij")
    vid = (gi * ntheta + gj) * nr + gk
    cells = np.ones((nphi - 1, ntheta - 1, nr - 1), dtype=bool)
    phic = 0.5 * (phi[:-1] + phi[1:])
    in_mouth = np.abs(np.rad2deg(phic)) <= mouth_half_angle
    cells[np.ix_(in_mouth, [jm], np.arange(min(slit_layers, nr - 1)))] = False
    tets = _kuhn_tets(vid, cells)
    rest = pos.reshape(-1, 3).astype(np.float64)
    rest, tets, remap = _compact(rest, tets)
    tets = _orient(rest, tets)
    keep = remap >= 0
    gi_, gj_, gk_ = gi.ravel()[keep], gj.ravel()[keep], gk.ravel()[keep]
    pinned = (gk_ == nr - 1).astype(np.uint8)
    phv = np.rad2deg(phi[gi_])
    thv = np.rad2deg(theta[gj_])
    in_region = ((np.abs(phv) <= proxy_phi) & (np.abs(thv - theta_mouth) <= proxy_theta)
                 & (pinned == 0))
    bf = boundary_faces(tets)
    faces = bf[in_region[bf].all(axis=1)]
    tris, rowptr, col, val = _proxy_from_faces(rest.shape[0], faces)
    diag = float(np.linalg.norm(rest.max(0) - rest.min(0)))
    return MeshInput(name=f"face_shell_{rest.shape[0]}", rest=rest,
                     tets=tets.astype(np.int32), pinned=pinned, proxy_tris=tris,
                     W_rowptr=rowptr, W_col=col, W_val=val, region=None,
                     dhat=dhat_rel * diag, weight_scale=weight_scale,
                     tol_abs=tol_abs, tol_rel=tol_rel,
                     grid={"nphi": nphi, "ntheta": ntheta, "nr": nr, "jm": jm,
                           "gi": gi_, "gj": gj_, "gk": gk_,
                           "theta_mouth": theta_mouth})


# ----------------------------------------------------------------------------
# embedded finer proxy surface (general barycentric rows of W)
# ----------------------------------------------------------------------------
def embed_finer_surface(mesh: MeshInput, levels: int = 2, relief: float = 0.15,
                        seed: int = 7) -> MeshInput:
    """Replace a selection proxy by a finer surface embedded in the tet mesh.

    Sec. 3.1 lets the collision proxy be a surface finer than the simulation
    mesh, each proxy vertex interpolated from the tet that contains it (s = W x
    with barycentric rows).  Every proxy triangle (a boundary face of one tet)
    is split 4^levels ways on the lattice of step 1/2^levels.  Lattice points
    on the face's corners and edges stay on the face (rows of 1 and 2 entries,
    shared by the neighbouring faces); interior lattice points are pulled into
    the owning tet towards its fourth vertex by a seeded fraction
    mu ~ U[0, relief] of the way (rows of 4 entries), which gives the finer
    surface its own small relief below the coarse one.
    """
    if not np.all(np.diff(mesh.W_rowptr) == 1) or not np.all(mesh.W_val == 1.0):
        raise ValueError("embed_finer_surface expects a selection proxy")
    if levels < 1:
        raise ValueError("levels must be >= 1")
    N = 1 << levels
    faces = mesh.W_col[mesh.W_rowptr[:-1]][mesh.proxy_tris].astype(np.int64)   # mesh ids
    # owning tet of each face and its fourth vertex
    tets = mesh.tets.astype(np.int64)
    owner = {}
    for t in range(tets.shape[0]):
        q = tets[t]
        for drop in range(4):
            f = tuple(sorted(np.delete(q, drop).tolist()))
            owner.setdefault(f, []).append((t, int(q[drop])))
    apex = np.empty(faces.shape[0], dtype=np.int64)
    for k in range(faces.shape[0]):
        own = owner[tuple(sorted(faces[k].tolist()))]
        if len(own) != 1:
            raise ValueError("proxy face is not a boundary face")
        apex[k] = own[0][1]
    rng = np.random.default_rng(seed)
    points = {}      # lattice key -> proxy id
    rows = []        # proxy id -> {mesh vertex: weight}

    def point(k, i, j):
        a, b, c = (int(v) for v in faces[k])
        lam = {a: (N - i - j) / N, b: i / N, c: j / N}
        nz = [v for v in (a, b, c) if lam[v] != 0.0]
        if len(nz) == 1:
            key = ("v", nz[0])
        elif len(nz) == 2:
            lo, hi = min(nz), max(nz)
            key = ("e", lo, hi, round(lam[hi] * N))
        else:
            key = ("f", k, i, j)
        pid = points.get(key)
        if pid is not None:
            return pid
        row = {v: lam[v] for v in nz}
        if len(nz) == 3:
            mu = relief * rng.uniform()
            row = {v: (1.0 - mu) * w for v, w in row.items()}
            row[int(apex[k])] = mu
        pid = len(rows)
        points[key] = pid
        rows.append(row)
        return pid

    tris = []
    for k in range(faces.shape[0]):
        idx = {}
        for i in range(N + 1):
            for j in range(N + 1 - i):
                idx[i, j] = point(k, i, j)
        for i in range(N):
            for j in range(N - i):
                tris.append((idx[i, j], idx[i + 1, j], idx[i, j + 1]))
                if i + j <= N - 2:
                    tris.append((idx[i + 1, j], idx[i + 1, j + 1], idx[i, j + 1]))
    rowptr = np.zeros(len(rows) + 1, dtype=np.int64)
    col, val = [], []
    for r, row in enumerate(rows):
        for v in sorted(row):
            col.append(v)
            val.append(row[v])
        rowptr[r + 1] = len(col)
    return MeshInput(name=f"{mesh.name}_embedded{levels}", rest=mesh.rest, tets=mesh.tets,
                     pinned=mesh.pinned, proxy_tris=np.asarray(tris, dtype=np.int32),
                     W_rowptr=rowptr, W_col=np.asarray(col, dtype=np.int32),
                     W_val=np.asarray(val, dtype=np.float64), region=mesh.region,
                     dhat=mesh.dhat, weight_scale=mesh.weight_scale, tol_abs=mesh.tol_abs,
                     tol_rel=mesh.tol_rel, grid=mesh.grid)


@dataclass
class BumpField:
    """Gaussian bumps g_k(y) = exp(-|y - c_k|^2 / (2 s_k^2)) over tet centroids."""
    centres: np.ndarray   # (K, 3)
    sigmas: np.ndarray    # (K,)
    fiber: np.ndarray     # (T, 3) per-tet random unit fibre
    basis: np.ndarray     # (T, K) bump values at tet centroids


def bump_field(mesh: MeshInput, n_bumps: int = 16, seed: int = 2,
               sigma_range=(0.01, 0.03)) -> BumpField:
    """Seeded bump centres on the outer skin near the mouth; random fibres."""
    rng = np.random.default_rng(seed)
    g = mesh.grid
    skin = np.nonzero(g["gk"] == 0)[0]
    # centres: half near the mouth, half anywhere on the outer skin
    rest = mesh.rest
    tm = g["theta_mouth"]
    ys = rest[skin, 1]
    ymouth = np.median(rest[skin][np.abs(np.rad2deg(np.arcsin(np.clip(
        ys / 0.11, -1, 1))) - tm) < 6.0, 1]) if skin.size else 0.0
    near = skin[np.abs(ys - ymouth) < 0.02]
    pick = np.concatenate([rng.choice(near, size=n_bumps // 2, replace=near.size < n_bumps // 2),
                           rng.choice(skin, size=n_bumps - n_bumps // 2, replace=False)])
    centres = rest[pick].copy()
    sigmas = rng.uniform(sigma_range[0], sigma_range[1], size=n_bumps)
    f = rng.normal(size=(mesh.T, 3))
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    cent = rest[mesh.tets].mean(axis=1)
    d2 = ((cent[:, None, :] - centres[None, :, :]) ** 2).sum(-1)
    basis = np.exp(-d2 / (2.0 * sigmas[None, :] ** 2))
    return BumpField(centres=centres, sigmas=sigmas, fiber=f, basis=basis)


def bump_actuation(field: BumpField, coeffs: np.ndarray, depth: float = 0.4) -> Actuation:
    """stretch = 1 - depth * clamp(sum_k c_k g_k, 0, 1), in [1 - depth, 1]."""
    s = field.basis @ np.asarray(coeffs, dtype=np.float64)
    stretch = 1.0 - depth * np.clip(s, 0.0, 1.0)
    return Actuation(fiber=field.fiber.copy(), stretch=stretch)


def keyframe_coeffs(n_bumps: int = 16, n_keys: int = 5, n_frames: int = 100,
                    seed: int = 3) -> np.ndarray:
    """(n_frames, n_bumps) coefficients linearly interpolated between keyframes."""
    rng = np.random.default_rng(seed)
    keys = rng.uniform(0.0, 1.0, size=(n_keys, n_bumps))
    keys[0] = 0.0                     # the sequence starts from the rest pose
    tpos = np.linspace(0.0, n_keys - 1, n_frames)
    lo = np.minimum(np.floor(tpos).astype(int), n_keys - 2)
    fr = (tpos - lo)[:, None]
    return (1.0 - fr) * keys[lo] + fr * keys[lo + 1]


def request_coeffs(n_requests: int, n_bumps: int = 64, seed: int = 5) -> np.ndarray:
    """Serving requests: c ~ U[0,1]^n_bumps per request."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(n_requests, n_bumps))


def perturbed_positions(mesh: MeshInput, scale: float, seed: int = 7) -> np.ndarray:
    """Rest positions plus seeded noise on free vertices (for unit tests)."""
    rng = np.random.default_rng(seed)
    x = mesh.rest.copy()
    free = mesh.pinned == 0
    x[free] += scale * rng.standard_normal((int(free.sum()), 3))
    return x
