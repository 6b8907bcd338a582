"""Oracle: IPC constraint set, barrier energy and derivatives, PSD projection,
additive CCD.

Paper passages followed (Sec. 2.2, Algorithm 1, Sec. 3.1):
* Sec. 2.2 -- primitive pairs are vertex-triangle and edge-edge; the unsigned
  distance d_k feeds a log-like barrier b(d_k) that is active only for
  d_k < d0; the active pairs form the constraint set C.
* Eq. 3 -- B(x) = kappa * sum_{k in C} b(d_k(x)).
* Algorithm 1 -- UpdateConstraintSet(x, d0); PositiveDefinite(B(x, C));
  alpha_m = CCD(x, dx).
* Sec. 3.1 -- the proxy s = W x carries all contact quantities; gradient and
  Hessian map back as W^T grad B(s) and W^T hess B(s) W.

Readings where the paper is silent:
* barrier b(d) = -(d - dhat)^2 ln(d / dhat) for 0 < d < dhat, else 0 (the IPC
  barrier on the unsquared distance); active iff d < dhat strictly.
* pairs: proxy vertex vs proxy triangle not containing it; proxy edges that
  share no vertex; every pair is its own term.
* PositiveDefinite: each pair's 12x12 Hessian in s-space is projected onto
  the PSD cone by clamping negative eigenvalues to zero.
* optional EE mollifier (the paper uses IPC; IPC multiplies each edge-edge
  term by a mollifier of the squared edge cross product, Li et al. 2020,
  "Incremental Potential Contact"): m(c) = (2 - c/eps) c/eps below
  eps = 1e-3 |E_a|^2 |E_b|^2 (rest edges), else 1.
* CCD: additive CCD (Li, Kaufman & Jiang 2021, "Codimensional Incremental
  Potential Contact") with gap ratio s = 0.1 and zero thickness, on every pair
  whose swept boxes (over the step), inflated by dhat, overlap; the step bound
  is alpha_m = min(1, min over pairs of the time of impact).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import distance as D
from .distance import Hd, distance, distance_hd

ACCD_MAX_ITERS = 2000


# ---------------------------------------------------------------------------
# barrier (Eq. 3 reading)
# ---------------------------------------------------------------------------
def barrier(d, dhat):
    """b(d) = -(d - dhat)^2 ln(d/dhat) on 0 < d < dhat, 0 beyond."""
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    m = d < dhat
    out[m] = -((d[m] - dhat) ** 2) * np.log(d[m] / dhat)
    return out


def barrier_hd(d: Hd, dhat: float) -> Hd:
    """b(d) as an Hd number (for pairs already known to have d < dhat)."""
    u = d - dhat
    return -(u * u) * (d / dhat).log()


# ---------------------------------------------------------------------------
# primitives and constraint set (UpdateConstraintSet of Algorithm 1)
# ---------------------------------------------------------------------------
def proxy_edges(tris: np.ndarray) -> np.ndarray:
    """Unique undirected edges of the proxy triangles, (lo, hi) sorted rows."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def _boxes(P: np.ndarray):
    return P.min(axis=1), P.max(axis=1)


def _overlap_pairs(lo_a, hi_a, lo_b, hi_b, pad, chunk=2048):
    """All (i, j) with closed boxes [lo_a-pad, hi_a+pad] and [lo_b, hi_b] overlapping."""
    out_i, out_j = [], []
    for s in range(0, lo_a.shape[0], chunk):
        la, ha = lo_a[s:s + chunk, None, :], hi_a[s:s + chunk, None, :]
        ok = ((la - pad <= hi_b[None]) & (lo_b[None] <= ha + pad)).all(axis=2)
        i, j = np.nonzero(ok)
        out_i.append(i + s)
        out_j.append(j)
    return np.concatenate(out_i), np.concatenate(out_j)


def candidate_pairs(s: np.ndarray, tris: np.ndarray, edges: np.ndarray,
                    pad: float, s_end: np.ndarray | None = None):
    """PT and EE pairs whose (swept) boxes inflated by ``pad`` overlap.

    Adjacent pairs (PT with the point in the triangle, EE sharing a vertex)
    are excluded.  With ``s_end`` the boxes cover both endpoints of the step.
    Returns int64 arrays (type, i, j): type 0 = PT (vertex i, triangle j),
    type 1 = EE (edge i < edge j).
    """
    pts = s[:, None, :] if s_end is None else np.stack([s, s_end], axis=1)
    tri_pts = s[tris] if s_end is None else np.concatenate([s[tris], s_end[tris]], axis=1)
    edg_pts = s[edges] if s_end is None else np.concatenate([s[edges], s_end[edges]], axis=1)
    vlo, vhi = _boxes(pts)
    tlo, thi = _boxes(tri_pts)
    elo, ehi = _boxes(edg_pts)
    vi, tj = _overlap_pairs(vlo, vhi, tlo, thi, pad)
    keep = ~(tris[tj] == vi[:, None]).any(axis=1)
    vi, tj = vi[keep], tj[keep]
    ei, ej = _overlap_pairs(elo, ehi, elo, ehi, pad)
    keep = ei < ej
    ei, ej = ei[keep], ej[keep]
    share = ((edges[ei][:, :, None] == edges[ej][:, None, :]).any(axis=(1, 2)))
    ei, ej = ei[~share], ej[~share]
    typ = np.concatenate([np.zeros(vi.size, np.int64), np.ones(ei.size, np.int64)])
    return typ, np.concatenate([vi, ei]).astype(np.int64), np.concatenate([tj, ej]).astype(np.int64)


def pair_vertices(typ, i, j, tris, edges) -> np.ndarray:
    """Proxy vertex ids (P,4): PT -> (p, t0, t1, t2); EE -> (a0, a1, b0, b1)."""
    V = np.empty((typ.size, 4), dtype=np.int64)
    pt = typ == 0
    V[pt, 0] = i[pt]
    V[pt, 1:] = tris[j[pt]]
    V[~pt, 0:2] = edges[i[~pt]]
    V[~pt, 2:4] = edges[j[~pt]]
    return V


def constraint_set(s: np.ndarray, tris: np.ndarray, edges: np.ndarray, dhat: float):
    """C = all PT/EE pairs with d < dhat, sorted by (type, i, j); plus d.

    Every pair is considered: a box test inflated by dhat only skips pairs
    whose coordinate gap alone already exceeds dhat (then d > dhat).
    """
    typ, i, j = candidate_pairs(s, tris, edges, dhat)
    V = pair_vertices(typ, i, j, tris, edges)
    d = distance(s[V], typ == 1)
    m = d < dhat
    typ, i, j, d = typ[m], i[m], j[m], d[m]
    order = np.lexsort((j, i, typ))
    return typ[order], i[order], j[order], d[order]


def barrier_energy(s, tris, edges, dhat, kappa, s_rest=None) -> float:
    """B = kappa * sum over C of b(d_k) at proxy positions s (Eq. 3); with
    s_rest, EE terms carry the mollifier m(c_k)."""
    typ, i, j, d = constraint_set(s, tris, edges, dhat)
    return float(kappa * pair_barrier_values(s, typ, i, j, d, tris, edges, dhat, s_rest).sum())


# ---------------------------------------------------------------------------
# edge-edge mollifier (IPC's treatment of nearly parallel edges; optional)
# ---------------------------------------------------------------------------
# For an edge-edge pair with edges e_a, e_b let c = |e_a x e_b|^2.  Below the
# threshold eps_x = MOLLIFIER_EPS_SCALE |E_a|^2 |E_b|^2 (rest edge vectors E)
# the pair's barrier is multiplied by m(c) = (2 - c/eps_x) c/eps_x, which is 0
# for parallel edges, 1 with zero slope at c = eps_x, and 1 beyond; so the
# pair's term kappa m(c) b(d) stays C^1 where the closest features of two
# edges jump as they turn parallel.
MOLLIFIER_EPS_SCALE = 1e-3


def ee_mollifier_eps(s_rest: np.ndarray, edges: np.ndarray, i: np.ndarray, j: np.ndarray):
    """eps_x of EE pairs (edge i, edge j) from the rest proxy positions."""
    ea = s_rest[edges[i, 1]] - s_rest[edges[i, 0]]
    eb = s_rest[edges[j, 1]] - s_rest[edges[j, 0]]
    return MOLLIFIER_EPS_SCALE * np.einsum("ij,ij->i", ea, ea) * np.einsum("ij,ij->i", eb, eb)


def edge_cross_sq(X: np.ndarray) -> np.ndarray:
    """c = |(a1 - a0) x (b1 - b0)|^2 for EE pairs X (P,4,3) = (a0, a1, b0, b1)."""
    w = np.cross(X[:, 1] - X[:, 0], X[:, 3] - X[:, 2])
    return np.einsum("ij,ij->i", w, w)


def mollifier(c: np.ndarray, eps: np.ndarray) -> np.ndarray:
    q = c / eps
    return np.where(c < eps, (2.0 - q) * q, 1.0)


def mollifier_hd(X: np.ndarray, eps: np.ndarray) -> Hd:
    """m(c) with gradient and Hessian in the pair's 12 coordinates."""
    a0, a1, b0, b1 = (D._vec(X, k) for k in range(4))
    w = D._cross3(D._sub3(a1, a0), D._sub3(b1, b0))
    c = D._dot3(w, w)
    q = c * (1.0 / eps)
    m = (2.0 - q) * q
    one = Hd(np.ones(X.shape[0]), np.zeros_like(m.g), np.zeros_like(m.h))
    return m.select(c.v < eps, one)


def pair_barrier_values(s, typ, i, j, d, tris, edges, dhat, s_rest=None) -> np.ndarray:
    """b(d_k), times m(c_k) for EE pairs when s_rest (mollifier) is given."""
    b = barrier(d, dhat)
    if s_rest is not None:
        ee = np.nonzero(typ == 1)[0]
        if ee.size:
            V = pair_vertices(typ[ee], i[ee], j[ee], tris, edges)
            b[ee] *= mollifier(edge_cross_sq(s[V]), ee_mollifier_eps(s_rest, edges, i[ee], j[ee]))
    return b


# ---------------------------------------------------------------------------
# barrier derivatives and PSD projection
# ---------------------------------------------------------------------------
def psd_project(Hs: np.ndarray) -> np.ndarray:
    """Project symmetric matrices onto the PSD cone (clamp eigenvalues < 0)."""
    lam, Q = np.linalg.eigh(0.5 * (Hs + np.swapaxes(Hs, -1, -2)))
    lam = np.maximum(lam, 0.0)
    return np.einsum("pik,pk,pjk->pij", Q, lam, Q)


def pair_barrier_derivatives(s, typ, i, j, tris, edges, dhat, kappa, project=True, s_rest=None):
    """Per-pair kappa*b(d) gradient (P,12) and (PSD) Hessian (P,12,12); with
    s_rest, EE pairs take kappa*m(c)*b(d) (the mollified term)."""
    V = pair_vertices(typ, i, j, tris, edges)
    d = distance_hd(s[V], typ == 1)
    b = barrier_hd(d, dhat)
    if s_rest is not None:
        ee = np.nonzero(typ == 1)[0]
        if ee.size:
            m = mollifier_hd(s[V[ee]], ee_mollifier_eps(s_rest, edges, i[ee], j[ee]))
            be = Hd(b.v[ee], b.g[ee], b.h[ee]) * m
            b.v[ee], b.g[ee], b.h[ee] = be.v, be.g, be.h
    g = kappa * b.g
    h = kappa * b.h
    if project:
        h = psd_project(h)
    return V, g, h


# ---------------------------------------------------------------------------
# additive CCD
# ---------------------------------------------------------------------------
def accd_toi(X: np.ndarray, dX: np.ndarray, is_ee: np.ndarray, s_ratio: float = 0.1,
             t_max: float = 1.0, max_iters: int = ACCD_MAX_ITERS) -> np.ndarray:
    """Conservative time of impact per pair by additive CCD (zero thickness).

    The mean displacement is removed (distance is translation invariant) and
    l_p bounds how fast the distance can shrink per unit time: PT uses
    |dp| + max |dt_k|, EE max |da| + max |db|.  Starting from t = 0, each step
    advances by a fraction of (current distance / l_p) -- (1 - s) for the
    first, 0.9 afterwards -- so the pair never touches; the march stops when
    a step would bring the distance below s * d(0) (the pair's TOI is then the
    time before that step) or when it passes t_max (no impact: TOI = t_max).
    """
    P = X.shape[0]
    toi = np.full(P, t_max)
    if P == 0:
        return toi
    dX = dX - dX.mean(axis=1, keepdims=True)
    nrm = np.linalg.norm(dX, axis=2)
    lp = np.where(is_ee, np.maximum(nrm[:, 0], nrm[:, 1]) + np.maximum(nrm[:, 2], nrm[:, 3]),
                  nrm[:, 0] + nrm[:, 1:].max(axis=1))
    act = lp > 0.0
    d0 = distance(X, is_ee)
    gap = s_ratio * d0
    t = np.zeros(P)
    step = np.where(act, (1.0 - s_ratio) * d0 / np.where(act, lp, 1.0), 0.0)
    Xc = X.copy()
    for _ in range(max_iters):
        idx = np.nonzero(act)[0]
        if idx.size == 0:
            break
        Xc[idx] += step[idx, None, None] * dX[idx]
        d = distance(Xc[idx], is_ee[idx])
        hit = (t[idx] > 0.0) & (d < gap[idx])
        toi[idx[hit]] = t[idx[hit]]
        act[idx[hit]] = False
        go = idx[~hit]
        dgo = d[~hit]
        t[go] += step[go]
        done = t[go] > t_max
        act[go[done]] = False
        cont = go[~done]
        step[cont] = 0.9 * dgo[~done] / lp[cont]
    # pairs still marching after max_iters keep the time reached (safe)
    toi[act] = np.minimum(t[act], t_max)
    return toi


def ccd_step_bound(s: np.ndarray, ds: np.ndarray, tris, edges, dhat: float,
                   s_ratio: float = 0.1) -> float:
    """alpha_m = min(1, min TOI) over pairs whose swept boxes (+dhat) overlap."""
    typ, i, j = candidate_pairs(s, tris, edges, dhat, s_end=s + ds)
    if typ.size == 0:
        return 1.0
    V = pair_vertices(typ, i, j, tris, edges)
    toi = accd_toi(s[V], ds[V], typ == 1, s_ratio=s_ratio)
    return float(min(1.0, toi.min()))
