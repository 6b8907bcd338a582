"""Pins for a collision proxy embedded in the tets with barycentric rows of W.

Sec. 3.1 allows the proxy to be a finer surface than the simulation mesh,
each proxy vertex interpolated inside one tet (s = W x).  References used:
exact geometry of the lattice refinement (points on the coarse faces, areas
that add up, unchanged Euler characteristic), finite differences of the
barrier energy taken through the barycentric W, the three algebraically equal
global steps (direct, Schur 3-step of Eq. 8, push-through Woodbury of Eq. 11)
when W couples interior vertices into x2, and IPC's solver invariants.
"""
import numpy as np
import pytest

from oracle import contact as C
from oracle import distance as D
from oracle import solver as S
from paper_2312_02999_gb300 import inputs as I

rng = np.random.default_rng(17)


def _coarse(nx=3, nz=2, gap=0.0004):
    return I.two_slabs(nx, nx, nz, gap=gap)


def _tri_area(P, tris):
    a, b, c = P[tris[:, 0]], P[tris[:, 1]], P[tris[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def _euler(ns, tris):
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [0, 2]]]), axis=1)
    return ns - np.unique(e, axis=0).shape[0] + tris.shape[0]


@pytest.mark.parametrize("levels", [1, 2])
def test_rows_are_barycentric_in_the_owning_tet(levels):
    m = _coarse()
    e = I.embed_finer_surface(m, levels=levels, relief=0.2)
    nnz = np.diff(e.W_rowptr)
    assert set(np.unique(nnz).tolist()) <= {1, 2, 4}
    assert (nnz == 4).any() == (levels >= 2)      # interior lattice points need levels >= 2
    assert e.W_val.min() > 0.0
    sums = np.add.reduceat(e.W_val, e.W_rowptr[:-1])
    assert np.abs(sums - 1.0).max() <= 1e-15
    coarse_v = set(m.W_col.tolist())
    coarse_e = set()
    for t in m.W_col[m.proxy_tris]:
        for a, b in ((0, 1), (1, 2), (0, 2)):
            coarse_e.add((min(t[a], t[b]), max(t[a], t[b])))
    tets = set(tuple(sorted(t)) for t in m.tets.tolist())
    for r in range(e.Ns):
        cols = e.W_col[e.W_rowptr[r]:e.W_rowptr[r + 1]].tolist()
        if len(cols) == 1:
            assert cols[0] in coarse_v
        elif len(cols) == 2:
            assert tuple(sorted(cols)) in coarse_e
        else:
            assert tuple(sorted(cols)) in tets
    # corners keep the coarse positions exactly; refinement multiplies the
    # triangle count by 4^levels
    s = e.rest[e.W_col[e.W_rowptr[:-1]]]
    one = nnz == 1
    assert np.array_equal(s[one], e.rest[e.W_col[e.W_rowptr[:-1][one]]])
    assert e.proxy_tris.shape[0] == m.proxy_tris.shape[0] * 4 ** levels


def test_flat_refinement_tiles_the_coarse_surface():
    m = _coarse()
    e = I.embed_finer_surface(m, levels=2, relief=0.0)
    W = S.sp.csr_matrix((e.W_val, e.W_col, e.W_rowptr), shape=(e.Ns, e.n))
    s = W @ e.rest
    sc = m.rest[m.W_col]
    area_c = _tri_area(sc, m.proxy_tris.astype(np.int64))
    area_f = _tri_area(s, e.proxy_tris.astype(np.int64))
    assert abs(area_f.sum() - area_c.sum()) <= 1e-13 * area_c.sum()
    # every fine triangle is 1/16 of its coarse parent (uniform lattice)
    assert np.allclose(np.sort(area_f), np.repeat(np.sort(area_c), 16) / 16.0, rtol=1e-12)
    # no two proxy vertices coincide (shared edge points are merged): the
    # closest pair is one across the 0.0004 gap between the slabs
    d = np.linalg.norm(s[:, None] - s[None], axis=2) + np.eye(e.Ns)
    assert abs(d.min() - 0.0004) <= 1e-12
    assert _euler(e.Ns, e.proxy_tris) == _euler(m.Ns, m.proxy_tris)


def test_barrier_gradient_through_barycentric_rows_matches_finite_differences():
    m = I.embed_finer_surface(_coarse(nx=2, nz=2), levels=2, relief=0.02)
    p = S.Params(dhat=m.dhat)
    pr = S.Problem(m.rest, m.tets, m.pinned, m.proxy_tris, m.W_rowptr, m.W_col, m.W_val, p)
    act = I.slab_actuation(m, lo=1.0, hi=1.0)
    pr.set_actuation(act.fiber, act.stretch)
    x = m.rest.copy()
    free = np.nonzero(m.pinned == 0)[0]
    x[free] += 5e-5 * rng.normal(size=(free.size, 3))
    ev = pr.evaluate(x)
    assert ev["C"][0].size > 0
    V, gp, _ = pr._pair_terms(ev, project=False)
    gs = np.zeros((pr.W.shape[0], 3))
    np.add.at(gs, V.ravel(), gp.reshape(-1, 3))
    gB = (pr.W.T @ gs).ravel()
    HB = pr.barrier_hessian(ev, project=False).toarray()
    # some active proxy vertex is interpolated from four mesh vertices
    nnz = np.diff(m.W_rowptr)
    assert (nnz[np.unique(V)] == 4).any()
    apex = set(m.W_col[np.repeat(nnz == 4, nnz)].tolist()) - set(
        m.W_col[np.repeat(nnz < 4, nnz)].tolist())
    touched = np.nonzero(np.abs(gB) > 0)[0]
    touched_apex = [k for k in touched if k // 3 in apex]
    assert touched_apex

    def Bx(xx):
        return C.barrier_energy(pr.W @ xx, pr.tris, pr.edges, m.dhat, pr.kappa)

    eps = 1e-9
    pick = list(rng.choice(touched, size=min(8, touched.size), replace=False)) + touched_apex[:4]
    for k in pick:
        xp, xm = x.ravel().copy(), x.ravel().copy()
        xp[k] += eps
        xm[k] -= eps
        fd = (Bx(xp.reshape(-1, 3)) - Bx(xm.reshape(-1, 3))) / (2 * eps)
        assert abs(fd - gB[k]) <= 1e-5 * max(1.0, abs(gB[k]))

    def mapped_grad(xx):
        ss = pr.W @ xx.reshape(-1, 3)
        Vv, g2, _ = C.pair_barrier_derivatives(ss, *ev["C"][:3], pr.tris, pr.edges,
                                               m.dhat, pr.kappa, project=False)
        out = np.zeros((pr.W.shape[0], 3))
        np.add.at(out, Vv.ravel(), g2.reshape(-1, 3))
        return (pr.W.T @ out).ravel()

    # an apex moves its proxy points by mu <= relief times its own step, so
    # the difference step is larger than for a selection row
    for k in touched_apex[:2]:
        xp, xm = x.ravel().copy(), x.ravel().copy()
        xp[k] += 1e-8
        xm[k] -= 1e-8
        col = (mapped_grad(xp) - mapped_grad(xm)) / 2e-8
        assert np.allclose(col, HB[:, k], rtol=1e-4, atol=1e-4 * np.abs(HB[:, k]).max())


def _embedded_problem(nx=3, nz=2, gap=0.0004, levels=2, relief=0.02, lo=0.7, region=None):
    m = I.embed_finer_surface(_coarse(nx=nx, nz=nz, gap=gap), levels=levels, relief=relief)
    a = I.slab_actuation(m, seed=5, lo=lo)
    pr = S.Problem(m.rest, m.tets, m.pinned, m.proxy_tris, m.W_rowptr, m.W_col, m.W_val,
                   S.Params(dhat=m.dhat, tol_abs=1e-8), region=region)
    pr.set_actuation(a.fiber, a.stretch)
    return m, pr


def test_schur_and_woodbury_equal_direct_with_barycentric_rows():
    m, pr = _embedded_problem()
    x = m.rest.copy()
    free = np.nonzero(m.pinned == 0)[0]
    x[free] += 1e-4 * rng.normal(size=(free.size, 3))
    ev = pr.evaluate(x)
    assert ev["C"][0].size > 0
    g = pr.gradient(x, ev).ravel()[pr.free_dofs]
    B = pr.free_part(pr.barrier_hessian(ev))
    dx = pr.global_step_direct(g, B)
    Hd, Bd = pr.H.toarray(), B.toarray()
    i1, i2 = pr.split_dofs()
    # x2 (support of W) now holds interior vertices, and B still lives on it alone
    assert pr.x2_mask.sum() > np.unique(m.W_col[np.repeat(np.diff(m.W_rowptr) < 4,
                                                          np.diff(m.W_rowptr))]).size
    assert np.abs(Bd[np.ix_(i1, i1)]).max() == 0 and np.abs(Bd[np.ix_(i1, i2)]).max() == 0
    scale = np.abs(dx).max()
    assert np.abs(S.schur_three_step(Hd, Bd, g, i1, i2) - dx).max() <= 1e-10 * scale
    # Eq. 11 goes through the explicit Sigma^-1, which is not backward stable:
    # its forward error grows like cond(H-hat) * eps (here cond ~ 8e4, with
    # thousands of pairs down to 0.28 dhat)
    bound = 1e3 * np.finfo(float).eps * np.linalg.cond(Hd + Bd)
    assert np.abs(S.woodbury_global_step(Hd, Bd, g, i1, i2) - dx).max() <= bound * scale


def test_algorithm1_invariants_with_an_embedded_proxy():
    m, pr = _embedded_problem(nx=2, nz=2, gap=0.005, levels=2, lo=0.85)
    iterates = []
    x, st = pr.solve_frame(m.rest, callback=iterates.append)
    assert st.status == S.STATUS_OK
    assert st.grad_norms[-1] <= 1e-8
    assert max(st.contacts) > 0
    E = np.array(st.energies)
    assert (np.diff(E) <= S.LS_SLACK * np.abs(E[:-1])).all()
    for xi in iterates:          # pairs whose boxes are apart are apart
        s = pr.W @ xi
        typ, i, j = C.candidate_pairs(s, pr.tris, pr.edges, m.dhat)
        V = C.pair_vertices(typ, i, j, pr.tris, pr.edges)
        assert D.distance(s[V], typ == 1).min() > 0.0
    assert all(a <= am for a, am in zip(st.alphas, st.alpha_ms))
