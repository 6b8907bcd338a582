"""Pins for the oracle's optional edge-edge mollifier (IPC's treatment of
nearly parallel edges; the paper builds on IPC, Sec. 2.2).

References used: the closed form of m(c) and its C^1 join at eps, Lagrange's
identity for c = |e_a x e_b|^2, central finite differences of the mollifier
and of the mollified pair term kappa m(c) b(d), the exact vanishing of the
term and its gradient for parallel edges, the unmollified term beyond eps,
and IPC's solver invariants on slabs whose facing edges are parallel.
"""
import numpy as np

from oracle import contact as C
from oracle import distance as D
from oracle import solver as S
from paper_2312_02999_gb300 import inputs as I

rng = np.random.default_rng(23)
NT = np.zeros((0, 3), dtype=np.int64)     # no triangles: the pairs below are all EE


def test_mollifier_closed_form_and_c1_join():
    eps = np.full(5, 2.0)
    c = np.array([0.0, 0.5, 1.0, 2.0, 3.0])
    m = C.mollifier(c, eps)
    assert np.allclose(m, [0.0, 0.4375, 0.75, 1.0, 1.0], rtol=0, atol=1e-15)
    # value and slope join at c = eps: m(eps - h) = 1 - (h/eps)^2
    h = 1e-4
    assert abs(C.mollifier(np.array([2.0 - h]), np.array([2.0]))[0] - (1 - (h / 2) ** 2)) < 1e-15
    grid = np.linspace(0.0, 2.0, 101)
    assert (np.diff(C.mollifier(grid, np.full(101, 2.0))) > 0).all()


def _near_parallel_pairs(n, dist=3e-4, tilt=1e-3):
    """EE pairs (a0, a1, b0, b1): edge b is edge a tilted by ~tilt radians and
    lifted by ~dist, so c is far below eps at unit-length rest edges."""
    X = np.zeros((n, 4, 3))
    for k in range(n):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        p = rng.normal(size=3) * 0.1
        nrm = np.cross(u, rng.normal(size=3))
        nrm /= np.linalg.norm(nrm)
        v = u + tilt * np.cross(u, nrm) * rng.uniform(0.3, 1.0)
        v /= np.linalg.norm(v)
        X[k, 0], X[k, 1] = p - 0.5 * u, p + 0.5 * u
        off = p + dist * rng.uniform(0.5, 1.0) * nrm + 0.2 * u * rng.uniform(-1, 1)
        X[k, 2], X[k, 3] = off - 0.5 * v, off + 0.5 * v
    return X


def test_cross_product_square_and_mollifier_derivatives():
    X = _near_parallel_pairs(6)
    ea, eb = X[:, 1] - X[:, 0], X[:, 3] - X[:, 2]
    lag = (ea * ea).sum(1) * (eb * eb).sum(1) - (ea * eb).sum(1) ** 2
    c = C.edge_cross_sq(X)
    assert np.allclose(c, lag, rtol=1e-9, atol=1e-22)
    eps = np.full(6, 1e-3)
    assert (c < eps).all()
    m = C.mollifier_hd(X, eps)
    assert np.allclose(m.v, C.mollifier(c, eps), rtol=1e-13)
    h = 1e-7
    for k in range(12):
        Xp, Xm = X.copy(), X.copy()
        Xp[:, k // 3, k % 3] += h
        Xm[:, k // 3, k % 3] -= h
        fd = (C.mollifier(C.edge_cross_sq(Xp), eps) - C.mollifier(C.edge_cross_sq(Xm), eps)) / (2 * h)
        assert np.allclose(m.g[:, k], fd, rtol=1e-5, atol=1e-7)
        mp, mm = C.mollifier_hd(Xp, eps), C.mollifier_hd(Xm, eps)
        assert np.allclose(m.h[:, :, k], (mp.g - mm.g) / (2 * h), rtol=1e-4, atol=1e-6)


def _pair_setup(X):
    """Proxy arrays for P independent EE pairs: s, edges, (typ, i, j)."""
    P = X.shape[0]
    s = X.reshape(-1, 3).copy()
    edges = np.arange(4 * P).reshape(-1, 2)
    typ = np.ones(P, dtype=np.int64)
    i, j = 2 * np.arange(P), 2 * np.arange(P) + 1
    return s, edges, typ, i, j


def test_mollified_pair_term_matches_finite_differences():
    X = _near_parallel_pairs(5, dist=3e-4, tilt=2e-3)
    s, edges, typ, i, j = _pair_setup(X)
    s_rest = s.copy()                      # eps = 1e-3 at unit rest edges
    dhat, kappa = 1e-3, 7.0
    V, g, h = C.pair_barrier_derivatives(s, typ, i, j, NT, edges, dhat, kappa, project=False,
                                         s_rest=s_rest)
    c = C.edge_cross_sq(s[V])
    assert (c < C.ee_mollifier_eps(s_rest, edges, i, j)).all()

    def term(ss):
        d = D.distance(ss[V], typ == 1)
        return kappa * C.pair_barrier_values(ss, typ, i, j, d, NT, edges, dhat, s_rest)

    # the line-line distance of nearly parallel edges loses digits to
    # cancellation, so the differences use a step of 1e-7 (error ~ step^2)
    step = 1e-7
    for k in range(12):
        sp_, sm_ = s.copy(), s.copy()
        sp_[V[:, k // 3], k % 3] += step
        sm_[V[:, k // 3], k % 3] -= step
        fd = (term(sp_) - term(sm_)) / (2 * step)
        assert (np.abs(fd - g[:, k]) <= 1e-6 * np.abs(g).max(axis=1)).all()
    # Hessian columns by differencing the analytic gradient
    for k in (0, 4, 11):
        sp_, sm_ = s.copy(), s.copy()
        for p in range(X.shape[0]):
            sp_[V[p, k // 3], k % 3] += step
            sm_[V[p, k // 3], k % 3] -= step
        _, gp, _ = C.pair_barrier_derivatives(sp_, typ, i, j, NT, edges, dhat, kappa, False, s_rest)
        _, gm, _ = C.pair_barrier_derivatives(sm_, typ, i, j, NT, edges, dhat, kappa, False, s_rest)
        col = (gp - gm) / (2 * step)
        assert np.allclose(col, h[:, :, k], rtol=1e-4, atol=1e-4 * np.abs(h).max())


def test_parallel_edges_have_no_term_and_no_gradient():
    X = _near_parallel_pairs(4, dist=4e-4, tilt=0.0)
    s, edges, typ, i, j = _pair_setup(X)
    assert np.allclose(C.edge_cross_sq(s.reshape(-1, 4, 3)), 0.0, atol=1e-30)
    d = D.distance(X, np.ones(4, bool))
    assert (d < 1e-3).all()
    vals = C.pair_barrier_values(s, typ, i, j, d, NT, edges, 1e-3, s.copy())
    assert np.abs(vals).max() <= 1e-25
    _, g, _ = C.pair_barrier_derivatives(s, typ, i, j, NT, edges, 1e-3, 1.0, project=False,
                                         s_rest=s.copy())
    unm = C.pair_barrier_derivatives(s, typ, i, j, NT, edges, 1e-3, 1.0, project=False)[1]
    assert np.abs(g).max() <= 1e-12 * np.abs(unm).max()


def test_wide_angles_are_not_mollified():
    X = _near_parallel_pairs(4, dist=3e-4, tilt=0.3)
    s, edges, typ, i, j = _pair_setup(X)
    assert (C.edge_cross_sq(X) > C.ee_mollifier_eps(s, edges, i, j)).all()
    a = C.pair_barrier_derivatives(s, typ, i, j, NT, edges, 1e-3, 3.0, True, s.copy())
    b = C.pair_barrier_derivatives(s, typ, i, j, NT, edges, 1e-3, 3.0, True)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_algorithm1_invariants_with_the_mollifier():
    # the facing faces of the slabs carry exactly parallel grid edges, so
    # many active EE pairs sit at c = 0 (m = 0) and near it
    m = I.two_slabs(3, 3, 2)
    a = I.slab_actuation(m, seed=5)
    pr = S.Problem(m.rest, m.tets, m.pinned, m.proxy_tris, m.W_rowptr, m.W_col, m.W_val,
                   S.Params(dhat=m.dhat, tol_abs=1e-8, ee_mollifier=True))
    pr.set_actuation(a.fiber, a.stretch)
    iterates = []
    x, st = pr.solve_frame(m.rest, callback=iterates.append)
    assert st.status == S.STATUS_OK and st.grad_norms[-1] <= 1e-8
    ev = pr.evaluate(x)
    typ, i, j, d = ev["C"]
    ee = typ == 1
    V = C.pair_vertices(typ[ee], i[ee], j[ee], pr.tris, pr.edges)
    cm = C.edge_cross_sq(ev["s"][V]) < C.ee_mollifier_eps(pr.s_rest, pr.edges, i[ee], j[ee])
    assert cm.sum() > 0                          # mollified pairs are active at the solution
    E = np.array(st.energies)
    assert (np.diff(E) <= S.LS_SLACK * np.abs(E[:-1])).all()
    for xi in iterates:
        s = pr.W @ xi
        t2, i2, j2 = C.candidate_pairs(s, pr.tris, pr.edges, m.dhat)
        V2 = C.pair_vertices(t2, i2, j2, pr.tris, pr.edges)
        assert D.distance(s[V2], t2 == 1).min() > 0.0
