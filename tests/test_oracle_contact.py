"""Pins for the oracle's barrier, constraint set, PSD projection and CCD.

References used: closed-form barrier values and derivatives, an all-pairs
distance sweep with no box pre-filter, finite differences of the barrier
energy through the embedding W, eigen-decomposition identities, and dense
time sampling of the swept motion for the CCD bound.
"""
import numpy as np

from oracle import contact as C
from oracle import distance as D
from oracle import solver as S
from paper_2312_02999_gb300 import inputs as I

rng = np.random.default_rng(5)


def test_barrier_closed_form_and_limits():
    dhat = 1e-3
    d = np.array([0.25e-3, 0.5e-3, 0.999e-3, 1e-3, 2e-3])
    b = C.barrier(d, dhat)
    ref = -((d - dhat) ** 2) * np.log(d / dhat)
    assert np.allclose(b[:3], ref[:3], rtol=1e-15)
    assert b[3] == 0.0 and b[4] == 0.0
    assert (b[:3] > 0).all()
    assert C.barrier(np.array([1e-300]), dhat)[0] > C.barrier(np.array([1e-9]), dhat)[0] > 0


def test_barrier_derivatives_through_hd_match_closed_forms():
    dhat = 1e-3
    d = np.linspace(0.05e-3, 0.95e-3, 11)
    hd = D.Hd(d.copy(), np.ones((11, 1)), np.zeros((11, 1, 1)))
    b = C.barrier_hd(hd, dhat)
    u, L = d - dhat, np.log(d / dhat)
    b1 = -2 * u * L - u * u / d
    b2 = -2 * L - 4 * u / d + u * u / (d * d)
    assert np.allclose(b.g[:, 0], b1, rtol=1e-12)
    assert np.allclose(b.h[:, 0, 0], b2, rtol=1e-12)
    # C^1 at dhat: value and slope vanish (finite differences from below)
    eps = 1e-9
    assert abs(C.barrier(np.array([dhat - eps]), dhat)[0]) < 1e-20


def _slab_mesh(gap=0.0004, nx=3, nz=1):
    return I.two_slabs(nx, nx, nz, gap=gap)


def test_constraint_set_equals_unfiltered_all_pairs_sweep():
    m = _slab_mesh()
    s = m.rest[m.W_col] + 0.0002 * rng.normal(size=(m.Ns, 3))
    edges = C.proxy_edges(m.proxy_tris.astype(np.int64))
    tris = m.proxy_tris.astype(np.int64)
    typ, i, j, d = C.constraint_set(s, tris, edges, m.dhat)
    # reference: every PT and EE pair, no box test
    Ns = s.shape[0]
    vi, tj = np.meshgrid(np.arange(Ns), np.arange(tris.shape[0]), indexing="ij")
    vi, tj = vi.ravel(), tj.ravel()
    ok = ~(tris[tj] == vi[:, None]).any(1)
    vi, tj = vi[ok], tj[ok]
    ea, eb = np.triu_indices(edges.shape[0], 1)
    ok = ~(edges[ea][:, :, None] == edges[eb][:, None, :]).any((1, 2))
    ea, eb = ea[ok], eb[ok]
    T = np.concatenate([np.zeros(vi.size, int), np.ones(ea.size, int)])
    A = np.concatenate([vi, ea])
    B = np.concatenate([tj, eb])
    V = C.pair_vertices(T, A, B, tris, edges)
    dd = D.distance(s[V], T == 1)
    m_ = dd < m.dhat
    ref = sorted(zip(T[m_], A[m_], B[m_]))
    assert ref == list(zip(typ, i, j))
    assert len(ref) > 0


def test_constraint_set_empty_when_separated_and_rigid_invariant():
    m = _slab_mesh(gap=0.0004)
    tris = m.proxy_tris.astype(np.int64)
    edges = C.proxy_edges(tris)
    s = m.rest[m.W_col].copy()
    mid = s[:, 2].min() + 0.0002
    s_sep = s.copy()
    s_sep[s[:, 2] > mid, 2] += 2 * m.dhat
    assert C.constraint_set(s_sep, tris, edges, m.dhat)[0].size == 0
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    s2 = s @ Q.T + np.array([0.3, -0.2, 0.1])
    a = C.constraint_set(s, tris, edges, m.dhat)
    b = C.constraint_set(s2, tris, edges, m.dhat)
    assert list(zip(*a[:3])) == list(zip(*b[:3]))
    # facing grids at gap 0.4 dhat: only cross-slab pairs are active
    V = C.pair_vertices(a[0], a[1], a[2], tris, edges)
    z = s[V, 2]
    assert ((z.min(1) < mid) & (z.max(1) > mid)).all()


def test_psd_projection_identities():
    M = rng.normal(size=(30, 12, 12))
    M = M + np.swapaxes(M, 1, 2)
    P = C.psd_project(M)
    assert (np.linalg.eigvalsh(P) > -1e-10).all()
    assert np.allclose(C.psd_project(P), P, atol=1e-10)          # idempotent
    Q = rng.normal(size=(30, 12, 12))
    Spsd = Q @ np.swapaxes(Q, 1, 2)
    assert np.allclose(C.psd_project(Spsd), Spsd, atol=1e-10)    # identity on PSD
    # distance to the cone: P - M is NSD and orthogonal to P (Moreau decomposition)
    N = P - M
    assert (np.linalg.eigvalsh(N) > -1e-10).all()
    assert np.allclose(np.einsum("pij,pij->p", P, M - P), 0.0, atol=1e-8)


def test_barrier_gradient_through_embedding_matches_finite_differences():
    m = _slab_mesh(gap=0.0004, nx=2)
    p = S.Params(dhat=m.dhat)
    pr = S.Problem(m.rest, m.tets, m.pinned, m.proxy_tris, m.W_rowptr, m.W_col, m.W_val, p)
    act = I.slab_actuation(m, lo=1.0, hi=1.0)
    pr.set_actuation(act.fiber, act.stretch)
    x = m.rest.copy()
    free = np.nonzero(m.pinned == 0)[0]
    x[free] += 5e-5 * rng.normal(size=(free.size, 3))
    ev = pr.evaluate(x)
    typ = ev["C"][0]
    assert typ.size > 0
    V, gp, hp = pr._pair_terms(ev, project=False)
    gs = np.zeros((pr.W.shape[0], 3))
    np.add.at(gs, V.ravel(), gp.reshape(-1, 3))
    gB = (pr.W.T @ gs).ravel()
    HB = pr.barrier_hessian(ev, project=False).toarray()

    def Bx(xx):
        return C.barrier_energy(pr.W @ xx, pr.tris, pr.edges, m.dhat, pr.kappa)

    eps = 1e-9
    touched = np.nonzero(np.abs(gB) > 0)[0]
    for k in rng.choice(touched, size=min(12, touched.size), replace=False):
        xp, xm = x.ravel().copy(), x.ravel().copy()
        xp[k] += eps
        xm[k] -= eps
        fd = (Bx(xp.reshape(-1, 3)) - Bx(xm.reshape(-1, 3))) / (2 * eps)
        assert abs(fd - gB[k]) <= 1e-5 * max(1.0, abs(gB[k]))
    # Hessian column by differencing the mapped gradient (constraint set frozen)
    k = touched[0]
    xp, xm = x.ravel().copy(), x.ravel().copy()
    xp[k] += 1e-10
    xm[k] -= 1e-10

    def mapped_grad(xx):
        ss = pr.W @ xx.reshape(-1, 3)
        Vv, g2, _ = C.pair_barrier_derivatives(ss, *ev["C"][:3], pr.tris, pr.edges,
                                               m.dhat, pr.kappa, project=False)
        out = np.zeros((pr.W.shape[0], 3))
        np.add.at(out, Vv.ravel(), g2.reshape(-1, 3))
        return (pr.W.T @ out).ravel()

    col = (mapped_grad(xp) - mapped_grad(xm)) / 2e-10
    assert np.allclose(col, HB[:, k], rtol=1e-4, atol=1e-4 * np.abs(HB[:, k]).max())


def _accd_cases(n=80, approach=True):
    X = rng.normal(size=(n, 4, 3)) * 0.1
    dX = rng.normal(size=(n, 4, 3)) * 0.1
    if approach:  # drive the first vertex group toward the second
        dX[:, 0] += (X[:, 2] - X[:, 0]) * 1.5
    return X, dX


def test_accd_is_conservative_under_dense_sampling():
    for ee in (False, True):
        X, dX = _accd_cases()
        is_ee = np.full(X.shape[0], ee)
        toi = C.accd_toi(X, dX, is_ee)
        d0 = D.distance(X, is_ee)
        taus = np.linspace(0.0, 1.0, 801)
        for k in range(X.shape[0]):
            ts = taus[taus <= toi[k]]
            Y = X[k][None] + ts[:, None, None] * dX[k][None]
            dk = D.distance(Y, np.full(ts.size, ee))
            assert (dk > 0).all()
            # at the returned time the pair keeps at least s * d(0)
            dt = D.distance((X[k] + toi[k] * dX[k])[None], [ee])[0]
            assert dt >= 0.1 * d0[k] * (1 - 1e-9)
        # some pairs really are stopped early
        assert (toi < 1.0).any()


def test_accd_pure_translation_and_separation_give_full_step():
    X, _ = _accd_cases(20, approach=False)
    dX = np.repeat(rng.normal(size=(20, 1, 3)), 4, axis=1)     # rigid translation
    assert (C.accd_toi(X, dX, np.zeros(20, bool)) == 1.0).all()
    dX = np.zeros_like(X)
    dX[:, 0] = -(X[:, 2] - X[:, 0])                            # move apart (short)
    dX[:, 0] *= 0.01
    assert (C.accd_toi(X, dX, np.ones(20, bool)) == 1.0).all()


def test_ccd_step_bound_prevents_interpenetration():
    m = _slab_mesh(gap=0.0004, nx=3)
    tris = m.proxy_tris.astype(np.int64)
    edges = C.proxy_edges(tris)
    s = m.rest[m.W_col].copy()
    ds = np.zeros_like(s)
    top = s[:, 2] > s[:, 2].min() + 0.0002
    ds[top, 2] = -0.003 + 1e-4 * rng.normal(size=int(top.sum()))   # would cross
    ds[top, :2] = 1e-4 * rng.normal(size=(int(top.sum()), 2))
    a = C.ccd_step_bound(s, ds, tris, edges, m.dhat)
    assert 0.0 < a < 1.0
    for tau in np.linspace(0.0, a, 41):
        st = s + tau * ds
        typ, i, j = C.candidate_pairs(st, tris, edges, 10.0)
        V = C.pair_vertices(typ, i, j, tris, edges)
        assert D.distance(st[V], typ == 1).min() > 0.0
