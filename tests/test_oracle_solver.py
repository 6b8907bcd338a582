"""Pins for the oracle's global step (Eq. 4, Eq. 8-9, Eq. 11) and Algorithm 1.

References: the linear-system residual, agreement of three algebraically
equivalent solves (direct sparse LU, the Schur 3-step of Eq. 8, the Woodbury
update of Eq. 11 in printed and push-through forms), independence from the
choice of the collision-aware set, and the solver invariants of IPC (energy
never increases, the proxy never touches, the stop criterion holds).
"""
import numpy as np
import pytest

from oracle import contact as C
from oracle import distance as D
from oracle import solver as S
from paper_2312_02999_gb300 import inputs as I


def _problem(nx=3, nz=2, gap=0.0004, region=None, seed=5):
    m = I.two_slabs(nx, nx, nz, gap=gap)
    a = I.slab_actuation(m, seed=seed)
    p = S.Params(dhat=m.dhat, tol_abs=1e-8)
    pr = S.Problem(m.rest, m.tets, m.pinned, m.proxy_tris, m.W_rowptr, m.W_col,
                   m.W_val, p, region=region)
    pr.set_actuation(a.fiber, a.stretch)
    return m, pr


def _contact_state(m, pr, seed=3):
    rng = np.random.default_rng(seed)
    x = m.rest.copy()
    free = np.nonzero(m.pinned == 0)[0]
    x[free] += 1e-4 * rng.normal(size=(free.size, 3))
    ev = pr.evaluate(x)
    assert ev["C"][0].size > 0
    g = pr.gradient(x, ev).ravel()[pr.free_dofs]
    B = pr.free_part(pr.barrier_hessian(ev))
    return x, ev, g, B


def test_direct_global_step_solves_the_system():
    m, pr = _problem()
    _, _, g, B = _contact_state(m, pr)
    dx = pr.global_step_direct(g, B)
    res = (pr.H + B) @ dx + g
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(g)
    # a descent direction for E-hat
    assert g @ dx < 0


def test_schur_three_step_and_woodbury_equal_direct():
    m, pr = _problem()
    _, _, g, B = _contact_state(m, pr)
    dx = pr.global_step_direct(g, B)
    Hd, Bd = pr.H.toarray(), B.toarray()
    i1, i2 = pr.split_dofs()
    # B vanishes outside the x2 block (the embedding only touches x2)
    assert np.abs(Bd[np.ix_(i1, i1)]).max() == 0 and np.abs(Bd[np.ix_(i1, i2)]).max() == 0
    dx_s = S.schur_three_step(Hd, Bd, g, i1, i2)
    dx_w = S.woodbury_global_step(Hd, Bd, g, i1, i2, push_through=True)
    scale = np.abs(dx).max()
    assert np.abs(dx_s - dx).max() <= 1e-10 * scale
    assert np.abs(dx_w - dx).max() <= 1e-10 * scale


def test_printed_woodbury_equals_push_through_when_invertible():
    m, pr = _problem()
    _, _, g, B = _contact_state(m, pr)
    Hd, Bd = pr.H.toarray(), B.toarray()
    i1, i2 = pr.split_dofs()
    # make B-check invertible on its support by a small SPD shift there
    B22 = Bd[np.ix_(i2, i2)].copy()
    rows = np.unique(np.nonzero(np.abs(B22).sum(1) > 0)[0] // 3)
    c = (3 * rows[:, None] + np.arange(3)).ravel()
    B22[np.ix_(c, c)] += 1e-2 * np.abs(B22).max() * np.eye(c.size)
    Sigma_inv = np.linalg.inv(S.schur_complement(Hd, i1, i2))
    y = np.random.default_rng(0).normal(size=i2.size)
    a = S.woodbury_apply(Sigma_inv, B22, y, push_through=False)
    b = S.woodbury_apply(Sigma_inv, B22, y, push_through=True)
    ref = np.linalg.solve(np.linalg.inv(Sigma_inv) + B22, y)
    assert np.allclose(a, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(b, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_choice_of_collision_aware_set_does_not_change_the_step():
    m, pr = _problem()
    _, _, g, B = _contact_state(m, pr)
    Hd, Bd = pr.H.toarray(), B.toarray()
    i1, i2 = pr.split_dofs()
    dx_a = S.woodbury_global_step(Hd, Bd, g, i1, i2)
    # enlarge x2 with every free vertex adjacent (shares a tet) to the proxy
    region = pr.x2_mask.copy()
    for t in pr.tets:
        if region[t].any():
            region[t] = True
    m2, pr2 = _problem(region=region.astype(np.uint8))
    assert pr2.x2_mask.sum() > pr.x2_mask.sum()
    j1, j2 = pr2.split_dofs()
    dx_b = S.woodbury_global_step(Hd, Bd, g, j1, j2)
    assert np.abs(dx_a - dx_b).max() <= 1e-10 * np.abs(dx_a).max()


def test_algorithm1_invariants_on_tiny_slabs():
    m, pr = _problem(nx=3, nz=2, gap=0.005)
    iterates = []
    x, st = pr.solve_frame(m.rest, callback=iterates.append)
    assert st.status == S.STATUS_OK
    assert st.grad_norms[-1] <= 1e-8
    assert max(st.contacts) > 0                 # contact really happened
    E = np.array(st.energies)
    assert (np.diff(E) <= S.LS_SLACK * np.abs(E[:-1])).all()
    for xi in iterates:                         # the proxy never touches
        s = pr.W @ xi
        typ, i, j = C.candidate_pairs(s, pr.tris, pr.edges, 10.0)
        V = C.pair_vertices(typ, i, j, pr.tris, pr.edges)
        assert D.distance(s[V], typ == 1).min() > 0.0
    # every accepted step obeyed its CCD bound
    assert all(a <= am for a, am in zip(st.alphas, st.alpha_ms))
    # deterministic
    x2, st2 = pr.solve_frame(m.rest)
    assert np.array_equal(x, x2) and st2.iterations == st.iterations


def test_iteration_cap_reports_not_converged():
    m, pr = _problem(nx=2, nz=1, gap=0.005)
    _, st = pr.solve_frame(m.rest, max_iters=1)
    assert st.status == S.STATUS_NOT_CONVERGED and st.iterations == 1


def test_direct_solver_step_is_independent_of_kappa_scaling_of_h():
    # Sec. 4: the direct method does not depend on a preconditioner; its step
    # solves the system exactly for any barrier stiffness
    m, pr = _problem()
    _, _, g, B = _contact_state(m, pr)
    for k in (1.0, 10.0, 100.0):
        dx = pr.global_step_direct(g, k * B)
        res = (pr.H + k * B) @ dx + g
        assert np.linalg.norm(res) <= 1e-11 * np.linalg.norm(g)


def _near_contact_slab(adaptive):
    mesh = I.two_slabs(4, 4, 2, gap=0.004)
    act = I.slab_actuation(mesh, seed=11)
    pr = S.Problem(mesh.rest, mesh.tets, mesh.pinned, mesh.proxy_tris, mesh.W_rowptr, mesh.W_col,
                   mesh.W_val, S.Params(dhat=mesh.dhat, adaptive_kappa=adaptive,
                                        weight_scale=mesh.weight_scale), region=mesh.region)
    pr.set_actuation(act.fiber, act.stretch)
    rng = np.random.default_rng(9)
    x = mesh.rest.copy()
    free = mesh.pinned == 0
    x[free] += 3e-4 * rng.standard_normal((int(free.sum()), 3))
    top = mesh.rest[:, 2] > mesh.rest[:, 2].mean()
    x[top & free, 2] -= 0.0035           # one pair at ~0.003 dhat
    return mesh, pr, x


def test_adaptive_kappa_follows_its_rule():
    # IPC's adaptive stiffness (Sec. 4): kappa doubles at an iterate whose
    # smallest active distance is below 0.1 dhat and below the previous
    # iterate's, never beyond 100 kappa_0, and restarts every frame
    mesh, pr, x0 = _near_contact_slab(True)
    x, st = pr.solve_frame(x0)
    assert st.status == S.STATUS_OK
    expect, prev, kap = 0, np.inf, 1.0
    for d in st.d_mins:
        if d < S.KAPPA_GROW_BELOW * mesh.dhat and d < prev and 2 * kap <= S.KAPPA_MAX_RATIO:
            expect += 1
            kap *= 2
        prev = d
    assert st.kappa_doublings == expect >= 1
    assert pr.kappa == pr.kappa0 * 2 ** expect
    assert min(st.d_mins) > 0.0
    # the next frame starts from kappa_0 again
    x2, st2 = pr.solve_frame(x)
    assert st2.kappa_doublings == 0 and pr.kappa == pr.kappa0
    # without adaptation the same start converges with kappa_0 throughout
    _, pr0, _ = _near_contact_slab(False)
    _, st0 = pr0.solve_frame(x0)
    assert st0.status == S.STATUS_OK and st0.kappa_doublings == 0 and pr0.kappa == pr0.kappa0
