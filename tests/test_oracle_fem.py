"""Pins for the oracle's elastic part (Eq. 1, Eq. 2, local step, Eq. 4 elastic term).

Each check is against something other than the oracle's own formulas:
closed forms, a library routine (scipy.linalg.polar), brute-force search over
rotations, finite differences, and algebraic structure (Kronecker form).
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.spatial.transform import Rotation

from oracle import fem
from oracle import solver as S
from paper_2312_02999_gb300 import inputs as I

rng = np.random.default_rng(1234)


def _rand_M(n, det_sign=1):
    M = rng.normal(size=(n, 3, 3))
    d = np.linalg.det(M)
    flip = np.sign(d) != det_sign
    M[flip, :, 0] *= -1
    return M


def test_rotation_is_special_orthogonal():
    M = rng.normal(size=(200, 3, 3))
    R = fem.closest_rotation(M)
    assert np.allclose(R @ np.swapaxes(R, 1, 2), np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-13)


def test_rotation_matches_scipy_polar_for_positive_det():
    M = _rand_M(50, +1)
    R = fem.closest_rotation(M)
    for k in range(M.shape[0]):
        U, _ = sla.polar(M[k])
        assert np.allclose(R[k], U, atol=1e-12)


def test_polar_property_symmetric_psd_stretch():
    M = _rand_M(100, +1)
    R = fem.closest_rotation(M)
    Sm = np.swapaxes(R, 1, 2) @ M
    assert np.allclose(Sm, np.swapaxes(Sm, 1, 2), atol=1e-12)
    assert (np.linalg.eigvalsh(0.5 * (Sm + np.swapaxes(Sm, 1, 2))) > -1e-12).all()


def test_diagonal_distinct_positive_gives_identity():
    M = np.array([np.diag([3.0, 2.0, 0.5]), np.diag([0.1, 5.0, 1.0])])
    assert np.allclose(fem.closest_rotation(M), np.eye(3), atol=1e-14)


def test_rotation_maximises_trace_against_sampled_rotations():
    # brute force: no sampled rotation beats R for max tr(Q^T M) (incl. det M < 0)
    Qs = Rotation.random(4000, random_state=7).as_matrix()
    for sign in (+1, -1):
        M = _rand_M(5, sign)
        R = fem.closest_rotation(M)
        best = np.einsum("tij,tij->t", R, M)
        for k in range(M.shape[0]):
            tr = np.einsum("qij,ij->q", Qs, M[k])
            assert tr.max() <= best[k] + 1e-12


def test_local_step_minimises_element_energy():
    # ||F - R A|| over rotations: R from the local step beats sampled rotations
    F = rng.normal(size=(4, 3, 3))
    f = rng.normal(size=(4, 3))
    A = fem.actuation_matrices(f, rng.uniform(0.6, 1.0, 4))
    R, P = fem.local_step(F, A)
    Qs = Rotation.random(3000, random_state=3).as_matrix()
    for k in range(4):
        e_best = np.sum((F[k] - P[k]) ** 2)
        e = np.sum((F[k][None] - Qs @ A[k]) ** 2, axis=(1, 2))
        assert e.min() >= e_best - 1e-12


def test_actuation_matrix_properties():
    f = rng.normal(size=(20, 3))
    a = rng.uniform(0.5, 1.5, 20)
    A = fem.actuation_matrices(f, a)
    assert np.allclose(A, np.swapaxes(A, 1, 2))
    assert np.allclose(np.linalg.det(A), 1.0)
    fn = f / np.linalg.norm(f, axis=1, keepdims=True)
    assert np.allclose(np.einsum("tij,tj->ti", A, fn), a[:, None] * fn)
    assert np.allclose(fem.actuation_matrices(f, np.ones(20)), np.eye(3))


def test_deformation_gradient_exact_for_affine_maps():
    m = I.two_slabs(2, 2, 1)
    _, gradN, _ = fem.tet_rest_data(m.rest, m.tets.astype(np.int64), 1.0)
    G = fem.gradient_operators(gradN)
    Maff = rng.normal(size=(3, 3))
    x = m.rest @ Maff.T + rng.normal(size=3)
    F = fem.deformation_gradients(x, m.tets.astype(np.int64), G)
    assert np.allclose(F, Maff[None], atol=1e-12)


def test_tet_volume_weights_sum_to_slab_volume():
    m = I.two_slabs(3, 2, 2, h=0.1)
    _, _, w = fem.tet_rest_data(m.rest, m.tets.astype(np.int64), 1e3)
    assert np.isclose(w.sum(), 1e3 * 2 * (0.3 * 0.2 * 0.2))


def _small_problem(a_range=(0.7, 1.0), gap=0.005, nz=1, nx=2):
    m = I.two_slabs(nx, nx, nz, gap=gap)
    a = I.slab_actuation(m, seed=5, lo=a_range[0], hi=a_range[1])
    p = S.Params(dhat=m.dhat, tol_abs=1e-8)
    pr = S.Problem(m.rest, m.tets, m.pinned, m.proxy_tris, m.W_rowptr, m.W_col, m.W_val, p)
    pr.set_actuation(a.fiber, a.stretch)
    return m, pr


def _elastic_energy(pr, x):
    F = fem.deformation_gradients(x, pr.tets, pr.G)
    _, P = fem.local_step(F, pr.A)
    return fem.elastic_energy(F, P, pr.w)


def test_elastic_gradient_matches_central_differences():
    # envelope theorem: sum w G^T (G x - p(x)) is the exact gradient of E(x)
    m, pr = _small_problem(gap=0.5)
    x = I.perturbed_positions(m, 0.01, seed=11)
    F = fem.deformation_gradients(x, pr.tets, pr.G)
    _, P = fem.local_step(F, pr.A)
    g = fem.elastic_gradient(x, pr.tets, pr.G, P, pr.w).ravel()
    eps = 1e-6
    for k in rng.choice(3 * m.n, size=40, replace=False):
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[k] += eps
        xm[k] -= eps
        fd = (_elastic_energy(pr, xp.reshape(-1, 3)) - _elastic_energy(pr, xm.reshape(-1, 3))) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k]))


def test_pd_matrix_is_hessian_for_fixed_projection():
    # d/dx sum w G^T (G x - p) with p frozen equals H (Eq. 2)
    m, pr = _small_problem(gap=0.5)
    x = I.perturbed_positions(m, 0.01, seed=12)
    F = fem.deformation_gradients(x, pr.tets, pr.G)
    _, P = fem.local_step(F, pr.A)
    H = fem.pd_matrix(m.n, pr.tets, pr.G, pr.w).toarray()
    eps = 1e-6
    for k in rng.choice(3 * m.n, size=10, replace=False):
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[k] += eps
        xm[k] -= eps
        gp = fem.elastic_gradient(xp.reshape(-1, 3), pr.tets, pr.G, P, pr.w).ravel()
        gm = fem.elastic_gradient(xm.reshape(-1, 3), pr.tets, pr.G, P, pr.w).ravel()
        assert np.allclose((gp - gm) / (2 * eps), H[:, k], atol=1e-6)


def test_pd_matrix_has_kronecker_structure():
    m = I.two_slabs(3, 2, 2)
    _, gradN, w = fem.tet_rest_data(m.rest, m.tets.astype(np.int64), 1e3)
    G = fem.gradient_operators(gradN)
    H = fem.pd_matrix(m.n, m.tets.astype(np.int64), G, w).toarray()
    K = fem.scalar_laplacian(m.n, m.tets.astype(np.int64), gradN, w).toarray()
    assert np.allclose(H, np.kron(K, np.eye(3)), atol=1e-10)
    # Laplacian structure: rows sum to zero, symmetric PSD
    assert np.allclose(K.sum(axis=1), 0.0, atol=1e-9)
    assert np.allclose(K, K.T)


def test_rest_pose_without_actuation_is_an_exact_equilibrium():
    m, pr = _small_problem(a_range=(1.0, 1.0))
    # F = Dm Dm^-1 and the SVD are exact up to rounding only
    ev = pr.evaluate(m.rest.copy())
    assert ev["E"] < 1e-28
    g = pr.gradient(m.rest.copy(), ev)
    assert np.abs(g).max() < 1e-12
    x, st = pr.solve_frame(m.rest)
    assert st.status == S.STATUS_OK and st.iterations == 0
    assert np.array_equal(x, m.rest)


def test_pd_fixed_point_without_contact():
    # gap >> dhat: C stays empty and the result solves H x = sum w G^T p(x) (Eq. 2)
    m, pr = _small_problem(gap=0.5, nz=1, nx=2)
    x, st = pr.solve_frame(m.rest)
    assert st.status == S.STATUS_OK
    assert max(st.contacts) == 0
    F = fem.deformation_gradients(x, pr.tets, pr.G)
    _, P = fem.local_step(F, pr.A)
    idx = (3 * pr.tets[:, :, None] + np.arange(3)).reshape(-1, 12)
    rhs = np.zeros(3 * m.n)
    np.add.at(rhs, idx.ravel(),
              (pr.w[:, None] * np.einsum("tji,tj->ti", pr.G, P.reshape(-1, 9))).ravel())
    Hfull = fem.pd_matrix(m.n, pr.tets, pr.G, pr.w)
    res = (Hfull @ x.ravel() - rhs)[pr.free_dofs]
    assert np.linalg.norm(res) <= 1e-8
