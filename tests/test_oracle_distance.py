"""Pins for the oracle's primitive distances and their derivatives (Sec. 2.2).

Checked against brute-force minimisation over the primitives' parameter
domains, closed-form geometric configurations, and finite differences of the
value (gradient) and of the gradient (Hessian) in every closest-feature case.
"""
import numpy as np
import pytest

from oracle import distance as D

rng = np.random.default_rng(99)


def _brute_pt(X, n=301):
    u, v = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n), indexing="ij")
    m = u + v <= 1.0
    u, v = u[m], v[m]
    p, a, b, c = X
    q = a[None] + u[:, None] * (b - a)[None] + v[:, None] * (c - a)[None]
    return np.sqrt(((q - p[None]) ** 2).sum(1)).min()


def _brute_ee(X, n=401):
    s, t = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n), indexing="ij")
    s, t = s.ravel(), t.ravel()
    a0, a1, b0, b1 = X
    pa = a0[None] + s[:, None] * (a1 - a0)[None]
    pb = b0[None] + t[:, None] * (b1 - b0)[None]
    return np.sqrt(((pa - pb) ** 2).sum(1)).min()


def test_point_triangle_matches_brute_force():
    X = rng.normal(size=(60, 4, 3))
    d = D.distance(X, np.zeros(60, bool))
    for k in range(60):
        db = _brute_pt(X[k])
        scale = np.abs(X[k]).max() * 2 / 300
        assert d[k] <= db + 1e-12
        assert db - d[k] <= 2 * scale


def test_edge_edge_matches_brute_force():
    X = rng.normal(size=(60, 4, 3))
    d = D.distance(X, np.ones(60, bool))
    for k in range(60):
        db = _brute_ee(X[k])
        scale = np.abs(X[k]).max() * 2 / 400
        assert d[k] <= db + 1e-12
        assert db - d[k] <= 2 * scale


def test_closed_form_configurations():
    # point above the triangle interior: distance = height
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    X = np.array([np.vstack([[0.2, 0.3, 0.7], tri])])
    assert D.pt_case(X)[0] == D.PT_FACE
    assert np.isclose(D.distance(X, [False])[0], 0.7, rtol=0, atol=1e-15)
    # beyond the hypotenuse: distance to the line x + y = 1 in the plane, plus height
    X = np.array([np.vstack([[1.0, 1.0, 0.5], tri])])
    assert D.pt_case(X)[0] == D.PT_E12
    assert np.isclose(D.distance(X, [False])[0], np.sqrt(0.5 + 0.25))
    # beyond vertex 1
    X = np.array([np.vstack([[2.0, -1.0, 0.0], tri])])
    assert D.pt_case(X)[0] == D.PT_V1
    assert np.isclose(D.distance(X, [False])[0], np.sqrt(2.0))
    # skew perpendicular edges crossing at their midpoints, offset h
    h = 0.37
    X = np.array([[[-1, 0, 0], [1, 0, 0], [0, -1, h], [0, 1, h]]], float)
    assert D.ee_case(X)[0] == D.EE_INT
    assert np.isclose(D.distance(X, [True])[0], h)
    # parallel edges: closest feature on the boundary, exact separation
    X = np.array([[[0, 0, 0], [1, 0, 0], [0.5, 0.2, 0], [1.5, 0.2, 0]]], float)
    assert D.ee_case(X)[0] != D.EE_INT
    assert np.isclose(D.distance(X, [True])[0], 0.2)
    # collinear, disjoint: endpoint to endpoint
    X = np.array([[[0, 0, 0], [1, 0, 0], [1.5, 0, 0], [3, 0, 0]]], float)
    assert D.ee_case(X)[0] == D.EE_A1B0
    assert np.isclose(D.distance(X, [True])[0], 0.5)


def _configs_for_every_case():
    """Generic pairs (random perturbations) that land in every case code."""
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    pts = {D.PT_FACE: [0.2, 0.2, 0.3], D.PT_E01: [0.5, -0.4, 0.3], D.PT_E12: [0.8, 0.8, 0.2],
           D.PT_E20: [-0.4, 0.5, 0.3], D.PT_V0: [-0.4, -0.5, 0.2], D.PT_V1: [1.6, -0.3, 0.2],
           D.PT_V2: [-0.3, 1.6, 0.2]}
    pt = []
    for code, p in pts.items():
        X = np.vstack([p, tri]) + 0.01 * rng.normal(size=(4, 3))
        assert D.pt_case(X[None])[0] == code
        pt.append(X)
    a = np.array([[0, 0, 0], [1, 0, 0]], float)
    ees = {D.EE_INT: [[0.5, -1, 0.3], [0.5, 1, 0.4]],
           D.EE_A0_B: [[-0.3, -1, 0.3], [-0.2, 1, 0.4]],
           D.EE_A1_B: [[1.3, -1, 0.3], [1.2, 1, 0.4]],
           D.EE_B0_A: [[0.5, 0.3, 0.2], [0.6, 1.3, 0.9]],
           D.EE_B1_A: [[0.6, 1.3, 0.9], [0.5, 0.3, 0.2]],
           D.EE_A0B0: [[-0.3, -0.2, 0.2], [-1.0, -1.3, 0.5]],
           D.EE_A0B1: [[-1.0, -1.3, 0.5], [-0.3, -0.2, 0.2]],
           D.EE_A1B0: [[1.3, -0.2, 0.2], [2.0, -1.3, 0.5]],
           D.EE_A1B1: [[2.0, -1.3, 0.5], [1.3, -0.2, 0.2]]}
    ee = []
    for code, b in ees.items():
        X = np.vstack([a, b]) + 0.01 * rng.normal(size=(4, 3))
        assert D.ee_case(X[None])[0] == code, code
        ee.append(X)
    return np.array(pt), np.array(ee)


@pytest.mark.parametrize("kind", ["pt", "ee"])
def test_distance_gradient_and_hessian_match_finite_differences(kind):
    pt, ee = _configs_for_every_case()
    X = pt if kind == "pt" else ee
    is_ee = np.full(X.shape[0], kind == "ee")
    hd = D.distance_hd(X, is_ee)
    assert np.allclose(hd.v, D.distance(X, is_ee), rtol=1e-14, atol=0)
    eps = 1e-6
    for c in range(12):
        Xp, Xm = X.copy(), X.copy()
        Xp[:, c // 3, c % 3] += eps
        Xm[:, c // 3, c % 3] -= eps
        fd_g = (D.distance(Xp, is_ee) - D.distance(Xm, is_ee)) / (2 * eps)
        assert np.allclose(fd_g, hd.g[:, c], atol=1e-8)
        fd_h = (D.distance_hd(Xp, is_ee).g - D.distance_hd(Xm, is_ee).g) / (2 * eps)
        assert np.allclose(fd_h, hd.h[:, :, c], atol=1e-6)
    # Hessians are symmetric
    assert np.allclose(hd.h, np.swapaxes(hd.h, 1, 2), atol=1e-12)


def test_distance_invariant_under_rigid_motion():
    X = rng.normal(size=(50, 4, 3))
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Y = X @ Q.T + rng.normal(size=3)
    for ee in (False, True):
        is_ee = np.full(50, ee)
        assert np.allclose(D.distance(X, is_ee), D.distance(Y, is_ee), rtol=1e-12)


def test_hd_arithmetic_matches_finite_differences():
    X = rng.uniform(1.0, 2.0, size=(5, 4, 3))
    X[:, 1, 1] += 3.0          # keeps b - c > 0 (log domain)
    a = D.Hd.variable(X[:, 0, 0], 0)
    b = D.Hd.variable(X[:, 1, 1], 4)
    c = D.Hd.variable(X[:, 2, 2], 8)
    f = lambda a, b, c: ((a * b + c / a).sqrt() * (b - c)).log() if isinstance(a, D.Hd) else \
        np.log(np.sqrt(a * b + c / a) * (b - c))
    v = f(a, b, c)
    base = np.array([X[:, 0, 0], X[:, 1, 1], X[:, 2, 2]])
    slots = [0, 4, 8]
    eps = 1e-6
    assert np.all(np.isfinite(v.v))
    for k in range(3):
        bp, bm = base.copy(), base.copy()
        bp[k] += eps
        bm[k] -= eps
        fd = (f(*bp) - f(*bm)) / (2 * eps)
        assert np.allclose(fd, v.g[:, slots[k]], atol=1e-7)
