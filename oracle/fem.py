"""Oracle: shape-targeting elastic energy and the PD local/global quantities.

Paper passages followed (Sec. 2.1):
* Eq. 1  -- E_i(x) = min_{R in SO(3)} ||F_i(x) - R_i A_i||_F^2 = ||G_i x - p_i||^2,
            A_i symmetric actuation, G_i the (9 x 12) map x -> vec(F_i),
            p_i = vec(R_i A_i).
* local step -- R_i is the rotation of the polar decomposition of F_i A_i.
* Eq. 2  -- H = sum_i w_i G_i^T G_i, w_i the rest volume (scaled).
* Eq. 4  -- elastic part of the gradient: sum_i w_i G_i^T (G_i x - p_i).

Readings: the energy carries a factor 1/2 (E = 1/2 sum w ||F - RA||^2) so
that Eq. 2 and Eq. 4 are its exact Hessian (in the PD sense) and gradient;
the actuation matrix is A = a f f^T + a^(-1/2) (I - f f^T) (volume
preserving, A = I at a = 1); w_i = weight_scale * rest volume.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def tet_rest_data(rest: np.ndarray, tets: np.ndarray, weight_scale: float):
    """Rest-shape data per tet: Dm^-1 (T,3,3), shape gradients (T,4,3), w (T,).

    Dm = [X1-X0, X2-X0, X3-X0] (columns); F = Ds Dm^-1, so the gradient of
    the linear shape function of vertex a (a = 1..3) is row a-1 of Dm^-1 and
    that of vertex 0 is minus their sum.  w = weight_scale * |det Dm| / 6.
    """
    X = rest[tets]
    Dm = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    vol = np.abs(np.linalg.det(Dm)) / 6.0
    Dm_inv = np.linalg.inv(Dm)
    gradN = np.empty((tets.shape[0], 4, 3))
    gradN[:, 1:, :] = Dm_inv
    gradN[:, 0, :] = -Dm_inv.sum(axis=1)
    return Dm_inv, gradN, weight_scale * vol


def actuation_matrices(fiber: np.ndarray, stretch: np.ndarray) -> np.ndarray:
    """A = a f f^T + a^(-1/2) (I - f f^T), symmetric with det A = 1."""
    f = fiber / np.linalg.norm(fiber, axis=1, keepdims=True)
    ff = f[:, :, None] * f[:, None, :]
    a = stretch[:, None, None]
    return a * ff + (1.0 / np.sqrt(a)) * (np.eye(3)[None] - ff)


def gradient_operators(gradN: np.ndarray) -> np.ndarray:
    """G_i (T, 9, 12): vec(F)[3d+j] = sum_a x_a[d] gradN_a[j]  (row-major vec)."""
    T = gradN.shape[0]
    G = np.zeros((T, 9, 12))
    for d in range(3):
        for j in range(3):
            for a in range(4):
                G[:, 3 * d + j, 3 * a + d] = gradN[:, a, j]
    return G


def deformation_gradients(x: np.ndarray, tets: np.ndarray, G: np.ndarray) -> np.ndarray:
    """F_i (T,3,3) from G_i applied to the stacked tet vertex positions."""
    xl = x[tets].reshape(-1, 12)
    return np.einsum("tij,tj->ti", G, xl).reshape(-1, 3, 3)


def closest_rotation(M: np.ndarray) -> np.ndarray:
    """Rotation factor of the polar decomposition of each 3x3 M (via SVD).

    With M = U diag(s) V^T (s descending), R = U diag(1, 1, sigma) V^T with
    sigma = sign det(U V^T): the maximiser of tr(R^T M) over SO(3).
    """
    U, _, Vt = np.linalg.svd(M)
    sig = np.where(np.linalg.det(U) * np.linalg.det(Vt) >= 0.0, 1.0, -1.0)
    D = np.ones((M.shape[0], 3))
    D[:, 2] = sig
    return np.einsum("tij,tj,tjk->tik", U, D, Vt)


def local_step(F: np.ndarray, A: np.ndarray):
    """GetProjection of Algorithm 1: R_i = polar(F_i A_i), p_i = vec(R_i A_i).

    Since A_i is symmetric, argmin_R ||F - R A||_F = argmax_R tr(R^T F A),
    i.e. the polar rotation of F A (Sec. 2.1, local step).
    """
    R = closest_rotation(F @ A)
    P = R @ A
    return R, P


def elastic_energy(F: np.ndarray, P: np.ndarray, w: np.ndarray) -> float:
    """E = 1/2 sum_i w_i ||F_i - R_i A_i||_F^2 (Eq. 1 with the 1/2 reading)."""
    D = F - P
    return 0.5 * float(np.sum(w * np.einsum("tij,tij->t", D, D)))


def elastic_gradient(x: np.ndarray, tets: np.ndarray, G: np.ndarray,
                     P: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_i w_i G_i^T (G_i x - p_i), scattered to vertices -> (n, 3)."""
    xl = x[tets].reshape(-1, 12)
    r = np.einsum("tij,tj->ti", G, xl) - P.reshape(-1, 9)
    gl = w[:, None] * np.einsum("tji,tj->ti", G, r)
    g = np.zeros(x.shape[0] * 3)
    idx = (3 * tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
    np.add.at(g, idx.ravel(), gl.ravel())
    return g.reshape(-1, 3)


def pd_matrix(n: int, tets: np.ndarray, G: np.ndarray, w: np.ndarray) -> sp.csr_matrix:
    """H = sum_i w_i G_i^T G_i over all 3n DOFs (Eq. 2), literal 12x12 blocks."""
    blocks = w[:, None, None] * np.einsum("tki,tkj->tij", G, G)
    idx = (3 * tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
    rows = np.repeat(idx, 12, axis=1).ravel()
    cols = np.tile(idx, (1, 12)).ravel()
    return sp.csr_matrix((blocks.ravel(), (rows, cols)), shape=(3 * n, 3 * n))


def scalar_laplacian(n: int, tets: np.ndarray, gradN: np.ndarray, w: np.ndarray) -> sp.csr_matrix:
    """K_ab = sum_i w_i gradN_a . gradN_b (n x n); Eq. 2 claims H = K (x) I_3."""
    blocks = w[:, None, None] * np.einsum("tad,tbd->tab", gradN, gradN)
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    return sp.csr_matrix((blocks.ravel(), (rows, cols)), shape=(n, n))
