"""Oracle: global step of Eq. 4 and the outer loop of Algorithm 1.

Paper passages followed:
* Eq. 4 -- (H + B(x)) dx = -(sum_i w_i G_i^T (G_i x - p_i) + grad B(x)),
  with B(x) the (PSD-projected) barrier Hessian.  The oracle assembles the
  full sparse H-hat over the free DOFs and factors it directly (SuperLU)
  at every iteration: no prefactorisation, no reduction.
* Eq. 8-9 (Sec. 3.1) -- Schur-complement form: with x = [x1; x2] (x2 the
  collision-aware vertices), H11 = L1 L1^T, Sigma-hat = H22-hat - H21 H11^-1
  H12, and the 3-step solve (lower, diagonal, upper).  Dense; for pins.
* Eq. 10-11 (Sec. 3.2) -- low-rank update of Sigma^-1 on the n_c vertices
  touched by the barrier.  Dense; for pins.  The paper inverts B-check; the
  push-through form (I + B S)^-1 B with S = Q Sigma^-1 Q^T equals it whenever
  B-check is invertible and stays defined when it is singular (reading).
* Algorithm 1 -- projection, constraint set, PSD Hessian, gradient, solve,
  CCD, line search, update, until the gradient norm is below tolerance.

Readings: Dirichlet vertices keep their rest positions (all three DOFs are
eliminated); the update uses the current iterate (x <- x + alpha dx; the
listing's x_t there is taken as a typo); backtracking halves alpha from
alpha_m and accepts when E-hat does not increase (beyond a relative slack of
LS_SLACK, i.e. within FP64 rounding of the energy sums), at most MAX_LS
halvings; convergence when ||g_free||_2 <= max(tol_abs, tol_rel ||g(x_t)||);
kappa defaults to the mean diagonal entry of H over the free DOFs.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import contact as C
from . import fem

LS_SLACK = 1e-12

STATUS_OK = 0
STATUS_NOT_CONVERGED = -5
STATUS_LS_FAIL = -6


@dataclass
class Params:
    dhat: float
    kappa: float | None = None      # None: mean diag(H) over free DOFs
    tol_abs: float = 1e-8
    tol_rel: float = 0.0
    max_iters: int = 500
    max_ls: int = 40
    ccd_s: float = 0.1
    weight_scale: float = 1e3
    # IPC's adaptive stiffness, as the paper uses it (Sec. 4: kappa is
    # initialised from the soft body's average stiffness and adapted): each
    # iteration of a frame doubles kappa when the smallest active distance is
    # below KAPPA_GROW_BELOW * dhat and smaller than at the previous iterate,
    # up to KAPPA_MAX_RATIO times its initial value; every frame starts from
    # the initial value
    adaptive_kappa: bool = False
    # IPC's edge-edge mollifier (contact.mollifier): EE terms become
    # kappa m(c) b(d) with eps from the rest proxy (off: plain b(d))
    ee_mollifier: bool = False


KAPPA_GROW_BELOW = 0.1
KAPPA_MAX_RATIO = 100.0


@dataclass
class FrameStats:
    status: int = STATUS_OK
    iterations: int = 0
    kappa_doublings: int = 0
    d_mins: list = field(default_factory=list)       # smallest active distance per iterate
    grad_norms: list = field(default_factory=list)
    energies: list = field(default_factory=list)
    alphas: list = field(default_factory=list)
    alpha_ms: list = field(default_factory=list)
    contacts: list = field(default_factory=list)
    n_c: list = field(default_factory=list)
    ls_halvings: list = field(default_factory=list)


class Problem:
    """One mesh with its collision proxy, ready for frame solves."""

    def __init__(self, rest, tets, pinned, proxy_tris, W_rowptr, W_col, W_val,
                 params: Params, region=None):
        self.rest = np.asarray(rest, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.n = self.rest.shape[0]
        self.pinned = np.asarray(pinned).astype(bool)
        self.tris = np.asarray(proxy_tris, dtype=np.int64)
        Ns = len(W_rowptr) - 1
        self.W = sp.csr_matrix((np.asarray(W_val, float), np.asarray(W_col, np.int64),
                                np.asarray(W_rowptr, np.int64)), shape=(Ns, self.n))
        self.edges = C.proxy_edges(self.tris)
        self.p = params
        self.Dm_inv, self.gradN, self.w = fem.tet_rest_data(self.rest, self.tets,
                                                            params.weight_scale)
        self.G = fem.gradient_operators(self.gradN)
        self.free = np.nonzero(~self.pinned)[0]
        self.free_dofs = (3 * self.free[:, None] + np.arange(3)).ravel()
        H_all = fem.pd_matrix(self.n, self.tets, self.G, self.w)
        self.H = H_all[self.free_dofs][:, self.free_dofs].tocsr()
        self.kappa = (float(self.H.diagonal().mean()) if params.kappa is None
                      else float(params.kappa))
        self.kappa0 = self.kappa
        # collision-aware set x2 (Sec. 3.1: x2 embeds s): the free support of
        # W, plus the marked region when one is given
        x2 = np.zeros(self.n, dtype=bool)
        x2[np.unique(self.W.indices)] = True
        if region is not None:
            x2 |= np.asarray(region).astype(bool)
        x2 &= ~self.pinned
        self.x2_mask = x2
        self.s_rest = (self.W @ self.rest) if params.ee_mollifier else None
        self.A = None

    # -- actuation ---------------------------------------------------------
    def set_actuation(self, fiber, stretch):
        self.A = fem.actuation_matrices(np.asarray(fiber, float), np.asarray(stretch, float))

    # -- evaluation at a configuration ---------------------------------------
    def proxy(self, x):
        return self.W @ x

    def evaluate(self, x):
        """Local step + constraint set + energies at x (one call of each)."""
        F = fem.deformation_gradients(x, self.tets, self.G)
        R, P = fem.local_step(F, self.A)
        E = fem.elastic_energy(F, P, self.w)
        s = self.proxy(x)
        typ, i, j, d = C.constraint_set(s, self.tris, self.edges, self.p.dhat)
        B = float(self.kappa * C.pair_barrier_values(s, typ, i, j, d, self.tris, self.edges,
                                                     self.p.dhat, self.s_rest).sum())
        return {"F": F, "R": R, "P": P, "E": E, "s": s, "C": (typ, i, j, d), "B": B}

    def energy(self, x):
        ev = self.evaluate(x)
        return ev["E"] + ev["B"]

    def _pair_terms(self, ev, project=True):
        typ, i, j, _ = ev["C"]
        return C.pair_barrier_derivatives(ev["s"], typ, i, j, self.tris, self.edges,
                                          self.p.dhat, self.kappa, project=project,
                                          s_rest=self.s_rest)

    def gradient(self, x, ev):
        """g-hat over all vertices (n,3): elastic term + W^T grad B(s)."""
        g = fem.elastic_gradient(x, self.tets, self.G, ev["P"], self.w)
        V, gp, _ = self._pair_terms(ev, project=False)
        if V.shape[0]:
            gs = np.zeros((self.W.shape[0], 3))
            np.add.at(gs, V.ravel(), gp.reshape(-1, 3))
            g = g + self.W.T @ gs
        return g

    def barrier_hessian(self, ev, project=True) -> sp.csr_matrix:
        """W^T PositiveDefinite(hess B(s)) W over all 3n DOFs."""
        V, _, hp = self._pair_terms(ev, project=project)
        Ns3 = 3 * self.W.shape[0]
        if V.shape[0] == 0:
            return sp.csr_matrix((3 * self.n, 3 * self.n))
        idx = (3 * V[:, :, None] + np.arange(3)).reshape(-1, 12)
        rows = np.repeat(idx, 12, axis=1).ravel()
        cols = np.tile(idx, (1, 12)).ravel()
        Hs = sp.csr_matrix((hp.ravel(), (rows, cols)), shape=(Ns3, Ns3))
        W3 = sp.kron(self.W, sp.identity(3), format="csr")
        return (W3.T @ Hs @ W3).tocsr()

    def free_part(self, M):
        return M[self.free_dofs][:, self.free_dofs].tocsr()

    # -- global steps --------------------------------------------------------
    def global_step_direct(self, g_free, Bfree):
        """dx = -(H + B)^-1 g, full sparse factorisation every call (Eq. 4)."""
        Hhat = (self.H + Bfree).tocsc()
        return -spla.spsolve(Hhat, g_free)

    def split_dofs(self):
        """Free-DOF positions of x1 and x2 (vertex-major, 3 per vertex)."""
        x2v = self.x2_mask[self.free]
        d2 = np.repeat(x2v, 3)
        return np.nonzero(~d2)[0], np.nonzero(d2)[0]

    # -- Algorithm 1 -----------------------------------------------------------
    def solve_frame(self, x_t, max_iters=None, record=True, callback=None):
        """Run Algorithm 1 from x_t; returns (x, FrameStats).

        ``callback(x)`` (optional) sees every accepted iterate.
        """
        p = self.p
        max_iters = p.max_iters if max_iters is None else max_iters
        st = FrameStats()
        x = np.array(x_t, dtype=np.float64, copy=True)
        x[self.pinned] = self.rest[self.pinned]
        tol = None
        self.kappa = self.kappa0
        d_prev = np.inf
        while True:
            ev = self.evaluate(x)                          # GetProjection, C
            d_min = float(ev["C"][3].min()) if ev["C"][3].size else np.inf
            if record:
                st.d_mins.append(d_min)
            if p.adaptive_kappa:
                if (d_min < KAPPA_GROW_BELOW * p.dhat and d_min < d_prev
                        and 2.0 * self.kappa <= KAPPA_MAX_RATIO * self.kappa0):
                    ev["B"] *= 2.0                          # B is linear in kappa
                    self.kappa *= 2.0
                    st.kappa_doublings += 1
                d_prev = d_min
            g_all = self.gradient(x, ev)                   # g-hat
            g = g_all.ravel()[self.free_dofs]
            gn = float(np.linalg.norm(g))
            Ehat = ev["E"] + ev["B"]
            if tol is None:
                tol = max(p.tol_abs, p.tol_rel * gn)
            if record:
                st.grad_norms.append(gn)
                st.energies.append(Ehat)
                st.contacts.append(int(ev["C"][0].size))
            if gn <= tol:
                st.status = STATUS_OK
                break
            if st.iterations >= max_iters:
                st.status = STATUS_NOT_CONVERGED
                break
            Ball = self.barrier_hessian(ev, project=True)  # PositiveDefinite
            if record:
                rows = np.unique(Ball.nonzero()[0] // 3)
                st.n_c.append(int(np.count_nonzero(self.x2_mask[rows])) if rows.size else 0)
            dx_free = self.global_step_direct(g, self.free_part(Ball))
            dx = np.zeros_like(x)
            dx.reshape(-1)[self.free_dofs] = dx_free
            ds = self.proxy(dx)
            alpha_m = C.ccd_step_bound(ev["s"], ds, self.tris, self.edges, p.dhat, p.ccd_s)
            alpha = alpha_m
            accepted = False
            for k in range(p.max_ls + 1):
                xt = x + alpha * dx
                Et = self.energy(xt)
                if Et <= Ehat + LS_SLACK * abs(Ehat):
                    accepted = True
                    break
                alpha *= 0.5
            if record:
                st.alpha_ms.append(alpha_m)
                st.alphas.append(alpha if accepted else 0.0)
                st.ls_halvings.append(k)
            if not accepted:
                st.status = STATUS_LS_FAIL
                break
            x = xt
            st.iterations += 1
            if callback is not None:
                callback(x)
        return x, st


# ---------------------------------------------------------------------------
# dense Schur / Woodbury global steps (Sec. 3.1-3.2), for pins on tiny meshes
# ---------------------------------------------------------------------------
def schur_three_step(H: np.ndarray, Bm: np.ndarray, g: np.ndarray,
                     i1: np.ndarray, i2: np.ndarray) -> np.ndarray:
    """Solve (H + B) dx = -g by the block factorisation of Eq. 8.

    B must vanish outside the (i2, i2) block.  L1 is the Cholesky factor of
    H11; Sigma-hat = H22 + B22 - H21 H11^-1 H12 (Eq. 9); then one lower
    triangular, one (block-)diagonal and one upper triangular solve.
    """
    H11, H12 = H[np.ix_(i1, i1)], H[np.ix_(i1, i2)]
    H21, H22 = H[np.ix_(i2, i1)], H[np.ix_(i2, i2)] + Bm[np.ix_(i2, i2)]
    L1 = sla.cholesky(H11, lower=True)
    r1, r2 = -g[i1], -g[i2]
    # lower: [L1 0; H21 L1^-T I]
    y1 = sla.solve_triangular(L1, r1, lower=True)
    W12 = sla.solve_triangular(L1, H12, lower=True)          # L1^-1 H12
    y2 = r2 - W12.T @ y1
    # diagonal: [I 0; 0 Sigma-hat]
    Sig_hat = H22 - W12.T @ W12
    z2 = sla.solve(Sig_hat, y2, assume_a="sym")
    # upper: [L1^T L1^-1 H12; 0 I]
    dx1 = sla.solve_triangular(L1.T, y1 - W12 @ z2, lower=False)
    dx = np.zeros_like(g)
    dx[i1], dx[i2] = dx1, z2
    return dx


def schur_complement(H: np.ndarray, i1: np.ndarray, i2: np.ndarray) -> np.ndarray:
    """Sigma = H22 - H21 H11^-1 H12 (constant part of Eq. 9)."""
    H11, H12 = H[np.ix_(i1, i1)], H[np.ix_(i1, i2)]
    return H[np.ix_(i2, i2)] - H12.T @ sla.solve(H11, H12, assume_a="pos")


def woodbury_apply(Sigma_inv: np.ndarray, B22: np.ndarray, y: np.ndarray,
                   push_through: bool = True) -> np.ndarray:
    """Sigma-hat^-1 y with Sigma-hat = Sigma + Q^T B-check Q (Eq. 10-11).

    Q-check picks the rows/columns where B22 is non-zero (n_c vertices, 3
    DOFs each).  push_through=False uses the printed form with B-check^-1
    (requires B-check invertible); True uses (I + B-check S)^-1 B-check.
    """
    nz = np.nonzero(np.abs(B22).sum(axis=1) > 0)[0]
    verts = np.unique(nz // 3)
    c = (3 * verts[:, None] + np.arange(3)).ravel()
    u = Sigma_inv @ y
    if c.size == 0:
        return u
    Bc = B22[np.ix_(c, c)]
    S = Sigma_inv[np.ix_(c, c)]
    if push_through:
        v = np.linalg.solve(np.eye(c.size) + Bc @ S, Bc @ u[c])
    else:
        v = np.linalg.solve(np.linalg.inv(Bc) + S, u[c])
    return u - Sigma_inv[:, c] @ v


def woodbury_global_step(H: np.ndarray, Bm: np.ndarray, g: np.ndarray,
                         i1: np.ndarray, i2: np.ndarray, push_through=True) -> np.ndarray:
    """Eq. 8 with the diagonal solve done by the low-rank update of Eq. 11."""
    H11, H12 = H[np.ix_(i1, i1)], H[np.ix_(i1, i2)]
    L1 = sla.cholesky(H11, lower=True)
    Sigma = schur_complement(H, i1, i2)
    Sigma_inv = np.linalg.inv(Sigma)
    r1, r2 = -g[i1], -g[i2]
    y1 = sla.solve_triangular(L1, r1, lower=True)
    W12 = sla.solve_triangular(L1, H12, lower=True)
    y2 = r2 - W12.T @ y1
    z2 = woodbury_apply(Sigma_inv, Bm[np.ix_(i2, i2)], y2, push_through=push_through)
    dx1 = sla.solve_triangular(L1.T, y1 - W12 @ z2, lower=False)
    dx = np.zeros_like(g)
    dx[i1], dx[i2] = dx1, z2
    return dx
