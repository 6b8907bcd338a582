"""Oracle: unsigned primitive distances with exact gradient and Hessian.

Sec. 2.2: for every point-triangle (PT) and edge-edge (EE) pair of the proxy
surface the unsigned distance d_k enters the barrier.  The distance is
piecewise smooth: which closest features meet (vertex, edge interior, face
interior) decides a closed form for d^2:

* point-point   d^2 = |p - q|^2
* point-line    d^2 = |(p - a) x (b - a)|^2 / |b - a|^2
* point-plane   d^2 = ((p - a) . n)^2 / |n|^2,  n = (b - a) x (c - a)
* line-line     d^2 = ((a0 - b0) . n)^2 / |n|^2, n = (a1 - a0) x (b1 - b0)

Derivatives are exact: each closed form is evaluated on ``Hd`` numbers that
carry the value, the 12-gradient and the 12x12 Hessian with respect to the
pair's four vertices (second-order forward-mode differentiation).

Reading (no EE mollifier in the paper): nearly parallel edges, whose 2x2
line-line system has ``a*c - b^2 <= PARALLEL_EPS * a * c``, take the closest
pair among the four endpoint-to-segment distances, which is exact for
parallel edges.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

PARALLEL_EPS = 1e-10

# case codes ------------------------------------------------------------------
# PT: vertex order (p, t0, t1, t2)
PT_FACE, PT_E01, PT_E12, PT_E20, PT_V0, PT_V1, PT_V2 = range(7)
# EE: vertex order (a0, a1, b0, b1)
EE_INT, EE_A0_B, EE_A1_B, EE_B0_A, EE_B1_A, EE_A0B0, EE_A0B1, EE_A1B0, EE_A1B1 = range(9)


class Hd:
    """Value, gradient (P,12) and Hessian (P,12,12) of P scalar functions."""
    __slots__ = ("v", "g", "h")

    def __init__(self, v, g, h):
        self.v, self.g, self.h = v, g, h

    @staticmethod
    def variable(values: np.ndarray, index: int, nvar: int = 12) -> "Hd":
        P = values.shape[0]
        g = np.zeros((P, nvar))
        g[:, index] = 1.0
        return Hd(values.astype(np.float64), g, np.zeros((P, nvar, nvar)))

    def _lift(self, o):
        if isinstance(o, Hd):
            return o
        o = np.broadcast_to(np.asarray(o, dtype=np.float64), self.v.shape)
        return Hd(o, np.zeros_like(self.g), np.zeros_like(self.h))

    def __add__(self, o):
        o = self._lift(o)
        return Hd(self.v + o.v, self.g + o.g, self.h + o.h)

    __radd__ = __add__

    def __neg__(self):
        return Hd(-self.v, -self.g, -self.h)

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        o = self._lift(o)
        a, b = self, o
        gg = a.g[:, :, None] * b.g[:, None, :]
        return Hd(a.v * b.v,
                  a.v[:, None] * b.g + b.v[:, None] * a.g,
                  a.v[:, None, None] * b.h + b.v[:, None, None] * a.h + gg
                  + np.swapaxes(gg, 1, 2))

    __rmul__ = __mul__

    def reciprocal(self):
        v = 1.0 / self.v
        return Hd(v, -self.g * (v * v)[:, None],
                  -self.h * (v * v)[:, None, None]
                  + 2.0 * (v ** 3)[:, None, None] * self.g[:, :, None] * self.g[:, None, :])

    def __truediv__(self, o):
        return self * self._lift(o).reciprocal()

    def sqrt(self):
        r = np.sqrt(self.v)
        return Hd(r, self.g / (2.0 * r)[:, None],
                  self.h / (2.0 * r)[:, None, None]
                  - self.g[:, :, None] * self.g[:, None, :] / (4.0 * r ** 3)[:, None, None])

    def log(self):
        return Hd(np.log(self.v), self.g / self.v[:, None],
                  self.h / self.v[:, None, None]
                  - self.g[:, :, None] * self.g[:, None, :] / (self.v ** 2)[:, None, None])

    def select(self, mask, other: "Hd") -> "Hd":
        """Elementwise choice: self where mask, else other."""
        return Hd(np.where(mask, self.v, other.v),
                  np.where(mask[:, None], self.g, other.g),
                  np.where(mask[:, None, None], self.h, other.h))


def _vec(X: np.ndarray, vtx: int):
    """Hd 3-vector for vertex ``vtx`` of pairs X (P,4,3)."""
    return [Hd.variable(X[:, vtx, c], 3 * vtx + c) for c in range(3)]


def _sub3(a, b):
    return [a[i] - b[i] for i in range(3)]


def _dot3(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross3(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def d2_point_point(p, q):
    r = _sub3(p, q)
    return _dot3(r, r)


def d2_point_line(p, a, b):
    e = _sub3(b, a)
    c = _cross3(_sub3(p, a), e)
    return _dot3(c, c) / _dot3(e, e)


def d2_point_plane(p, a, b, c):
    n = _cross3(_sub3(b, a), _sub3(c, a))
    s = _dot3(_sub3(p, a), n)
    return s * s / _dot3(n, n)


def d2_line_line(a0, a1, b0, b1):
    n = _cross3(_sub3(a1, a0), _sub3(b1, b0))
    s = _dot3(_sub3(a0, b0), n)
    return s * s / _dot3(n, n)


# ---------------------------------------------------------------------------
# closest-feature classification (plain float64 geometry)
# ---------------------------------------------------------------------------
def _seg_param(p, a, b):
    """Clamped parameter of the closest point of segment ab to p, and d^2."""
    e = b - a
    t = np.einsum("ij,ij->i", p - a, e) / np.einsum("ij,ij->i", e, e)
    t = np.clip(t, 0.0, 1.0)
    r = p - (a + t[:, None] * e)
    return t, np.einsum("ij,ij->i", r, r)


def pt_case(X: np.ndarray) -> np.ndarray:
    """Closest-feature case of point X[:,0] against triangle X[:,1:4]."""
    p, a, b, c = X[:, 0], X[:, 1], X[:, 2], X[:, 3]
    e1, e2, r = b - a, c - a, p - a
    a11 = np.einsum("ij,ij->i", e1, e1)
    a12 = np.einsum("ij,ij->i", e1, e2)
    a22 = np.einsum("ij,ij->i", e2, e2)
    r1 = np.einsum("ij,ij->i", e1, r)
    r2 = np.einsum("ij,ij->i", e2, r)
    det = a11 * a22 - a12 * a12
    u = (a22 * r1 - a12 * r2) / det
    v = (a11 * r2 - a12 * r1) / det
    inside = (u >= 0.0) & (v >= 0.0) & (u + v <= 1.0)
    t01, d01 = _seg_param(p, a, b)
    t12, d12 = _seg_param(p, b, c)
    t20, d20 = _seg_param(p, c, a)
    D = np.stack([d01, d12, d20], axis=1)
    Tp = np.stack([t01, t12, t20], axis=1)
    k = np.argmin(D, axis=1)            # first minimum on ties
    t = Tp[np.arange(len(k)), k]
    # edge k runs from vertex k to vertex (k+1)%3 (triangle-local ids)
    case = np.where((t > 0.0) & (t < 1.0), PT_E01 + k,
                    np.where(t <= 0.0, PT_V0 + k, PT_V0 + (k + 1) % 3))
    return np.where(inside, PT_FACE, case).astype(np.int64)


def ee_case(X: np.ndarray) -> np.ndarray:
    """Closest-feature case of edge X[:,0:2] against edge X[:,2:4]."""
    a0, a1, b0, b1 = X[:, 0], X[:, 1], X[:, 2], X[:, 3]
    u, v, w0 = a1 - a0, b1 - b0, a0 - b0
    a = np.einsum("ij,ij->i", u, u)
    b = np.einsum("ij,ij->i", u, v)
    c = np.einsum("ij,ij->i", v, v)
    d = np.einsum("ij,ij->i", u, w0)
    e = np.einsum("ij,ij->i", v, w0)
    den = a * c - b * b
    ok = den > PARALLEL_EPS * a * c
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (b * e - c * d) / den
        t = (a * e - b * d) / den
    interior = ok & (s > 0.0) & (s < 1.0) & (t > 0.0) & (t < 1.0)
    # boundary candidates: a0|b, a1|b, b0|a, b1|a
    ta0, da0 = _seg_param(a0, b0, b1)
    ta1, da1 = _seg_param(a1, b0, b1)
    tb0, db0 = _seg_param(b0, a0, a1)
    tb1, db1 = _seg_param(b1, a0, a1)
    D = np.stack([da0, da1, db0, db1], axis=1)
    Tp = np.stack([ta0, ta1, tb0, tb1], axis=1)
    k = np.argmin(D, axis=1)
    t_ = Tp[np.arange(len(k)), k]
    mid = (t_ > 0.0) & (t_ < 1.0)
    at0 = t_ <= 0.0
    # point-point codes: (a0,b0)=5 (a0,b1)=6 (a1,b0)=7 (a1,b1)=8
    pp = np.select([k == 0, k == 1, k == 2, k == 3],
                   [np.where(at0, EE_A0B0, EE_A0B1), np.where(at0, EE_A1B0, EE_A1B1),
                    np.where(at0, EE_A0B0, EE_A1B0), np.where(at0, EE_A0B1, EE_A1B1)])
    case = np.where(mid, EE_A0_B + k, pp)
    return np.where(interior, EE_INT, case).astype(np.int64)


# ---------------------------------------------------------------------------
# distance with derivatives
# ---------------------------------------------------------------------------
def _d2_by_case_pt(X, case):
    V = [_vec(X, i) for i in range(4)]
    p, a, b, c = V
    forms = {
        PT_FACE: lambda: d2_point_plane(p, a, b, c),
        PT_E01: lambda: d2_point_line(p, a, b),
        PT_E12: lambda: d2_point_line(p, b, c),
        PT_E20: lambda: d2_point_line(p, c, a),
        PT_V0: lambda: d2_point_point(p, a),
        PT_V1: lambda: d2_point_point(p, b),
        PT_V2: lambda: d2_point_point(p, c),
    }
    return forms, case


def _d2_by_case_ee(X, case):
    V = [_vec(X, i) for i in range(4)]
    a0, a1, b0, b1 = V
    forms = {
        EE_INT: lambda: d2_line_line(a0, a1, b0, b1),
        EE_A0_B: lambda: d2_point_line(a0, b0, b1),
        EE_A1_B: lambda: d2_point_line(a1, b0, b1),
        EE_B0_A: lambda: d2_point_line(b0, a0, a1),
        EE_B1_A: lambda: d2_point_line(b1, a0, a1),
        EE_A0B0: lambda: d2_point_point(a0, b0),
        EE_A0B1: lambda: d2_point_point(a0, b1),
        EE_A1B0: lambda: d2_point_point(a1, b0),
        EE_A1B1: lambda: d2_point_point(a1, b1),
    }
    return forms, case


def squared_distance_hd(X: np.ndarray, is_ee: np.ndarray) -> Hd:
    """d^2 as an Hd number for pairs X (P,4,3); is_ee marks edge-edge pairs."""
    P = X.shape[0]
    out = Hd(np.zeros(P), np.zeros((P, 12)), np.zeros((P, 12, 12)))
    is_ee = np.asarray(is_ee, dtype=bool)
    for kind in (False, True):
        sel = np.nonzero(is_ee == kind)[0]
        if sel.size == 0:
            continue
        Xs = X[sel]
        case = ee_case(Xs) if kind else pt_case(Xs)
        for code in np.unique(case):
            sub = sel[case == code]
            Xc = X[sub]
            forms, _ = (_d2_by_case_ee if kind else _d2_by_case_pt)(Xc, None)
            r = forms[int(code)]()
            out.v[sub], out.g[sub], out.h[sub] = r.v, r.g, r.h
    return out


def distance_hd(X: np.ndarray, is_ee: np.ndarray) -> Hd:
    """Unsigned distance d = sqrt(d^2) with gradient and Hessian."""
    return squared_distance_hd(X, is_ee).sqrt()


def distance(X: np.ndarray, is_ee: np.ndarray) -> np.ndarray:
    """Unsigned distance values only (same closed forms, no derivatives)."""
    P = X.shape[0]
    d = np.zeros(P)
    is_ee = np.asarray(is_ee, dtype=bool)
    for kind in (False, True):
        sel = np.nonzero(is_ee == kind)[0]
        if sel.size == 0:
            continue
        case = ee_case(X[sel]) if kind else pt_case(X[sel])
        d[sel] = _distance_values(X[sel], case, kind)
    return d


def _distance_values(X, case, is_ee):
    """Value-only evaluation of the closed forms (float64 arrays)."""
    def dot(a, b):
        return np.einsum("ij,ij->i", a, b)

    def pp(p, q):
        r = p - q
        return dot(r, r)

    def pl(p, a, b):
        e = b - a
        c = np.cross(p - a, e)
        return dot(c, c) / dot(e, e)

    def pf(p, a, b, c):
        n = np.cross(b - a, c - a)
        s = dot(p - a, n)
        return s * s / dot(n, n)

    def ll(a0, a1, b0, b1):
        n = np.cross(a1 - a0, b1 - b0)
        s = dot(a0 - b0, n)
        return s * s / dot(n, n)

    out = np.zeros(X.shape[0])
    V = [X[:, i] for i in range(4)]
    if is_ee:
        a0, a1, b0, b1 = V
        table = {EE_INT: lambda m: ll(a0[m], a1[m], b0[m], b1[m]),
                 EE_A0_B: lambda m: pl(a0[m], b0[m], b1[m]),
                 EE_A1_B: lambda m: pl(a1[m], b0[m], b1[m]),
                 EE_B0_A: lambda m: pl(b0[m], a0[m], a1[m]),
                 EE_B1_A: lambda m: pl(b1[m], a0[m], a1[m]),
                 EE_A0B0: lambda m: pp(a0[m], b0[m]),
                 EE_A0B1: lambda m: pp(a0[m], b1[m]),
                 EE_A1B0: lambda m: pp(a1[m], b0[m]),
                 EE_A1B1: lambda m: pp(a1[m], b1[m])}
    else:
        p, a, b, c = V
        table = {PT_FACE: lambda m: pf(p[m], a[m], b[m], c[m]),
                 PT_E01: lambda m: pl(p[m], a[m], b[m]),
                 PT_E12: lambda m: pl(p[m], b[m], c[m]),
                 PT_E20: lambda m: pl(p[m], c[m], a[m]),
                 PT_V0: lambda m: pp(p[m], a[m]),
                 PT_V1: lambda m: pp(p[m], b[m]),
                 PT_V2: lambda m: pp(p[m], c[m])}
    for code in np.unique(case):
        m = case == code
        out[m] = table[int(code)](m)
    return np.sqrt(np.maximum(out, 0.0))
