// Point-triangle / edge-edge distance, closest-feature classification and the
// PSD-projected IPC barrier Hessian of one pair (device, float64).
//
// Sec. 2.2: every vertex-triangle and edge-edge pair k of the proxy with
// unsigned distance d_k < d0 contributes kappa * b(d_k) (Eq. 3).  Reading of
// the unprinted barrier: b(d) = -(d - dhat)^2 ln(d / dhat).
//
// Distance structure used here: the closest points are an affine combination
// v = sum_i c_i(beta) X_i of the pair's four vertices, with beta the k <= 2
// free parameters of the closest-feature case (face interior: k = 2, edge
// interior: k = 1, vertex: k = 0; edge-edge interior: k = 2 ...).  With
// f(x, beta) = |v|^2 minimised over beta, the envelope theorem and implicit
// differentiation give
//   grad d^2 = 2 c (x) v,
//   hess d^2 = 2 (c c^T) (x) I_3 - F (2 E^T E)^-1 F^T,
//   F_k = 2 (c'_k (x) v + c (x) E_k),  E_k = sum_i c'_k[i] X_i = dv/dbeta_k.
// Both live in the (3 + k)-dimensional span of {c^ (x) e_a} u {q_m (x) v^}
// where (c^, q_1.. q_k) orthonormalises (c, c'_1.. c'_k) in R^4, so the 12x12
// pair Hessian kappa (b'' grad d grad d^T + b' hess d) is formed, projected
// onto the PSD cone (PositiveDefinite of Algorithm 1) and lifted back exactly
// in that small basis.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace fsim {

// Classification threshold for nearly parallel edges (no mollifier: those
// pairs take the closest of the four endpoint-to-segment distances).
#define FSIM_PARALLEL_EPS 1e-10

struct PairGeom {
  double c[4];      // affine coefficients, v = sum_i c_i X_i
  double cp[2][4];  // d c / d beta_k
  int k;            // number of free parameters (0..2)
  double v[3];      // difference vector of the closest points
  double d2;        // |v|^2
};

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Closest point of segment [A, B] to P: clamped parameter and squared distance.
__device__ __forceinline__ void seg_closest(const double* P, const double* A, const double* B,
                                            double& t, double& d2) {
  double e[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
  double r[3] = {P[0] - A[0], P[1] - A[1], P[2] - A[2]};
  t = dot3(r, e) / dot3(e, e);
  t = fmin(fmax(t, 0.0), 1.0);
  double q[3] = {P[0] - (A[0] + t * e[0]), P[1] - (A[1] + t * e[1]), P[2] - (A[2] + t * e[2])};
  d2 = dot3(q, q);
}

__device__ __forceinline__ void geom_finish(PairGeom& g, const double X[4][3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d)
    g.v[d] = g.c[0] * X[0][d] + g.c[1] * X[1][d] + g.c[2] * X[2][d] + g.c[3] * X[3][d];
  g.d2 = dot3(g.v, g.v);
}

// point X[0] vs triangle X[1..3]
__device__ void pt_geometry(const double X[4][3], PairGeom& g) {
  const double* p = X[0];
  const double* a = X[1];
  const double* b = X[2];
  const double* c = X[3];
  double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double r[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  double a11 = dot3(e1, e1), a12 = dot3(e1, e2), a22 = dot3(e2, e2);
  double r1 = dot3(e1, r), r2 = dot3(e2, r);
  double det = a11 * a22 - a12 * a12;
  double u = (a22 * r1 - a12 * r2) / det;
  double w = (a11 * r2 - a12 * r1) / det;
#pragma unroll
  for (int i = 0; i < 4; ++i) { g.c[i] = 0.0; g.cp[0][i] = 0.0; g.cp[1][i] = 0.0; }
  if (u >= 0.0 && w >= 0.0 && u + w <= 1.0) {
    g.k = 2;
    g.c[0] = 1.0; g.c[1] = -(1.0 - u - w); g.c[2] = -u; g.c[3] = -w;
    g.cp[0][1] = 1.0; g.cp[0][2] = -1.0;   // d/du
    g.cp[1][1] = 1.0; g.cp[1][3] = -1.0;   // d/dw
  } else {
    double t0, d0, t1, d1, t2, d2;
    seg_closest(p, a, b, t0, d0);
    seg_closest(p, b, c, t1, d1);
    seg_closest(p, c, a, t2, d2);
    int k = 0; double t = t0, dm = d0;
    if (d1 < dm) { k = 1; t = t1; dm = d1; }
    if (d2 < dm) { k = 2; t = t2; dm = d2; }
    const int ia = 1 + k, ib = 1 + (k + 1) % 3;   // pair-local ids of the edge
    g.c[0] = 1.0;
    if (t > 0.0 && t < 1.0) {
      g.k = 1;
      g.c[ia] = -(1.0 - t); g.c[ib] = -t;
      g.cp[0][ia] = 1.0; g.cp[0][ib] = -1.0;
    } else {
      g.k = 0;
      g.c[t <= 0.0 ? ia : ib] = -1.0;
    }
  }
  geom_finish(g, X);
}

// edge X[0]X[1] vs edge X[2]X[3]
__device__ void ee_geometry(const double X[4][3], PairGeom& g) {
  const double* a0 = X[0];
  const double* a1 = X[1];
  const double* b0 = X[2];
  const double* b1 = X[3];
  double u[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
  double v[3] = {b1[0] - b0[0], b1[1] - b0[1], b1[2] - b0[2]};
  double w0[3] = {a0[0] - b0[0], a0[1] - b0[1], a0[2] - b0[2]};
  double A = dot3(u, u), B = dot3(u, v), C = dot3(v, v), D = dot3(u, w0), E = dot3(v, w0);
  double den = A * C - B * B;
#pragma unroll
  for (int i = 0; i < 4; ++i) { g.c[i] = 0.0; g.cp[0][i] = 0.0; g.cp[1][i] = 0.0; }
  bool interior = false;
  if (den > FSIM_PARALLEL_EPS * A * C) {
    double s = (B * E - C * D) / den;
    double t = (A * E - B * D) / den;
    if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
      interior = true;
      g.k = 2;
      g.c[0] = 1.0 - s; g.c[1] = s; g.c[2] = -(1.0 - t); g.c[3] = -t;
      g.cp[0][0] = -1.0; g.cp[0][1] = 1.0;
      g.cp[1][2] = 1.0; g.cp[1][3] = -1.0;
    }
  }
  if (!interior) {
    double ta0, da0, ta1, da1, tb0, db0, tb1, db1;
    seg_closest(a0, b0, b1, ta0, da0);
    seg_closest(a1, b0, b1, ta1, da1);
    seg_closest(b0, a0, a1, tb0, db0);
    seg_closest(b1, a0, a1, tb1, db1);
    int k = 0; double t = ta0, dm = da0;
    if (da1 < dm) { k = 1; t = ta1; dm = da1; }
    if (db0 < dm) { k = 2; t = tb0; dm = db0; }
    if (db1 < dm) { k = 3; t = tb1; dm = db1; }
    const bool mid = t > 0.0 && t < 1.0;
    if (k < 2) {            // point a_k vs segment b: v = a_k - (b0 + t (b1 - b0))
      g.c[k] = 1.0;
      if (mid) {
        g.k = 1; g.c[2] = -(1.0 - t); g.c[3] = -t;
        g.cp[0][2] = 1.0; g.cp[0][3] = -1.0;
      } else {
        g.k = 0; g.c[t <= 0.0 ? 2 : 3] = -1.0;
      }
    } else {                // point b_(k-2) vs segment a: v = (a0 + t (a1 - a0)) - b
      g.c[k] = -1.0;
      if (mid) {
        g.k = 1; g.c[0] = 1.0 - t; g.c[1] = t;
        g.cp[0][0] = -1.0; g.cp[0][1] = 1.0;
      } else {
        g.k = 0; g.c[t <= 0.0 ? 0 : 1] = 1.0;
      }
    }
  }
  geom_finish(g, X);
}

__device__ __forceinline__ void pair_geometry(int type, const double X[4][3], PairGeom& g) {
  if (type == 0) pt_geometry(X, g);
  else ee_geometry(X, g);
}

__device__ __forceinline__ double pair_distance(int type, const double X[4][3]) {
  PairGeom g;
  pair_geometry(type, X, g);
  return sqrt(g.d2);
}

// float32 distance of a pair given in coordinates relative to its first
// vertex (rounding error ~1e-7 of the pair's own extent).  Used only as a
// conservative filter: callers act on it only when it is far (>= 2x) from
// the threshold they test, so the float64 decision is never changed.
__device__ __forceinline__ float seg_d2f(const float* P, const float* A, const float* B) {
  const float e0 = B[0] - A[0], e1 = B[1] - A[1], e2 = B[2] - A[2];
  const float r0 = P[0] - A[0], r1 = P[1] - A[1], r2 = P[2] - A[2];
  const float ee = e0 * e0 + e1 * e1 + e2 * e2;
  float t = ee > 0.f ? (r0 * e0 + r1 * e1 + r2 * e2) / ee : 0.f;
  t = fminf(fmaxf(t, 0.f), 1.f);
  const float q0 = r0 - t * e0, q1 = r1 - t * e1, q2 = r2 - t * e2;
  return q0 * q0 + q1 * q1 + q2 * q2;
}

__device__ float pair_distance_f(int type, const float X[4][3]) {
  if (type == 0) {
    const float* p = X[0]; const float* a = X[1]; const float* b = X[2]; const float* c = X[3];
    const float e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const float e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const float r[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    const float a11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const float a12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    const float a22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    const float r1 = e1[0] * r[0] + e1[1] * r[1] + e1[2] * r[2];
    const float r2 = e2[0] * r[0] + e2[1] * r[1] + e2[2] * r[2];
    const float det = a11 * a22 - a12 * a12;
    if (det > 0.f) {
      const float u = (a22 * r1 - a12 * r2) / det, w = (a11 * r2 - a12 * r1) / det;
      if (u >= 0.f && w >= 0.f && u + w <= 1.f) {
        const float q0 = r[0] - u * e1[0] - w * e2[0], q1 = r[1] - u * e1[1] - w * e2[1],
                    q2 = r[2] - u * e1[2] - w * e2[2];
        return sqrtf(q0 * q0 + q1 * q1 + q2 * q2);
      }
    }
    return sqrtf(fminf(fminf(seg_d2f(p, a, b), seg_d2f(p, b, c)), seg_d2f(p, c, a)));
  }
  const float* a0 = X[0]; const float* a1 = X[1]; const float* b0 = X[2]; const float* b1 = X[3];
  const float u[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
  const float v[3] = {b1[0] - b0[0], b1[1] - b0[1], b1[2] - b0[2]};
  const float w0[3] = {a0[0] - b0[0], a0[1] - b0[1], a0[2] - b0[2]};
  const float A = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const float B = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  const float C = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const float D = u[0] * w0[0] + u[1] * w0[1] + u[2] * w0[2];
  const float E = v[0] * w0[0] + v[1] * w0[1] + v[2] * w0[2];
  const float den = A * C - B * B;
  if (den > 1e-6f * A * C) {
    const float s = (B * E - C * D) / den, t = (A * E - B * D) / den;
    if (s > 0.f && s < 1.f && t > 0.f && t < 1.f) {
      const float q0 = w0[0] + s * u[0] - t * v[0], q1 = w0[1] + s * u[1] - t * v[1],
                  q2 = w0[2] + s * u[2] - t * v[2];
      return sqrtf(q0 * q0 + q1 * q1 + q2 * q2);
    }
  }
  return sqrtf(fminf(fminf(seg_d2f(a0, b0, b1), seg_d2f(a1, b0, b1)),
                     fminf(seg_d2f(b0, a0, a1), seg_d2f(b1, a0, a1))));
}

// X relative to its first vertex, in float32
__device__ __forceinline__ void to_rel_f(const double X[4][3], float Y[4][3]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) Y[k][d] = (float)(X[k][d] - X[0][d]);
}

// IPC barrier and its first two derivatives (reading of Eq. 3's b).
__device__ __forceinline__ void barrier3(double d, double dhat, double& b, double& b1, double& b2) {
  const double u = d - dhat;
  const double L = log(d / dhat);
  b = -u * u * L;
  b1 = -2.0 * u * L - u * u / d;
  b2 = -2.0 * L - 4.0 * u / d + u * u / (d * d);
}

__device__ __forceinline__ double barrier_value(double d, double dhat) {
  if (!(d < dhat)) return 0.0;
  const double u = d - dhat;
  return -u * u * log(d / dhat);
}

// The pair Hessian kappa (b'' grad d grad d^T + b' hess d) in the reduced
// basis {c^ (x) e_a} u {q_m (x) v^} (n = 3 + k <= 5 coordinates), before the
// PSD projection, with everything the lift back to the 12x12 blocks needs.
struct PairReduced {
  int n, k;
  double d;            // unsigned distance
  double gfac;         // kappa b'(d): gradient of vertex i = gfac c_i v^
  double c[4];         // affine coefficients
  double ch[4];        // c / |c|
  double q[2][4];      // orthonormal complement directions in R^4
  double vh[3];        // v / |v|
  double A[5][5];      // reduced Hessian (n x n used)
};

__device__ void pair_reduced(int type, const double X[4][3], double dhat, double kappa,
                             PairReduced& r) {
  PairGeom g;
  pair_geometry(type, X, g);
  const double d = sqrt(g.d2);
  double b, b1, b2;
  barrier3(d, dhat, b, b1, b2);
  const int k = g.k, n = 3 + k;
  r.n = n; r.k = k; r.d = d; r.gfac = kappa * b1;
  // orthonormal (c^, q_1 .. q_k) in R^4
  const double cn = sqrt(g.c[0] * g.c[0] + g.c[1] * g.c[1] + g.c[2] * g.c[2] + g.c[3] * g.c[3]);
  for (int i = 0; i < 4; ++i) { r.c[i] = g.c[i]; r.ch[i] = g.c[i] / cn; }
  double qc[2][2] = {{0, 0}, {0, 0}};   // q_m . c'_k
  double chc[2] = {0, 0};                // c^ . c'_k
  for (int m = 0; m < k; ++m) {
    double w[4];
    for (int i = 0; i < 4; ++i) w[i] = g.cp[m][i];
    double a = 0;
    for (int i = 0; i < 4; ++i) a += r.ch[i] * w[i];
    for (int i = 0; i < 4; ++i) w[i] -= a * r.ch[i];
    for (int l = 0; l < m; ++l) {
      double bq = 0;
      for (int i = 0; i < 4; ++i) bq += r.q[l][i] * w[i];
      for (int i = 0; i < 4; ++i) w[i] -= bq * r.q[l][i];
    }
    const double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
    for (int i = 0; i < 4; ++i) r.q[m][i] = w[i] / wn;
  }
  for (int m = k; m < 2; ++m)
    for (int i = 0; i < 4; ++i) r.q[m][i] = 0.0;
  for (int kk = 0; kk < k; ++kk) {
    double t = 0;
    for (int i = 0; i < 4; ++i) t += r.ch[i] * g.cp[kk][i];
    chc[kk] = t;
    for (int m = 0; m < k; ++m) {
      double u = 0;
      for (int i = 0; i < 4; ++i) u += r.q[m][i] * g.cp[kk][i];
      qc[m][kk] = u;
    }
  }
  double E[2][3];
  for (int kk = 0; kk < k; ++kk)
    for (int dd = 0; dd < 3; ++dd)
      E[kk][dd] = g.cp[kk][0] * X[0][dd] + g.cp[kk][1] * X[1][dd] + g.cp[kk][2] * X[2][dd] +
                  g.cp[kk][3] * X[3][dd];
  // reduced hess d^2: diag(2|c|^2 I3, 0) - F (2 E^T E)^-1 F^T
  double Hd2[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) Hd2[i][j] = 0.0;
  for (int a = 0; a < 3; ++a) Hd2[a][a] = 2.0 * cn * cn;
  if (k > 0) {
    double Fr[5][2];
    for (int kk = 0; kk < k; ++kk) {
      for (int a = 0; a < 3; ++a) Fr[a][kk] = 2.0 * (chc[kk] * g.v[a] + cn * E[kk][a]);
      for (int m = 0; m < k; ++m) Fr[3 + m][kk] = 2.0 * qc[m][kk] * d;
    }
    double G[2][2], Gi[2][2];
    for (int a = 0; a < k; ++a)
      for (int bb = 0; bb < k; ++bb) G[a][bb] = 2.0 * dot3(E[a], E[bb]);
    if (k == 1) {
      Gi[0][0] = 1.0 / G[0][0];
    } else {
      const double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
      Gi[0][0] = G[1][1] / det; Gi[1][1] = G[0][0] / det;
      Gi[0][1] = -G[0][1] / det; Gi[1][0] = -G[1][0] / det;
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double t = 0.0;
        for (int a = 0; a < k; ++a)
          for (int bb = 0; bb < k; ++bb) t += Fr[i][a] * Gi[a][bb] * Fr[j][bb];
        Hd2[i][j] -= t;
      }
  }
  // grad d = (|c| v^, 0); hess d = hess d^2/(2d) - (|c|^2 v^ v^T (+) 0)/d
  for (int a = 0; a < 3; ++a) r.vh[a] = g.v[a] / d;
  const double gr[5] = {cn * r.vh[0], cn * r.vh[1], cn * r.vh[2], 0.0, 0.0};
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      if (i < n && j < n) {
        const double hdd = Hd2[i][j] / (2.0 * d) -
                           (i < 3 && j < 3 ? cn * cn * r.vh[i] * r.vh[j] / d : 0.0);
        r.A[i][j] = kappa * (b2 * gr[i] * gr[j] + b1 * hdd);
      } else {
        r.A[i][j] = 0.0;
      }
    }
}

// ---------------------------------------------------------------------------
// Edge-edge mollifier (optional; IPC's treatment of nearly parallel edges):
// with c = |e_a x e_b|^2 and eps = 1e-3 |E_a|^2 |E_b|^2 at rest, the EE term
// becomes kappa m(c) b(d), m(c) = (2 - c/eps) c/eps for c < eps, else 1.
// ---------------------------------------------------------------------------
#define FSIM_MOLLIFIER_EPS_SCALE 1e-3

struct EdgeCross {
  double ea[3], eb[3];   // a1 - a0, b1 - b0
  double aa, bb, ab;     // ea.ea, eb.eb, ea.eb
  double c;              // |ea x eb|^2
};

__device__ __forceinline__ void edge_cross(const double X[4][3], EdgeCross& e) {
  for (int d = 0; d < 3; ++d) {
    e.ea[d] = X[1][d] - X[0][d];
    e.eb[d] = X[3][d] - X[2][d];
  }
  const double w0 = e.ea[1] * e.eb[2] - e.ea[2] * e.eb[1];
  const double w1 = e.ea[2] * e.eb[0] - e.ea[0] * e.eb[2];
  const double w2 = e.ea[0] * e.eb[1] - e.ea[1] * e.eb[0];
  e.c = w0 * w0 + w1 * w1 + w2 * w2;
  e.aa = dot3(e.ea, e.ea);
  e.bb = dot3(e.eb, e.eb);
  e.ab = dot3(e.ea, e.eb);
}

__device__ __forceinline__ double mollifier_value(double c, double eps) {
  if (!(c < eps)) return 1.0;
  const double q = c / eps;
  return (2.0 - q) * q;
}

// d c / d X[I][al] (vertices a0, a1, b0, b1)
__device__ __forceinline__ double edge_cross_grad(const EdgeCross& e, int I, int al) {
  const double ga = 2.0 * (e.ea[al] * e.bb - e.ab * e.eb[al]);
  const double gb = 2.0 * (e.eb[al] * e.aa - e.ab * e.ea[al]);
  const double g = (I < 2) ? ga : gb;
  return (I == 0 || I == 2) ? -g : g;
}

// d^2 c / d X[I][al] d X[J][be]
__device__ __forceinline__ double edge_cross_hess(const EdgeCross& e, int I, int al, int J, int be) {
  const double dl = (al == be) ? 1.0 : 0.0;
  const int ei = I >> 1, ej = J >> 1;     // 0: edge a, 1: edge b
  double h;
  if (ei == 0 && ej == 0) h = 2.0 * e.bb * dl - 2.0 * e.eb[al] * e.eb[be];
  else if (ei == 1 && ej == 1) h = 2.0 * e.aa * dl - 2.0 * e.ea[al] * e.ea[be];
  else if (ei == 0) h = 4.0 * e.ea[al] * e.eb[be] - 2.0 * e.eb[al] * e.ea[be] - 2.0 * e.ab * dl;
  else h = 4.0 * e.ea[be] * e.eb[al] - 2.0 * e.eb[be] * e.ea[al] - 2.0 * e.ab * dl;
  const double si = (I == 0 || I == 2) ? -1.0 : 1.0, sj = (J == 0 || J == 2) ? -1.0 : 1.0;
  return si * sj * h;
}

}  // namespace fsim
