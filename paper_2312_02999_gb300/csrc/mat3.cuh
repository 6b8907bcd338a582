// Small fixed-size linear algebra for the per-tet local step (device).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace fsim {

template <typename T>
struct M3 {
  T m[3][3];
};

template <typename T>
__device__ __forceinline__ T sqrt_t(T v);
template <>
__device__ __forceinline__ double sqrt_t<double>(double v) { return sqrt(v); }
template <>
__device__ __forceinline__ float sqrt_t<float>(float v) { return sqrtf(v); }

// a / b and 1 / sqrt(v): exact float64 operations; in float32 the fast
// hardware forms (a few ulp), which the float32 polar rotation can use
// because the mixed local step refines its rotation in double-float
// arithmetic afterwards
template <typename T>
__device__ __forceinline__ T fdiv_t(T a, T b);
template <>
__device__ __forceinline__ double fdiv_t<double>(double a, double b) { return a / b; }
template <>
__device__ __forceinline__ float fdiv_t<float>(float a, float b) { return __fdividef(a, b); }
template <typename T>
__device__ __forceinline__ T rsqrt_t(T v);
template <>
__device__ __forceinline__ double rsqrt_t<double>(double v) { return 1.0 / sqrt(v); }
template <>
__device__ __forceinline__ float rsqrt_t<float>(float v) { return rsqrtf(v); }

template <typename T>
__device__ __forceinline__ void matmul(const T A[3][3], const T B[3][3], T C[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j];
}

// C = A^T B
template <typename T>
__device__ __forceinline__ void matmul_tn(const T A[3][3], const T B[3][3], T C[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[i][j] = A[0][i] * B[0][j] + A[1][i] * B[1][j] + A[2][i] * B[2][j];
}

// C = A B^T
template <typename T>
__device__ __forceinline__ void matmul_nt(const T A[3][3], const T B[3][3], T C[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[i][j] = A[i][0] * B[j][0] + A[i][1] * B[j][1] + A[i][2] * B[j][2];
}

template <typename T>
__device__ __forceinline__ T det3(const T A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// Rotation factor of the polar decomposition of M (closest rotation), by a
// one-sided (Hestenes) Jacobi SVD: plane rotations from the right
// orthogonalise the columns of M, M V = U diag(sigma) with V in SO(3).  The
// column with the smallest sigma is flipped when det M < 0, so that U is a
// rotation and R = U V^T maximises tr(R^T M) over SO(3).
template <typename T, int SWEEPS>
__device__ void polar_rotation(const T M[3][3], T R[3][3]) {
  T B[3][3], V[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      B[i][j] = M[i][j];
      V[i][j] = (i == j) ? T(1) : T(0);
    }
  const T tiny = sizeof(T) == 8 ? T(1e-300) : T(1e-30);
  const T eps = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
#pragma unroll 1
  for (int sw = 0; sw < SWEEPS; ++sw) {
    T off = T(0);
#pragma unroll
    for (int pair = 0; pair < 3; ++pair) {
      const int p = pair == 2 ? 1 : 0;
      const int q = pair == 0 ? 1 : 2;
      T a = B[0][p] * B[0][p] + B[1][p] * B[1][p] + B[2][p] * B[2][p];
      T b = B[0][q] * B[0][q] + B[1][q] * B[1][q] + B[2][q] * B[2][q];
      T g = B[0][p] * B[0][q] + B[1][p] * B[1][q] + B[2][p] * B[2][q];
      T ag = fabs(g);
      if (ag > eps * sqrt_t(a * b) && ag > tiny) {
        off += ag;
        T zeta = fdiv_t(b - a, T(2) * g);
        T t = fdiv_t(zeta >= T(0) ? T(1) : T(-1), fabs(zeta) + sqrt_t(T(1) + zeta * zeta));
        T c = rsqrt_t(T(1) + t * t);
        T s = c * t;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          T bp = B[i][p], bq = B[i][q];
          B[i][p] = c * bp - s * bq;
          B[i][q] = s * bp + c * bq;
          T vp = V[i][p], vq = V[i][q];
          V[i][p] = c * vp - s * vq;
          V[i][q] = s * vp + c * vq;
        }
      }
    }
    if (off == T(0)) break;
  }
  T sig[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) sig[j] = sqrt_t(B[0][j] * B[0][j] + B[1][j] * B[1][j] + B[2][j] * B[2][j]);
  int kmin = 0;
  if (sig[1] < sig[kmin]) kmin = 1;
  if (sig[2] < sig[kmin]) kmin = 2;
  // columns ka < kb are the two others; selects instead of indexing with
  // kmin keep every array in registers
  const T sa = kmin == 0 ? sig[1] : sig[0];
  const T sb = kmin == 2 ? sig[1] : sig[2];
  T a[3], b[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T ba = kmin == 0 ? B[i][1] : B[i][0];
    const T bb = kmin == 2 ? B[i][1] : B[i][2];
    a[i] = sa > tiny ? fdiv_t(ba, sa) : T(0);
    b[i] = sb > tiny ? fdiv_t(bb, sb) : T(0);
  }
  if (!(sa > tiny)) { a[0] = 1; a[1] = 0; a[2] = 0; }
  if (!(sb > tiny)) {  // any unit vector orthogonal to a
    T px = fabs(a[0]) < T(0.9) ? T(1) : T(0), py = fabs(a[0]) < T(0.9) ? T(0) : T(1), pz = T(0);
    T cx = a[1] * pz - a[2] * py, cy = a[2] * px - a[0] * pz, cz = a[0] * py - a[1] * px;
    T nn = sqrt_t(cx * cx + cy * cy + cz * cz);
    b[0] = cx / nn; b[1] = cy / nn; b[2] = cz / nn;
  }
  // the third column completes a right-handed frame in the orientation of
  // (ka, kb, kmin) inside V's frame: u_kmin = s * (u_ka x u_kb), where s is
  // the sign that makes det U = +1 for the cyclic order of the indices
  // (s = -1 only for (ka, kb, kmin) = (0, 2, 1))
  const T orient = kmin == 1 ? T(-1) : T(1);
  T c[3];
  c[0] = orient * (a[1] * b[2] - a[2] * b[1]);
  c[1] = orient * (a[2] * b[0] - a[0] * b[2]);
  c[2] = orient * (a[0] * b[1] - a[1] * b[0]);
  T U[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    U[i][0] = kmin == 0 ? c[i] : a[i];
    U[i][1] = kmin == 1 ? c[i] : (kmin == 0 ? a[i] : b[i]);
    U[i][2] = kmin == 2 ? c[i] : b[i];
  }
  // R = U V^T (V is a product of plane rotations, det V = +1)
  matmul_nt(U, V, R);
}

// One Newton correction of an approximate polar rotation R0 of M (float64):
// re-orthonormalise R0 (one Newton-Schulz step), then rotate by exp([w]) with
// w solving ((tr S) I - S) w = 2 axial(skew(R1^T M)), S = sym(R1^T M), the
// first-order condition for (R1 exp[w])^T M to be symmetric.
__device__ __forceinline__ void polar_refine(const double M[3][3], const double R0[3][3],
                                             double R[3][3]) {
  double G[3][3], R1[3][3], S[3][3];
  matmul_tn(R0, R0, G);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) G[i][j] = ((i == j) ? 1.5 : 0.0) - 0.5 * G[i][j];
  matmul(R0, G, R1);
  matmul_tn(R1, M, S);
  const double a0 = 0.5 * (S[2][1] - S[1][2]);
  const double a1 = 0.5 * (S[0][2] - S[2][0]);
  const double a2 = 0.5 * (S[1][0] - S[0][1]);
  const double s00 = S[0][0], s11 = S[1][1], s22 = S[2][2];
  const double s01 = 0.5 * (S[0][1] + S[1][0]);
  const double s02 = 0.5 * (S[0][2] + S[2][0]);
  const double s12 = 0.5 * (S[1][2] + S[2][1]);
  const double tr = s00 + s11 + s22;
  // A = tr I - S (symmetric); w = A^-1 (2a) by the adjugate
  const double A00 = tr - s00, A11 = tr - s11, A22 = tr - s22;
  const double A01 = -s01, A02 = -s02, A12 = -s12;
  const double c00 = A11 * A22 - A12 * A12, c01 = A02 * A12 - A01 * A22, c02 = A01 * A12 - A02 * A11;
  const double c11 = A00 * A22 - A02 * A02, c12 = A01 * A02 - A00 * A12, c22 = A00 * A11 - A01 * A01;
  const double det = A00 * c00 + A01 * c01 + A02 * c02;
  double w0 = 0.0, w1 = 0.0, w2 = 0.0;
  if (fabs(det) > 1e-300) {
    const double id = 2.0 / det;
    w0 = id * (c00 * a0 + c01 * a1 + c02 * a2);
    w1 = id * (c01 * a0 + c11 * a1 + c12 * a2);
    w2 = id * (c02 * a0 + c12 * a1 + c22 * a2);
  }
  // exp([w]) to second order (|w| ~ float32 rounding)
  double E[3][3];
  E[0][0] = 1.0 - 0.5 * (w1 * w1 + w2 * w2);
  E[1][1] = 1.0 - 0.5 * (w0 * w0 + w2 * w2);
  E[2][2] = 1.0 - 0.5 * (w0 * w0 + w1 * w1);
  E[0][1] = -w2 + 0.5 * w0 * w1;
  E[1][0] = w2 + 0.5 * w0 * w1;
  E[0][2] = w1 + 0.5 * w0 * w2;
  E[2][0] = -w1 + 0.5 * w0 * w2;
  E[1][2] = -w0 + 0.5 * w1 * w2;
  E[2][1] = w0 + 0.5 * w1 * w2;
  matmul(R1, E, R);
}

}  // namespace fsim
