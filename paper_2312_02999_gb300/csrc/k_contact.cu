// IPC work on the proxy surface: s = W x (Sec. 3.1), UpdateConstraintSet,
// barrier energy (Eq. 3), PSD barrier Hessian mapped through W into the
// reduced block B-check (Eq. 10) and the additive-CCD step bound (Algorithm 1).
//
// Broad phase: all point-triangle and edge-edge pairs are swept in tiles;
// each primitive's box is rounded outward to float32 so that the float32
// overlap test keeps every pair the exact float64 test keeps.  The float64
// test (boxes inflated by dhat, closed intervals) then decides CCD candidates
// exactly as the oracle does, and the float64 distance decides d < dhat.
#include <algorithm>
#include <mutex>

#include "contact.cuh"
#include "kernels.h"
#include "../../include/fsim.h"

namespace fsim {

constexpr int kTile = 128;

__device__ __forceinline__ unsigned long long pack_key(int type, int i, int j) {
  return ((unsigned long long)type << 62) | ((unsigned long long)i << 31) | (unsigned long long)j;
}
__device__ __forceinline__ void unpack_key(unsigned long long k, int& type, int& i, int& j) {
  type = (int)(k >> 62);
  i = (int)((k >> 31) & 0x7fffffffULL);
  j = (int)(k & 0x7fffffffULL);
}

__device__ __forceinline__ void k_proxy_body(int Ns, const int64_t* __restrict__ Wptr, const int* __restrict__ Wcol,
                        const double* __restrict__ Wval, const double* __restrict__ x,
                        double* __restrict__ s) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Ns) return;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t e = Wptr[r]; e < Wptr[r + 1]; ++e) {
    const double wv = Wval[e];
    const double* xv = x + 3 * (size_t)Wcol[e];
    a += wv * xv[0]; b += wv * xv[1]; c += wv * xv[2];
  }
  s[3 * (size_t)r] = a; s[3 * (size_t)r + 1] = b; s[3 * (size_t)r + 2] = c;
}
__global__ void k_proxy(int Ns, const int64_t* __restrict__ Wptr, const int* __restrict__ Wcol,
                        const double* __restrict__ Wval, const double* __restrict__ x,
                        double* __restrict__ s) {
  k_proxy_body(Ns, Wptr, Wcol, Wval, x, s);
}

// float64 box of a primitive (1 vertex, a triangle or an edge) over s and,
// with ds, over s + ds as well
template <int NV>
__device__ __forceinline__ void prim_box(const double* s, const double* ds, const int* ids,
                                         double lo[3], double hi[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) { lo[d] = 1e300; hi[d] = -1e300; }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double* p = s + 3 * (size_t)ids[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], p[d]); hi[d] = fmax(hi[d], p[d]);
      if (ds != nullptr) {
        const double e = p[d] + ds[3 * (size_t)ids[k] + d];
        lo[d] = fmin(lo[d], e); hi[d] = fmax(hi[d], e);
      }
    }
  }
}

// exact float64 test of the oracle: [lo_a - pad, hi_a + pad] vs [lo_b, hi_b]
__device__ __forceinline__ bool box_overlap64(const double la[3], const double ha[3],
                                              const double lb[3], const double hb[3], double pad) {
  return (la[0] - pad <= hb[0]) && (lb[0] <= ha[0] + pad) && (la[1] - pad <= hb[1]) &&
         (lb[1] <= ha[1] + pad) && (la[2] - pad <= hb[2]) && (lb[2] <= ha[2] + pad);
}

struct Box32 {
  float lo[3], hi[3];
};

__device__ __forceinline__ Box32 to_box32(const double lo[3], const double hi[3], double pad) {
  Box32 b;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = __double2float_rd(lo[d] - pad);
    b.hi[d] = __double2float_ru(hi[d] + pad);
  }
  return b;
}

__device__ __forceinline__ bool box_overlap32(const Box32& a, const Box32& b) {
  return a.lo[0] <= b.hi[0] && b.lo[0] <= a.hi[0] && a.lo[1] <= b.hi[1] && b.lo[1] <= a.hi[1] &&
         a.lo[2] <= b.hi[2] && b.lo[2] <= a.hi[2];
}

__device__ __forceinline__ void load_pair(int type, int i, int j, const int* tris, const int* edges,
                                          int V[4]) {
  if (type == 0) {
    V[0] = i; V[1] = tris[3 * j]; V[2] = tris[3 * j + 1]; V[3] = tris[3 * j + 2];
  } else {
    V[0] = edges[2 * i]; V[1] = edges[2 * i + 1]; V[2] = edges[2 * j]; V[3] = edges[2 * j + 1];
  }
}

__device__ __forceinline__ void gather_X(const double* s, const int V[4], double X[4][3]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) X[k][d] = s[3 * (size_t)V[k] + d];
}

__device__ __forceinline__ void append(unsigned long long key, unsigned long long* out, int* count,
                                       int* overflow, int64_t cap) {
  const int idx = atomicAdd(count, 1);
  // unsigned compare: a count that wrapped past 2^31 appends is an overflow,
  // never a negative index
  if ((unsigned long long)(unsigned)idx < (unsigned long long)cap) out[idx] = key;
  else atomicOr(overflow, 1);
}

// CCD candidates of caller-owned buffers (fsim_ccd_noalloc): point-triangle
// and edge-edge pairs whose swept boxes (inflated by dhat) overlap by the
// exact float64 test, after a float32 box prefilter.
__global__ void __launch_bounds__(kTile)
k_cand_pt(int Ns, int Nt, const double* __restrict__ s, const double* __restrict__ ds,
          const int* __restrict__ tris, double dhat, unsigned long long* __restrict__ out,
          int* counters, int64_t cap) {
  __shared__ Box32 tb[kTile];
  __shared__ int tid3[kTile][3];
  const int t0 = blockIdx.y * kTile;
  for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
    const int t = t0 + k;
    tid3[k][0] = -1;
    if (t < Nt) {
      int ids[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
      // caller-owned indices: a triangle with a vertex outside [0, Ns) is
      // skipped and reported (counters[3]) instead of being read
      if ((unsigned)ids[0] >= (unsigned)Ns || (unsigned)ids[1] >= (unsigned)Ns ||
          (unsigned)ids[2] >= (unsigned)Ns) {
        atomicExch(counters + 3, 1);
        continue;
      }
      double lo[3], hi[3];
      prim_box<3>(s, ds, ids, lo, hi);
      tb[k] = to_box32(lo, hi, 0.0);
      tid3[k][0] = ids[0]; tid3[k][1] = ids[1]; tid3[k][2] = ids[2];
    }
  }
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= Ns) return;
  double vlo[3], vhi[3];
  prim_box<1>(s, ds, &v, vlo, vhi);
  const Box32 vb = to_box32(vlo, vhi, dhat);
  const int nt = min(kTile, Nt - t0);
  for (int k = 0; k < nt; ++k) {
    if (tid3[k][0] < 0) continue;
    if (!box_overlap32(vb, tb[k])) continue;
    const int a = tid3[k][0], b = tid3[k][1], c = tid3[k][2];
    if (a == v || b == v || c == v) continue;
    double tlo[3], thi[3];
    int ids[3] = {a, b, c};
    prim_box<3>(s, ds, ids, tlo, thi);
    if (box_overlap64(vlo, vhi, tlo, thi, dhat))
      append(pack_key(0, v, t0 + k), out, counters + 1, counters + 2, cap);
  }
}

__global__ void __launch_bounds__(kTile)
k_cand_ee(int Ns, int Ne, const double* __restrict__ s, const double* __restrict__ ds,
          const int* __restrict__ edges, double dhat, unsigned long long* __restrict__ out,
          int* counters, int64_t cap) {
  if (blockIdx.y < blockIdx.x) return;        // tiles with j-tile >= i-tile
  __shared__ Box32 eb[kTile];
  __shared__ int eid[kTile][2];
  const int j0 = blockIdx.y * kTile;
  for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
    const int e = j0 + k;
    eid[k][0] = -1;
    if (e < Ne) {
      int ids[2] = {edges[2 * e], edges[2 * e + 1]};
      // an edge with an endpoint outside [0, Ns) is skipped and reported
      if ((unsigned)ids[0] >= (unsigned)Ns || (unsigned)ids[1] >= (unsigned)Ns) {
        atomicExch(counters + 3, 1);
        continue;
      }
      double lo[3], hi[3];
      prim_box<2>(s, ds, ids, lo, hi);
      eb[k] = to_box32(lo, hi, 0.0);
      eid[k][0] = ids[0]; eid[k][1] = ids[1];
    }
  }
  __syncthreads();
  const int i = blockIdx.x * kTile + threadIdx.x;
  if (i >= Ne) return;
  const int ia[2] = {edges[2 * i], edges[2 * i + 1]};
  if ((unsigned)ia[0] >= (unsigned)Ns || (unsigned)ia[1] >= (unsigned)Ns) return;  // flagged above
  double ilo[3], ihi[3];
  prim_box<2>(s, ds, ia, ilo, ihi);
  const Box32 ib = to_box32(ilo, ihi, dhat);
  const int ne = min(kTile, Ne - j0);
  for (int k = 0; k < ne; ++k) {
    const int j = j0 + k;
    if (j <= i) continue;
    if (eid[k][0] < 0) continue;
    if (!box_overlap32(ib, eb[k])) continue;
    const int b0 = eid[k][0], b1 = eid[k][1];
    if (b0 == ia[0] || b0 == ia[1] || b1 == ia[0] || b1 == ia[1]) continue;
    double jlo[3], jhi[3];
    int ids[2] = {b0, b1};
    prim_box<2>(s, ds, ids, jlo, jhi);
    if (box_overlap64(ilo, ihi, jlo, jhi, dhat))
      append(pack_key(1, i, j), out, counters + 1, counters + 2, cap);
  }
}

// Pass A, one warp per pair (single frames: few pairs, so the latency of
// a pair's chain sets the time and the lanes share its Jacobi rotations and
// lift).  Per-pair gradient and PSD Hessian blocks (PositiveDefinite of
// Algorithm 1); marks the touched x2 vertices.  One warp per pair: the
// reduced (n <= 5) Hessian is built redundantly by every lane, each cyclic
// Jacobi rotation updates its rows, columns and eigenvectors lane-parallel,
// and the 144 block entries of the lift are spread over the lanes.  ET is the
// type of the small eigen-solve (float64, or float32 in the mixed form).
// One pair-warp per CTA: the float64 geometry of a pair is a long chain of
// float64 instructions, and an SM's float64 pipe is narrow on this part, so
// the pairs are spread over as many SMs as possible.
constexpr int kPairWarps = 1;

template <typename ET>
__device__ __forceinline__ void k_barrier_pairs_warp_body(const int* __restrict__ count, int64_t cap, const unsigned long long* __restrict__ pairs,
                const double* __restrict__ s, const int* __restrict__ tris,
                const int* __restrict__ edges, const int64_t* __restrict__ Wptr,
                const int* __restrict__ Wcol, const int* __restrict__ x2of, double dhat,
                double kappa, double* __restrict__ pgrad, double* __restrict__ phess,
                int* __restrict__ x2mark) {
  __shared__ ET As[kPairWarps][5][5];
  __shared__ ET Qs[kPairWarps][5][5];
  __shared__ double Hp[kPairWarps][5][5];
  __shared__ double hv[kPairWarps][4][3];
  __shared__ double sq[kPairWarps][4][4];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t np = *count;
  np = np < cap ? np : cap;
  for (int64_t p = blockIdx.x * (int64_t)kPairWarps + w; p < np;
       p += (int64_t)gridDim.x * kPairWarps) {
    int type, i, j;
    unpack_key(pairs[p], type, i, j);
    int V[4];
    load_pair(type, i, j, tris, edges, V);
    double X[4][3];
    gather_X(s, V, X);
    PairReduced r;
    pair_reduced(type, X, dhat, kappa, r);
    const int n = r.n;
    if (lane < 25) {
      const int a = lane / 5, b = lane % 5;
      As[w][a][b] = (ET)r.A[a][b];
      Qs[w][a][b] = a == b ? ET(1) : ET(0);
    }
    __syncwarp();
    const ET tiny = sizeof(ET) == 8 ? ET(1e-300) : ET(1e-30);
    const ET tol = sizeof(ET) == 8 ? ET(1e-30) : ET(1e-13);
    for (int sweep = 0; sweep < 12; ++sweep) {
      ET off = 0, dia = 0;
      for (int a = 0; a < n; ++a) {
        dia += As[w][a][a] * As[w][a][a];
        for (int b = a + 1; b < n; ++b) off += As[w][a][b] * As[w][a][b];
      }
      if (!(off > tol * dia)) break;
      for (int pp = 0; pp < n - 1; ++pp)
        for (int qq = pp + 1; qq < n; ++qq) {
          const ET apq = As[w][pp][qq];
          if (!(fabs(apq) > tiny)) continue;
          const ET app = As[w][pp][pp], aqq = As[w][qq][qq];
          const ET th = (aqq - app) / (ET(2) * apq);
          const ET t = (th >= ET(0) ? ET(1) : ET(-1)) / (fabs(th) + sqrt(th * th + ET(1)));
          const ET c = ET(1) / sqrt(t * t + ET(1)), sn = t * c;
          ET x0 = 0, x1 = 0;
          const bool rowl = lane < n && lane != pp && lane != qq;
          const bool qlan = lane >= 8 && lane < 8 + n;
          if (rowl) { x0 = As[w][lane][pp]; x1 = As[w][lane][qq]; }
          if (qlan) { x0 = Qs[w][lane - 8][pp]; x1 = Qs[w][lane - 8][qq]; }
          __syncwarp();
          if (rowl) {
            const ET np_ = c * x0 - sn * x1, nq = sn * x0 + c * x1;
            As[w][lane][pp] = np_; As[w][pp][lane] = np_;
            As[w][lane][qq] = nq; As[w][qq][lane] = nq;
          }
          if (qlan) {
            Qs[w][lane - 8][pp] = c * x0 - sn * x1;
            Qs[w][lane - 8][qq] = sn * x0 + c * x1;
          }
          if (lane == 16) As[w][pp][pp] = app - t * apq;
          if (lane == 17) As[w][qq][qq] = aqq + t * apq;
          if (lane == 18) { As[w][pp][qq] = ET(0); As[w][qq][pp] = ET(0); }
          __syncwarp();
        }
    }
    // projection: keep eigenvalues above a relative floor (zero in float64;
    // float32 rounding noise of the largest one in the mixed form)
    ET lmax = 0;
    for (int a = 0; a < n; ++a) lmax = fmax(lmax, As[w][a][a]);
    const ET floor_ = sizeof(ET) == 8 ? ET(0) : ET(1e-6) * lmax;
    if (lane < 25) {
      const int a = lane / 5, b = lane % 5;
      double acc = 0.0;
      if (a < n && b < n)
        for (int l = 0; l < n; ++l) {
          const ET lam = As[w][l][l];
          if (lam > floor_) acc += (double)Qs[w][a][l] * (double)lam * (double)Qs[w][b][l];
        }
      Hp[w][a][b] = acc;
    }
    __syncwarp();
    const int k = r.k;
    if (lane < 12) {                  // hv[i][a] = sum_m q_m[i] Hp[a][3+m]
      const int ii = lane / 3, a = lane % 3;
      double acc = 0.0;
      for (int m = 0; m < k; ++m) acc += r.q[m][ii] * Hp[w][a][3 + m];
      hv[w][ii][a] = acc;
    } else if (lane < 28) {           // sq[i][j] = sum q_m[i] q_l[j] Hp[3+m][3+l]
      const int ii = (lane - 12) / 4, jj = (lane - 12) % 4;
      double acc = 0.0;
      for (int m = 0; m < k; ++m)
        for (int l = 0; l < k; ++l) acc += r.q[m][ii] * r.q[l][jj] * Hp[w][3 + m][3 + l];
      sq[w][ii][jj] = acc;
    }
    __syncwarp();
    if (lane < 12) pgrad[p * 12 + lane] = r.gfac * r.c[lane / 3] * r.vh[lane % 3];
    for (int e = lane; e < 144; e += 32) {
      const int ab = e / 9, rc = e % 9;
      const int ii = ab / 4, jj = ab % 4, a = rc / 3, b = rc % 3;
      phess[p * 144 + e] = r.ch[ii] * r.ch[jj] * Hp[w][a][b] + r.ch[ii] * hv[w][jj][a] * r.vh[b] +
                           r.ch[jj] * r.vh[a] * hv[w][ii][b] + sq[w][ii][jj] * r.vh[a] * r.vh[b];
    }
    if (lane < 4)
      for (int64_t e = Wptr[V[lane]]; e < Wptr[V[lane] + 1]; ++e) {
        const int q = x2of[Wcol[e]];
        if (q >= 0) x2mark[q] = 1;
      }
    __syncwarp();
  }
}

// Pass A: per-pair gradient and PSD Hessian blocks (PositiveDefinite of
// Algorithm 1); marks the touched x2 vertices.  One lane per pair: the
// distance, barrier and pair Hessian in a reduced basis of <= 5 coordinates
// (float64), a cyclic Jacobi eigen-solve of that <= 5 x 5 matrix in
// registers (ET: float64, or float32 in the mixed form), the projection, and
// the lift to the 12 gradient entries and 144 Hessian entries.  GB300 issues
// a warp-wide float64 instruction about every 64 cycles per SM
// sub-partition, so the float64 geometry costs per warp instruction: with a
// pair per lane one instruction serves 32 pairs (the warp-per-pair form
// spends it on one).  This is the form for batches, whose frames together
// have thousands of pairs; a single frame's hundred or so pairs finish sooner
// with a warp per pair, whose lanes share a pair's rotations and lift.  One
// warp per CTA spreads the pairs over as many SMs as possible.
constexpr int kPairLanes = 32;

template <typename ET>
__device__ __forceinline__ void barrier_pair_lane(int64_t p, const unsigned long long* __restrict__ pairs,
                const double* __restrict__ s, const int* __restrict__ tris,
                const int* __restrict__ edges, const int64_t* __restrict__ Wptr,
                const int* __restrict__ Wcol, const int* __restrict__ x2of, double dhat,
                double kappa, double* __restrict__ pgrad, double* __restrict__ phess,
                int* __restrict__ x2mark) {
  int type, i, j;
  unpack_key(pairs[p], type, i, j);
  int V[4];
  load_pair(type, i, j, tris, edges, V);
  double X[4][3];
  gather_X(s, V, X);
  PairReduced r;
  pair_reduced(type, X, dhat, kappa, r);
  const int n = r.n;
  ET A[5][5], Q[5][5];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      A[a][b] = (a < n && b < n) ? (ET)r.A[a][b] : ET(0);
      Q[a][b] = a == b ? ET(1) : ET(0);
    }
  const ET tiny = sizeof(ET) == 8 ? ET(1e-300) : ET(1e-30);
  const ET tol = sizeof(ET) == 8 ? ET(1e-30) : ET(1e-13);
  for (int sweep = 0; sweep < 12; ++sweep) {
    ET off = 0, dia = 0;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      if (a < n) dia += A[a][a] * A[a][a];
#pragma unroll
      for (int b = a + 1; b < 5; ++b)
        if (b < n) off += A[a][b] * A[a][b];
    }
    if (!(off > tol * dia)) break;
#pragma unroll
    for (int pp = 0; pp < 4; ++pp)
#pragma unroll
      for (int qq = pp + 1; qq < 5; ++qq) {
        if (qq >= n) continue;
        const ET apq = A[pp][qq];
        if (!(fabs(apq) > tiny)) continue;
        const ET app = A[pp][pp], aqq = A[qq][qq];
        const ET th = (aqq - app) / (ET(2) * apq);
        const ET t = (th >= ET(0) ? ET(1) : ET(-1)) / (fabs(th) + sqrt(th * th + ET(1)));
        const ET c = ET(1) / sqrt(t * t + ET(1)), sn = t * c;
#pragma unroll
        for (int l = 0; l < 5; ++l) {
          if (l == pp || l == qq || l >= n) continue;
          const ET x0 = A[l][pp], x1 = A[l][qq];
          const ET np_ = c * x0 - sn * x1, nq = sn * x0 + c * x1;
          A[l][pp] = np_; A[pp][l] = np_;
          A[l][qq] = nq; A[qq][l] = nq;
        }
#pragma unroll
        for (int l = 0; l < 5; ++l) {
          if (l >= n) continue;
          const ET x0 = Q[l][pp], x1 = Q[l][qq];
          Q[l][pp] = c * x0 - sn * x1;
          Q[l][qq] = sn * x0 + c * x1;
        }
        A[pp][pp] = app - t * apq;
        A[qq][qq] = aqq + t * apq;
        A[pp][qq] = ET(0); A[qq][pp] = ET(0);
      }
  }
  // projection: keep eigenvalues above a relative floor (zero in float64;
  // float32 rounding noise of the largest one in the mixed form)
  ET lmax = 0;
#pragma unroll
  for (int a = 0; a < 5; ++a)
    if (a < n) lmax = fmax(lmax, A[a][a]);
  const ET floor_ = sizeof(ET) == 8 ? ET(0) : ET(1e-6) * lmax;
  double Hp[5][5];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      double acc = 0.0;
      if (a < n && b < n)
#pragma unroll
        for (int l = 0; l < 5; ++l) {
          if (l >= n) continue;
          const ET lam = A[l][l];
          if (lam > floor_) acc += (double)Q[a][l] * (double)lam * (double)Q[b][l];
        }
      Hp[a][b] = acc;
    }
  const int k = r.k;
  double hv[4][3], sq[4][4];        // hv[i][a] = sum_m q_m[i] Hp[a][3+m]
#pragma unroll
  for (int ii = 0; ii < 4; ++ii) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 2; ++m)
        if (m < k) acc += r.q[m][ii] * Hp[a][3 + m];
      hv[ii][a] = acc;
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {  // sq[i][j] = sum q_m[i] q_l[j] Hp[3+m][3+l]
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int l = 0; l < 2; ++l)
          if (m < k && l < k) acc += r.q[m][ii] * r.q[l][jj] * Hp[3 + m][3 + l];
      sq[ii][jj] = acc;
    }
  }
#pragma unroll
  for (int e = 0; e < 12; ++e) pgrad[p * 12 + e] = r.gfac * r.c[e / 3] * r.vh[e % 3];
  // block (i, j) entry (a, b) of the lift, factored so that a lane's float64
  // operations fall from about 1,440 to about 540:
  //   ch_i (ch_j Hp[a][b] + hv[j][a] vh[b]) + vh[a] (ch_j hv[i][b] + sq[i][j] vh[b])
  double T1[4][3][3];
#pragma unroll
  for (int jj = 0; jj < 4; ++jj)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) T1[jj][a][b] = r.ch[jj] * Hp[a][b] + hv[jj][a] * r.vh[b];
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      double T2[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) T2[b] = r.ch[jj] * hv[ii][b] + sq[ii][jj] * r.vh[b];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          phess[p * 144 + (ii * 4 + jj) * 9 + a * 3 + b] =
              r.ch[ii] * T1[jj][a][b] + r.vh[a] * T2[b];
    }
#pragma unroll
  for (int a = 0; a < 4; ++a)
    for (int64_t e = Wptr[V[a]]; e < Wptr[V[a] + 1]; ++e) {
      const int q = x2of[Wcol[e]];
      if (q >= 0) x2mark[q] = 1;
    }
}

template <typename ET>
__device__ __forceinline__ void k_barrier_pairs_body(const int* __restrict__ count, int64_t cap, const unsigned long long* __restrict__ pairs,
                const double* __restrict__ s, const int* __restrict__ tris,
                const int* __restrict__ edges, const int64_t* __restrict__ Wptr,
                const int* __restrict__ Wcol, const int* __restrict__ x2of, double dhat,
                double kappa, double* __restrict__ pgrad, double* __restrict__ phess,
                int* __restrict__ x2mark) {
  int64_t np = *count;
  np = np < cap ? np : cap;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x)
    barrier_pair_lane<ET>(p, pairs, s, tris, edges, Wptr, Wcol, x2of, dhat, kappa, pgrad, phess,
                          x2mark);
}
template <typename ET>
__global__ void __launch_bounds__(kPairLanes) k_barrier_pairs_lanes(const int* __restrict__ count, int64_t cap, const unsigned long long* __restrict__ pairs,
                const double* __restrict__ s, const int* __restrict__ tris,
                const int* __restrict__ edges, const int64_t* __restrict__ Wptr,
                const int* __restrict__ Wcol, const int* __restrict__ x2of, double dhat,
                double kappa, double* __restrict__ pgrad, double* __restrict__ phess,
                int* __restrict__ x2mark) {
  k_barrier_pairs_body<ET>(count, cap, pairs, s, tris, edges, Wptr, Wcol, x2of, dhat, kappa, pgrad, phess, x2mark);
}
template <typename ET>
__global__ void __launch_bounds__(32 * kPairWarps) k_barrier_pairs(const int* __restrict__ count, int64_t cap, const unsigned long long* __restrict__ pairs,
                const double* __restrict__ s, const int* __restrict__ tris,
                const int* __restrict__ edges, const int64_t* __restrict__ Wptr,
                const int* __restrict__ Wcol, const int* __restrict__ x2of, double dhat,
                double kappa, double* __restrict__ pgrad, double* __restrict__ phess,
                int* __restrict__ x2mark) {
  k_barrier_pairs_warp_body<ET>(count, cap, pairs, s, tris, edges, Wptr, Wcol, x2of, dhat, kappa, pgrad, phess, x2mark);
}

// Edge-edge mollifier (optional): for EE pairs with c = |e_a x e_b|^2 below
// eps = 1e-3 |E_a|^2 |E_b|^2 the pair term is kappa m(c) b(d); this pass
// overwrites those pairs' gradient and Hessian blocks written by
// k_barrier_pairs.  The 12 x 12 Hessian
//   m H_b + kappa b (m'' grad c grad c^T + m' hess c) + m' (grad c G^T + G grad c^T)
// (H_b, G: kappa b's Hessian and gradient, lifted from the reduced basis) is
// projected onto the PSD cone by a cyclic Jacobi eigen-solve in float64 (one
// warp per pair, lane-parallel rotations), whatever the precision.
__device__ __forceinline__ void k_mollify_ee_body(const int* __restrict__ count, int64_t cap,
                                                   const unsigned long long* __restrict__ pairs,
                                                   const double* __restrict__ s,
                                                   const int* __restrict__ edges,
                                                   const double* __restrict__ elen2, double dhat,
                                                   double kappa, double* __restrict__ pgrad,
                                                   double* __restrict__ phess) {
  __shared__ double As[12][13];
  __shared__ double Qs[12][13];
  __shared__ double gcs[12], Gs[12];
  const int lane = threadIdx.x;
  int64_t np = *count;
  np = np < cap ? np : cap;
  for (int64_t p = blockIdx.x; p < np; p += gridDim.x) {
    int type, i, j;
    unpack_key(pairs[p], type, i, j);
    if (type != 1) continue;
    const double eps = FSIM_MOLLIFIER_EPS_SCALE * elen2[i] * elen2[j];
    int V[4];
    load_pair(type, i, j, nullptr, edges, V);
    double X[4][3];
    gather_X(s, V, X);
    EdgeCross ec;
    edge_cross(X, ec);
    if (!(ec.c < eps)) continue;                  // warp-uniform
    PairReduced r;
    pair_reduced(1, X, dhat, kappa, r);
    const double u = r.d - dhat;
    const double kb = kappa * (-u * u * log(r.d / dhat));
    const double q = ec.c / eps;
    const double m0 = (2.0 - q) * q, m1 = (2.0 - 2.0 * q) / eps, m2 = -2.0 / (eps * eps);
    if (lane < 12) {
      const int I = lane / 3, al = lane % 3;
      gcs[lane] = edge_cross_grad(ec, I, al);
      Gs[lane] = r.gfac * r.c[I] * r.vh[al];
    }
    __syncwarp();
    if (lane < 12) pgrad[p * 12 + lane] = m0 * Gs[lane] + kb * m1 * gcs[lane];
    for (int e = lane; e < 144; e += 32) {
      const int a = e / 12, b = e % 12;
      const int I = a / 3, al = a % 3, J = b / 3, be = b % 3;
      double bp[5], bq[5];
      for (int t = 0; t < 3; ++t) {
        bp[t] = (al == t) ? r.ch[I] : 0.0;
        bq[t] = (be == t) ? r.ch[J] : 0.0;
      }
      for (int t = 0; t < 2; ++t) {
        bp[3 + t] = r.q[t][I] * r.vh[al];
        bq[3 + t] = r.q[t][J] * r.vh[be];
      }
      double hb = 0.0;
      for (int x = 0; x < r.n; ++x)
        for (int y = 0; y < r.n; ++y) hb += bp[x] * r.A[x][y] * bq[y];
      As[a][b] = m0 * hb + kb * (m2 * gcs[a] * gcs[b] + m1 * edge_cross_hess(ec, I, al, J, be)) +
                 m1 * (gcs[a] * Gs[b] + Gs[a] * gcs[b]);
      Qs[a][b] = (a == b) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int sweep = 0; sweep < 30; ++sweep) {
      double off = 0.0, dia = 0.0;
      for (int a = 0; a < 12; ++a) {
        dia += As[a][a] * As[a][a];
        for (int b = a + 1; b < 12; ++b) off += As[a][b] * As[a][b];
      }
      if (!(off > 1e-30 * dia)) break;
      for (int pp = 0; pp < 11; ++pp)
        for (int qq = pp + 1; qq < 12; ++qq) {
          const double apq = As[pp][qq];
          if (!(fabs(apq) > 1e-300)) continue;
          const double app = As[pp][pp], aqq = As[qq][qq];
          const double th = (aqq - app) / (2.0 * apq);
          const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
          double x0 = 0.0, x1 = 0.0;
          const bool rowl = lane < 12 && lane != pp && lane != qq;
          const bool qlan = lane >= 16 && lane < 28;
          if (rowl) { x0 = As[lane][pp]; x1 = As[lane][qq]; }
          if (qlan) { x0 = Qs[lane - 16][pp]; x1 = Qs[lane - 16][qq]; }
          __syncwarp();
          if (rowl) {
            const double np_ = c * x0 - sn * x1, nq = sn * x0 + c * x1;
            As[lane][pp] = np_; As[pp][lane] = np_;
            As[lane][qq] = nq; As[qq][lane] = nq;
          }
          if (qlan) {
            Qs[lane - 16][pp] = c * x0 - sn * x1;
            Qs[lane - 16][qq] = sn * x0 + c * x1;
          }
          if (lane == 12) As[pp][pp] = app - t * apq;
          if (lane == 13) As[qq][qq] = aqq + t * apq;
          if (lane == 14) { As[pp][qq] = 0.0; As[qq][pp] = 0.0; }
          __syncwarp();
        }
    }
    for (int e = lane; e < 144; e += 32) {
      const int a = e / 12, b = e % 12;
      double acc = 0.0;
      for (int l = 0; l < 12; ++l) {
        const double lam = As[l][l];
        if (lam > 0.0) acc += Qs[a][l] * lam * Qs[b][l];
      }
      const int I = a / 3, al = a % 3, J = b / 3, be = b % 3;
      phess[p * 144 + (I * 4 + J) * 9 + al * 3 + be] = acc;
    }
    __syncwarp();
  }
}
__global__ void __launch_bounds__(32) k_mollify_ee(const int* __restrict__ count, int64_t cap,
                                                   const unsigned long long* __restrict__ pairs,
                                                   const double* __restrict__ s,
                                                   const int* __restrict__ edges,
                                                   const double* __restrict__ elen2, double dhat,
                                                   double kappa, double* __restrict__ pgrad,
                                                   double* __restrict__ phess) {
  k_mollify_ee_body(count, cap, pairs, s, edges, elen2, dhat, kappa, pgrad, phess);
}

// x2mark (0/1 flags) -> x2mark[q] = c position + 1 (0 if untouched); clist; nc.
__device__ __forceinline__ void k_mark_scan_body(int n2, int* __restrict__ x2mark, int* __restrict__ clist,
                            int* __restrict__ counters) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n2; base += blockDim.x) {
    const int q = base + threadIdx.x;
    const int f = (q < n2) ? (x2mark[q] != 0) : 0;
    int incl = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    const int before = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + incl - f;
    if (q < n2) {
      if (f) { x2mark[q] = before + 1; clist[before] = q; }
      else x2mark[q] = 0;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + f;
    __syncthreads();
  }
  if (threadIdx.x == 0) counters[3] = carry;
}
__global__ void k_mark_scan(int n2, int* __restrict__ x2mark, int* __restrict__ clist,
                            int* __restrict__ counters) {
  k_mark_scan_body(n2, x2mark, clist, counters);
}

// Pass C: scatter gradients (through W) into g and blocks into B-check.
// One thread per (pair, a, b): the pair's 12 x 12 block (a, b) mapped through
// the W rows of its vertices a and b into B-check, and (b == 0) vertex a's
// gradient into g.  n_c is read on the device; B-check is written only when
// it fits the reduced buffers (n_c <= nc_cap), else the host grows them and
// scatters the Hessian blocks again.  mode: 1 gradient, 2 B-check, 3 both.
__device__ __forceinline__ void k_barrier_scatter_body(int64_t np, const unsigned long long* __restrict__ pairs,
                                  const int* __restrict__ tris, const int* __restrict__ edges,
                                  const int64_t* __restrict__ Wptr, const int* __restrict__ Wcol,
                                  const double* __restrict__ Wval, const int* __restrict__ x2of,
                                  const int* __restrict__ x2mark, const double* __restrict__ pgrad,
                                  const double* __restrict__ phess, const int* __restrict__ ncp,
                                  int nc_cap, int mode, double* __restrict__ g,
                                  double* __restrict__ Bc, int* __restrict__ bocc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p = t >> 4;
  if (p >= np) return;
  const int a = (int)((t >> 2) & 3), b = (int)(t & 3);
  const int nc = *ncp;
  const bool grad = (mode & 1) && b == 0;
  const bool hess = (mode & 2) && nc <= nc_cap;
  if (!grad && !hess) return;
  int type, i, j;
  unpack_key(pairs[p], type, i, j);
  int V[4];
  load_pair(type, i, j, tris, edges, V);
  const int ld = 3 * nc;
  for (int64_t ea = Wptr[V[a]]; ea < Wptr[V[a] + 1]; ++ea) {
    const int va = Wcol[ea];
    const int qa = x2of[va];
    if (qa < 0) continue;                         // pinned: no DOF
    const double wa = Wval[ea];
    if (grad)
      for (int d = 0; d < 3; ++d) atomicAdd(g + 3 * (size_t)va + d, wa * pgrad[p * 12 + 3 * a + d]);
    if (!hess) continue;
    const int ca = x2mark[qa] - 1;
    if (ca < 0 || ca >= nc) continue;
    for (int64_t eb = Wptr[V[b]]; eb < Wptr[V[b] + 1]; ++eb) {
      const int qb = x2of[Wcol[eb]];
      if (qb < 0) continue;
      const int cb = x2mark[qb] - 1;
      if (cb < 0 || cb >= nc) continue;
      const double ww = wa * Wval[eb];
      const double* h = phess + p * 144 + (a * 4 + b) * 9;
      double* dst = Bc + (size_t)(3 * ca) * ld + 3 * cb;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) atomicAdd(dst + (size_t)r * ld + c, ww * h[3 * r + c]);
      bocc[(size_t)ca * nc + cb] = 1;
    }
  }
}
__global__ void k_barrier_scatter(int64_t np, const unsigned long long* __restrict__ pairs,
                                  const int* __restrict__ tris, const int* __restrict__ edges,
                                  const int64_t* __restrict__ Wptr, const int* __restrict__ Wcol,
                                  const double* __restrict__ Wval, const int* __restrict__ x2of,
                                  const int* __restrict__ x2mark, const double* __restrict__ pgrad,
                                  const double* __restrict__ phess, const int* __restrict__ ncp,
                                  int nc_cap, int mode, double* __restrict__ g,
                                  double* __restrict__ Bc, int* __restrict__ bocc) {
  k_barrier_scatter_body(np, pairs, tris, edges, Wptr, Wcol, Wval, x2of, x2mark, pgrad, phess, ncp, nc_cap, mode, g, Bc, bocc);
}

// Zero the first (3 n_c)^2 entries of B-check and n_c^2 of its block
// occupancy, n_c read on the device (nothing when n_c > nc_cap).
__device__ __forceinline__ void k_zero_reduced_body(const int* __restrict__ ncp, int nc_cap, double* __restrict__ Bc,
                               int* __restrict__ bocc) {
  const int nc = *ncp;
  if (nc <= 0 || nc > nc_cap) return;
  const int64_t nb = 9 * (int64_t)nc * nc, no = (int64_t)nc * nc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nb; e += stride) Bc[e] = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < no; e += stride) bocc[e] = 0;
}
__global__ void k_zero_reduced(const int* __restrict__ ncp, int nc_cap, double* __restrict__ Bc,
                               int* __restrict__ bocc) {
  k_zero_reduced_body(ncp, nc_cap, Bc, bocc);
}

// Additive CCD (Li, Kaufman & Jiang 2021) time of impact of one candidate.
__device__ double accd_toi(int type, double X[4][3], double dX[4][3], double s_ratio, int max_iters) {
  double mean[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) mean[d] = (((dX[0][d] + dX[1][d]) + dX[2][d]) + dX[3][d]) / 4.0;
  double nrm[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int d = 0; d < 3; ++d) dX[k][d] -= mean[d];
    nrm[k] = sqrt((dX[k][0] * dX[k][0] + dX[k][1] * dX[k][1]) + dX[k][2] * dX[k][2]);
  }
  const double lp = type == 1 ? fmax(nrm[0], nrm[1]) + fmax(nrm[2], nrm[3])
                              : nrm[0] + fmax(fmax(nrm[1], nrm[2]), nrm[3]);
  if (!(lp > 0.0)) return 1.0;
  {
    // The first advance is (1 - s) d0 / lp; when it already passes t = 1 the
    // answer is "no impact".  Decided in float32 only with a 0.1% margin, so
    // the float64 march would take the same branch.
    float Xf[4][3];
    to_rel_f(X, Xf);
    const double df = (double)pair_distance_f(type, Xf);
    if ((1.0 - s_ratio) * df * (1.0 - 1e-3) > lp * (1.0 + 1e-3)) return 1.0;
  }
  const double d0 = pair_distance(type, X);
  const double gap = s_ratio * d0;
  double t = 0.0;
  double step = (1.0 - s_ratio) * d0 / lp;
  for (int it = 0; it < max_iters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int d = 0; d < 3; ++d) X[k][d] += step * dX[k][d];
    const double d = pair_distance(type, X);
    if (t > 0.0 && d < gap) return t;
    t += step;
    if (t > 1.0) return 1.0;
    step = 0.9 * d / lp;
  }
  return fmin(t, 1.0);
}

// ---------------------------------------------------------------------------
// Broad phase with per-primitive data prepared once per call.  Primitive
// index space: vertices [0, Ns), triangles [Ns, Ns+Nt), edges [Ns+Nt, ..).
// Per primitive: float32 boxes rounded outward (inflated by pad, and plain)
// and the exact float64 bounds as order-preserving 64-bit keys, so that the
// inner loops are float32 and integer only.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long order_key(double v) {
  // +0.0 for -0.0, then flip so that unsigned order equals float64 order
  const unsigned long long u = (unsigned long long)__double_as_longlong(v + 0.0);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}

// The same key from the bits alone (-0.0 mapped to +0.0 by comparison, not
// by a float64 addition), and its inverse.  GB300 runs float64 compares,
// min / max and additions on its narrow float64 pipe, so the boxes take their
// min / max on the keys (integer pipe) and convert back once.
__device__ __forceinline__ unsigned long long order_key_bits(double v) {
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
  if (u == 0x8000000000000000ULL) u = 0;
  return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k;
  return __longlong_as_double((long long)u);
}

__device__ __forceinline__ void k_prim_prep_body(int Ns, int Nt, int Ne, const double* __restrict__ s,
                            const double* __restrict__ ds, const int* __restrict__ tris,
                            const int* __restrict__ edges, double pad, float* __restrict__ box,
                            unsigned long long* __restrict__ key, float* __restrict__ sf,
                            float* __restrict__ dsf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ns + Nt + Ne) return;
  int ids[3];
  int nv;
  if (p < Ns) { ids[0] = p; nv = 1; }
  else if (p < Ns + Nt) { const int t = p - Ns; ids[0] = tris[3 * t]; ids[1] = tris[3 * t + 1]; ids[2] = tris[3 * t + 2]; nv = 3; }
  else { const int e = p - Ns - Nt; ids[0] = edges[2 * e]; ids[1] = edges[2 * e + 1]; nv = 2; }
  unsigned long long klo[3] = {~0ULL, ~0ULL, ~0ULL}, khi[3] = {0ULL, 0ULL, 0ULL};
  for (int k = 0; k < nv; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double x = s[3 * (size_t)ids[k] + d];
      const unsigned long long kx = order_key_bits(x);
      klo[d] = min(klo[d], kx); khi[d] = max(khi[d], kx);
      if (ds != nullptr) {
        const unsigned long long ke = order_key_bits(x + ds[3 * (size_t)ids[k] + d]);
        klo[d] = min(klo[d], ke); khi[d] = max(khi[d], ke);
      }
    }
  float* b = box + 12 * (size_t)p;
  unsigned long long* kk = key + 12 * (size_t)p;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double lo = key_value(klo[d]), hi = key_value(khi[d]);
    const double la = lo - pad, ha = hi + pad;          // same rounding as the oracle's test
    b[d] = __double2float_rd(la);
    b[3 + d] = __double2float_ru(ha);
    b[6 + d] = __double2float_rd(lo);
    b[9 + d] = __double2float_ru(hi);
    kk[d] = order_key_bits(la);
    kk[3 + d] = order_key_bits(ha);
    kk[6 + d] = klo[d];
    kk[9 + d] = khi[d];
  }
  if (p < Ns) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      sf[3 * (size_t)p + d] = (float)s[3 * (size_t)p + d];
      if (dsf != nullptr) dsf[3 * (size_t)p + d] = (float)ds[3 * (size_t)p + d];
    }
  }
}
__global__ void k_prim_prep(int Ns, int Nt, int Ne, const double* __restrict__ s,
                            const double* __restrict__ ds, const int* __restrict__ tris,
                            const int* __restrict__ edges, double pad, float* __restrict__ box,
                            unsigned long long* __restrict__ key, float* __restrict__ sf,
                            float* __restrict__ dsf) {
  k_prim_prep_body(Ns, Nt, Ne, s, ds, tris, edges, pad, box, key, sf, dsf);
}

struct Box6 {
  float v[6];   // lo[3], hi[3]
};

__device__ __forceinline__ bool ov32(const float* a, const float* b) {   // a inflated, b plain
  return a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] && b[1] <= a[4] && a[2] <= b[5] && b[2] <= a[5];
}

__device__ __forceinline__ bool ov64(const unsigned long long* a, const unsigned long long* b) {
  return a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] && b[1] <= a[4] && a[2] <= b[5] && b[2] <= a[5];
}

__device__ __forceinline__ void gather_Xf(const float* sf, const int V[4], float X[4][3]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) X[k][d] = sf[3 * (size_t)V[k] + d];
}

// Tile-pair culling for the all-pairs sweeps: every thread of a kTile block
// contributes its i-side box (inflated, `a`; empty if out of range) and the
// j-tile box it staged (plain, `b`; empty if out of range); the block's
// unions are compared, and a tile pair whose unions do not overlap holds no
// overlapping pair (ov32 per axis), so the block may skip it.  Every thread
// of the block must call this.
__device__ __forceinline__ bool tile_pair_overlaps(const float* a, const float* b) {
  __shared__ float red[kTile / 32][12];
  float u[12];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    u[q] = a[q]; u[3 + q] = a[3 + q]; u[6 + q] = b[q]; u[9 + q] = b[3 + q];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const float w = __shfl_xor_sync(0xffffffffu, u[q], o);
      u[q] = (q % 6) < 3 ? fminf(u[q], w) : fmaxf(u[q], w);
    }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 12; ++q) red[wid][q] = u[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 12; ++q) {
    float r = red[0][q];
    for (int w = 1; w < kTile / 32; ++w) r = (q % 6) < 3 ? fminf(r, red[w][q]) : fmaxf(r, red[w][q]);
    u[q] = r;
  }
  return ov32(u, u + 6);
}

struct SweepArgs {
  int Ns, Nt, Ne;
  const float* box;
  const unsigned long long* key;
  const float* sf;
  const int* tris;
  const int* edges;
  float near;                   // float32 distance below which a pair is kept (MODE 0)
  unsigned long long* out;
  int* count;
  int* overflow;
  int64_t cap;
  const int* gate;              // if set, the sweep runs only when *gate != 0
};

// MODE 0: pairs whose float32 distance is within `near` (a superset of the
// d < dhat pairs; decided in float64 by k_near_pairs).  MODE 1: CCD
// candidates, whose swept boxes (+dhat) overlap by the exact float64 test.
// (The skin list is built with MODE 0 and a wider `near`.)
template <int MODE>
__device__ __forceinline__ void k_sweep_pt_body(SweepArgs a) {
  if (a.gate && *a.gate == 0) return;
  __shared__ float tb[kTile][6];
  __shared__ int tid3[kTile][3];
  __shared__ unsigned long long tk[MODE == 1 ? kTile : 1][6];
  const int t0 = blockIdx.y * kTile;
  for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
    const int t = t0 + k;
    if (t < a.Nt) {
      const float* b = a.box + 12 * (size_t)(a.Ns + t) + 6;
#pragma unroll
      for (int q = 0; q < 6; ++q) tb[k][q] = b[q];
      tid3[k][0] = a.tris[3 * t]; tid3[k][1] = a.tris[3 * t + 1]; tid3[k][2] = a.tris[3 * t + 2];
      if (MODE == 1) {
        const unsigned long long* kk = a.key + 12 * (size_t)(a.Ns + t) + 6;
#pragma unroll
        for (int q = 0; q < 6; ++q) tk[k][q] = kk[q];
      }
    }
  }
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  float vb[6], tbk[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float e = q < 3 ? INFINITY : -INFINITY;     // empty box
    vb[q] = v < a.Ns ? a.box[12 * (size_t)v + q] : e;
    tbk[q] = t0 + (int)threadIdx.x < a.Nt ? tb[threadIdx.x][q] : e;
  }
  if (!tile_pair_overlaps(vb, tbk)) return;
  if (v >= a.Ns) return;
  unsigned long long vk[6];
  if (MODE == 1) {
#pragma unroll
    for (int q = 0; q < 6; ++q) vk[q] = a.key[12 * (size_t)v + q];
  }
  const int nt = min(kTile, a.Nt - t0);
  for (int k = 0; k < nt; ++k) {
    if (!ov32(vb, tb[k])) continue;
    const int p0 = tid3[k][0], p1 = tid3[k][1], p2 = tid3[k][2];
    if (p0 == v || p1 == v || p2 == v) continue;
    if (MODE == 1) {
      if (ov64(vk, tk[k])) append(pack_key(0, v, t0 + k), a.out, a.count, a.overflow, a.cap);
    } else {
      const int V[4] = {v, p0, p1, p2};
      float X[4][3];
      gather_Xf(a.sf, V, X);
      if (pair_distance_f(0, X) <= a.near) append(pack_key(0, v, t0 + k), a.out, a.count, a.overflow, a.cap);
    }
  }
}
template <int MODE>
__global__ void __launch_bounds__(kTile) k_sweep_pt(SweepArgs a) {
  k_sweep_pt_body<MODE>(a);
}

template <int MODE>
__device__ __forceinline__ void k_sweep_ee_body(SweepArgs a) {
  if (blockIdx.y < blockIdx.x) return;        // tiles with j-tile >= i-tile
  if (a.gate && *a.gate == 0) return;
  __shared__ float eb[kTile][6];
  __shared__ int eid[kTile][2];
  __shared__ unsigned long long ek[MODE == 1 ? kTile : 1][6];
  const int j0 = blockIdx.y * kTile;
  const int eoff = a.Ns + a.Nt;
  for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
    const int e = j0 + k;
    if (e < a.Ne) {
      const float* b = a.box + 12 * (size_t)(eoff + e) + 6;
#pragma unroll
      for (int q = 0; q < 6; ++q) eb[k][q] = b[q];
      eid[k][0] = a.edges[2 * e]; eid[k][1] = a.edges[2 * e + 1];
      if (MODE == 1) {
        const unsigned long long* kk = a.key + 12 * (size_t)(eoff + e) + 6;
#pragma unroll
        for (int q = 0; q < 6; ++q) ek[k][q] = kk[q];
      }
    }
  }
  __syncthreads();
  const int i = blockIdx.x * kTile + threadIdx.x;
  float ib[6], ebk[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float e = q < 3 ? INFINITY : -INFINITY;     // empty box
    ib[q] = i < a.Ne ? a.box[12 * (size_t)(eoff + i) + q] : e;
    ebk[q] = j0 + (int)threadIdx.x < a.Ne ? eb[threadIdx.x][q] : e;
  }
  if (!tile_pair_overlaps(ib, ebk)) return;
  if (i >= a.Ne) return;
  const int i0 = a.edges[2 * i], i1 = a.edges[2 * i + 1];
  unsigned long long ikk[6];
  if (MODE == 1) {
#pragma unroll
    for (int q = 0; q < 6; ++q) ikk[q] = a.key[12 * (size_t)(eoff + i) + q];
  }
  const int ne = min(kTile, a.Ne - j0);
  for (int k = 0; k < ne; ++k) {
    const int j = j0 + k;
    if (j <= i) continue;
    if (!ov32(ib, eb[k])) continue;
    const int b0 = eid[k][0], b1 = eid[k][1];
    if (b0 == i0 || b0 == i1 || b1 == i0 || b1 == i1) continue;
    if (MODE == 1) {
      if (ov64(ikk, ek[k])) append(pack_key(1, i, j), a.out, a.count, a.overflow, a.cap);
    } else {
      const int V[4] = {i0, i1, b0, b1};
      float X[4][3];
      gather_Xf(a.sf, V, X);
      if (pair_distance_f(1, X) <= a.near) append(pack_key(1, i, j), a.out, a.count, a.overflow, a.cap);
    }
  }
}
template <int MODE>
__global__ void __launch_bounds__(kTile) k_sweep_ee(SweepArgs a) {
  k_sweep_ee_body<MODE>(a);
}

// float64 narrow phase of the near pairs (one pair per thread, fixed grid,
// length read on the device): d < dhat joins C and adds kappa b(d).
__device__ __forceinline__ void k_near_pairs_body(const int* __restrict__ near_count, int64_t cap, int64_t cap_act,
                             const unsigned long long* __restrict__ nearl,
                             const double* __restrict__ s, const int* __restrict__ tris,
                             const int* __restrict__ edges, double dhat, double kappa,
                             const double* __restrict__ elen2,
                             unsigned long long* __restrict__ pairs, int* counters,
                             double* __restrict__ scal) {
  int64_t n = *near_count;
  n = n < cap ? n : cap;
  double esum = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int type, i, j;
    unpack_key(nearl[p], type, i, j);
    int V[4];
    load_pair(type, i, j, tris, edges, V);
    double X[4][3];
    gather_X(s, V, X);
    const double d = pair_distance(type, X);
    if (d < dhat) {
      append(pack_key(type, i, j), pairs, counters + 0, counters + 2, cap_act);
      double bv = barrier_value(d, dhat);
      if (elen2 != nullptr && type == 1) {     // edge-edge mollifier
        EdgeCross ec;
        edge_cross(X, ec);
        bv *= mollifier_value(ec.c, FSIM_MOLLIFIER_EPS_SCALE * elen2[i] * elen2[j]);
      }
      esum += bv;
      if (!(d > 0.0)) atomicOr(counters + 5, 1);
      else   // smallest active distance (positive doubles order like their bits)
        atomicMin(reinterpret_cast<unsigned long long*>(scal + 4), (unsigned long long)__double_as_longlong(d));
    }
  }
  if (esum != 0.0) atomicAdd(scal + 0, kappa * esum);
}
__global__ void k_near_pairs(const int* __restrict__ near_count, int64_t cap, int64_t cap_act,
                             const unsigned long long* __restrict__ nearl,
                             const double* __restrict__ s, const int* __restrict__ tris,
                             const int* __restrict__ edges, double dhat, double kappa,
                             const double* __restrict__ elen2,
                             unsigned long long* __restrict__ pairs, int* counters,
                             double* __restrict__ scal) {
  k_near_pairs_body(near_count, cap, cap_act, nearl, s, tris, edges, dhat, kappa, elen2, pairs, counters, scal);
}

// ACCD over the candidate list (length read on the device); a float32
// early-out first: when (1 - s) d0 exceeds l_p by a clear margin the first
// advance passes t = 1 and the float64 march would return "no impact" too.
__device__ __forceinline__ void k_accd_list_body(const int* __restrict__ cand_count, int64_t cap,
                            const unsigned long long* __restrict__ cand,
                            const double* __restrict__ s, const double* __restrict__ ds,
                            const float* __restrict__ sf, const float* __restrict__ dsf,
                            const int* __restrict__ tris, const int* __restrict__ edges,
                            double s_ratio, int max_iters, float slack, double* __restrict__ alpha) {
  int64_t n = *cand_count;
  n = n < cap ? n : cap;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int type, i, j;
    unpack_key(cand[p], type, i, j);
    int V[4];
    load_pair(type, i, j, tris, edges, V);
    {
      float X[4][3], dX[4][3];
      gather_Xf(sf, V, X);
      gather_Xf(dsf, V, dX);
      float mean[3], nrm[4];
#pragma unroll
      for (int d = 0; d < 3; ++d) mean[d] = 0.25f * (dX[0][d] + dX[1][d] + dX[2][d] + dX[3][d]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float a0 = dX[k][0] - mean[0], a1 = dX[k][1] - mean[1], a2 = dX[k][2] - mean[2];
        nrm[k] = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
      }
      const float lp = type == 1 ? fmaxf(nrm[0], nrm[1]) + fmaxf(nrm[2], nrm[3])
                                 : nrm[0] + fmaxf(fmaxf(nrm[1], nrm[2]), nrm[3]);
      const float df = pair_distance_f(type, X);
      if ((1.0f - (float)s_ratio) * (df - slack) > lp * 1.001f + slack) continue;
    }
    double X[4][3], dX[4][3];
    gather_X(s, V, X);
    gather_X(ds, V, dX);
    const double toi = accd_toi(type, X, dX, s_ratio, max_iters);
    if (toi < 1.0)
      atomicMin(reinterpret_cast<unsigned long long*>(alpha), (unsigned long long)__double_as_longlong(toi));
  }
}
__global__ void k_accd_list(const int* __restrict__ cand_count, int64_t cap,
                            const unsigned long long* __restrict__ cand,
                            const double* __restrict__ s, const double* __restrict__ ds,
                            const float* __restrict__ sf, const float* __restrict__ dsf,
                            const int* __restrict__ tris, const int* __restrict__ edges,
                            double s_ratio, int max_iters, float slack, double* __restrict__ alpha) {
  k_accd_list_body(cand_count, cap, cand, s, ds, sf, dsf, tris, edges, s_ratio, max_iters, slack, alpha);
}

// ---------------------------------------------------------------------------
// Skin (Verlet) list.  The all-pairs sweep runs only when proxy vertices
// have moved far since the last build: the list holds every pair whose
// float32 distance at the build positions sb was within dhat + skin.  A
// pair's distance changes by at most the sum of its two largest vertex
// displacements, so while 2 max|s - sb| <= skin - margin every pair with
// d(s) < dhat is in the list (the constraint set is unchanged), and while
// 2 (max|s - sb| + max|ds|) <= 0.4 skin no pair outside it can come within
// s_ccd d0 of contact during the step (the CCD bound is unchanged).
// counters: [10] list length, [11] rebuild now, [12] list valid,
// [13] CCD needs the full sweep, [14] list overflow.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_max_d(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;   // valid in thread 0
}

// one CTA: decide whether the skin list must be rebuilt (detection) or the
// CCD step needs the full sweep (ds != nullptr); a rebuild records sb = s
__device__ __forceinline__ void k_skin_check_body(int Ns, const double* __restrict__ s, double* __restrict__ sb,
                             const double* __restrict__ ds, double skin, double margin,
                             int* counters, double* scal) {
  if (ds == nullptr && threadIdx.x == 0) scal[4] = __longlong_as_double(0x7ff0000000000000LL);  // d_min = inf
  // maxima of the squared lengths; one square root each at the end
  // (sqrt is monotone and correctly rounded, so this is max |.| exactly)
  double dmax = 0.0, smax = 0.0;
  for (int v = threadIdx.x; v < Ns; v += blockDim.x) {
    double d2 = 0.0, q2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double e = s[3 * v + d] - sb[3 * v + d];
      d2 += e * e;
      if (ds) q2 += ds[3 * v + d] * ds[3 * v + d];
    }
    dmax = fmax(dmax, d2);
    smax = fmax(smax, q2);
  }
  dmax = sqrt(block_max_d(dmax));
  __syncthreads();
  smax = sqrt(block_max_d(smax));
  __shared__ int rebuild;
  if (threadIdx.x == 0) {
    const bool valid = counters[12] == 1 && counters[14] == 0;
    if (ds) {
      counters[13] = (valid && 2.0 * (dmax + smax) <= 0.4 * skin) ? 0 : 1;
      rebuild = 0;
    } else {
      rebuild = (valid && 2.0 * dmax <= skin - margin) ? 0 : 1;
      counters[11] = rebuild;
      if (rebuild) { counters[10] = 0; counters[12] = 1; counters[14] = 0; }
    }
  }
  __syncthreads();
  if (rebuild)
    for (int e = threadIdx.x; e < 3 * Ns; e += blockDim.x) sb[e] = s[e];
}
__global__ void k_skin_check(int Ns, const double* __restrict__ s, double* __restrict__ sb,
                             const double* __restrict__ ds, double skin, double margin,
                             int* counters, double* scal) {
  k_skin_check_body(Ns, s, sb, ds, skin, margin, counters, scal);
}

// near list from the skin list: float32 distance at the current positions
__device__ __forceinline__ void k_skin_near_body(const int* __restrict__ counters, int64_t cap,
                            const unsigned long long* __restrict__ vlist, const float* __restrict__ sf,
                            const int* __restrict__ tris, const int* __restrict__ edges, float near,
                            unsigned long long* __restrict__ nearl, int* count, int* overflow) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && counters[14]) atomicOr(overflow, 1);   // list incomplete
  int64_t n = counters[10];
  n = n < cap ? n : cap;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int type, i, j;
    unpack_key(vlist[p], type, i, j);
    int V[4];
    load_pair(type, i, j, tris, edges, V);
    float X[4][3];
    gather_Xf(sf, V, X);
    if (pair_distance_f(type, X) <= near) append(vlist[p], nearl, count, overflow, cap);
  }
}
__global__ void k_skin_near(const int* __restrict__ counters, int64_t cap,
                            const unsigned long long* __restrict__ vlist, const float* __restrict__ sf,
                            const int* __restrict__ tris, const int* __restrict__ edges, float near,
                            unsigned long long* __restrict__ nearl, int* count, int* overflow) {
  k_skin_near_body(counters, cap, vlist, sf, tris, edges, near, nearl, count, overflow);
}

// CCD candidates from the skin list (when counters[13] == 0): the exact
// float64 swept-box test of the full sweep
__device__ __forceinline__ void k_skin_cand_body(int* counters, int64_t cap, const unsigned long long* __restrict__ vlist,
                            const unsigned long long* __restrict__ key, int Ns, int Nt,
                            unsigned long long* __restrict__ cand) {
  if (counters[13] != 0) return;
  int64_t n = counters[10];
  n = n < cap ? n : cap;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int type, i, j;
    unpack_key(vlist[p], type, i, j);
    const unsigned long long* ka = key + 12 * (size_t)(type == 0 ? i : Ns + Nt + i);
    const unsigned long long* kb = key + 12 * (size_t)(type == 0 ? Ns + j : Ns + Nt + j) + 6;
    if (ov64(ka, kb)) append(vlist[p], cand, counters + 1, counters + 9, cap);
  }
}
__global__ void k_skin_cand(int* counters, int64_t cap, const unsigned long long* __restrict__ vlist,
                            const unsigned long long* __restrict__ key, int Ns, int Nt,
                            unsigned long long* __restrict__ cand) {
  k_skin_cand_body(counters, cap, vlist, key, Ns, Nt, cand);
}

// ---------------------------------------------------------------------------
void launch_proxy(cudaStream_t st, const DevMesh& m, const double* x, double* sp) {
  k_proxy<<<(m.Ns + 255) / 256, 256, 0, st>>>(m.Ns, m.Wptr, m.Wcol, m.Wval, x, sp);
  count_launch();
}

namespace {
int nprim(const DevMesh& m) { return m.Ns + m.Nt + m.Ne; }
// float32 rounding allowance of the skin tests (as for the CCD early-out)
double skin_margin(const DevMesh& m, double dhat) { return fmax(0.01 * dhat, 1e-5 * m.coord_scale); }

void launch_sweeps(cudaStream_t st, const DevMesh& m, int mode, unsigned long long* out, int* count,
                   int* overflow, float nearf, const int* gate) {
  SweepArgs a{m.Ns, m.Nt, m.Ne, m.pbox, m.pkey, m.sf, m.tris, m.edges, nearf, out, count, overflow,
              m.cap, gate};
  if (m.Ns > 0 && m.Nt > 0) {
    dim3 gpt((m.Ns + kTile - 1) / kTile, (m.Nt + kTile - 1) / kTile);
    if (mode == 0) k_sweep_pt<0><<<gpt, kTile, 0, st>>>(a);
    else k_sweep_pt<1><<<gpt, kTile, 0, st>>>(a);
    count_launch();
  }
  if (m.Ne > 1) {
    const int ne = (m.Ne + kTile - 1) / kTile;
    if (mode == 0) k_sweep_ee<0><<<dim3(ne, ne), kTile, 0, st>>>(a);
    else k_sweep_ee<1><<<dim3(ne, ne), kTile, 0, st>>>(a);
    count_launch();
  }
}
}  // namespace

// Constraint set and barrier energy at sp: prep, float32 sweeps into the
// near list, float64 narrow phase.  Uses counters [0] |C|, [2] overflow,
// [5] touching, [8] near-list length (all zeroed by the caller).
void launch_detect(cudaStream_t st, const DevMesh& m, const double* sp, double dhat, double kappa) {
  ProfScope ps(PROF_DETECT, st);
  const int np = nprim(m);
  if (np == 0) return;
  // boxes inflated for a skin-list build (used only when it runs)
  const double pad = dhat + m.skin;
  const float margin = (float)skin_margin(m, dhat);
  k_prim_prep<<<(np + 255) / 256, 256, 0, st>>>(m.Ns, m.Nt, m.Ne, sp, nullptr, m.tris, m.edges, pad,
                                                m.pbox, m.pkey, m.sf, nullptr);
  k_skin_check<<<1, 512, 0, st>>>(m.Ns, sp, m.sb, nullptr, m.skin, margin, m.counters, m.scal);
  launch_sweeps(st, m, 0, m.vlist, m.counters + 10, m.counters + 14, (float)pad + margin,
                m.counters + 11);
  k_skin_near<<<2 * 152, 128, 0, st>>>(m.counters, m.cap, m.vlist, m.sf, m.tris, m.edges,
                                       2.0f * (float)dhat, m.nearl, m.counters + 8, m.counters + 2);
  k_near_pairs<<<2 * 152, 128, 0, st>>>(m.counters + 8, m.cap, m.cap_act, m.nearl, sp, m.tris,
                                        m.edges, dhat, kappa, m.ee_moll ? m.elen2 : nullptr,
                                        m.pairs, m.counters, m.scal);
  count_launch(4);
}

// CCD candidates of the step sp -> sp + dsp into m.cand ([1] length, [9]
// overflow) and the additive-CCD step bound (min into m.scal[1]).
void launch_ccd(cudaStream_t st, const DevMesh& m, const double* sp, const double* dsp, double dhat,
                double ccd_s, int accd_max_iters) {
  ProfScope ps(PROF_CCD, st);
  const int np = nprim(m);
  if (np == 0) return;
  k_prim_prep<<<(np + 255) / 256, 256, 0, st>>>(m.Ns, m.Nt, m.Ne, sp, dsp, m.tris, m.edges, dhat,
                                                m.pbox, m.pkey, m.sf, m.dsf);
  // candidates from the skin list when it still covers the step, else the
  // full sweep
  k_skin_check<<<1, 512, 0, st>>>(m.Ns, sp, m.sb, dsp, m.skin, 0.0, m.counters, m.scal);
  k_skin_cand<<<2 * 152, 128, 0, st>>>(m.counters, m.cap, m.vlist, m.pkey, m.Ns, m.Nt, m.cand);
  launch_sweeps(st, m, 1, m.cand, m.counters + 1, m.counters + 9, 0.0f, m.counters + 13);
  count_launch(2);
  // float32 coordinates round by ~6e-8 of their magnitude; the early-out
  // slack (1e-5 of twice the largest rest coordinate, at least 1% of dhat)
  // stays two orders of magnitude above that rounding
  const double slack = fmax(0.01 * dhat, 1e-5 * m.coord_scale);
  k_accd_list<<<4 * 152, 128, 0, st>>>(m.counters + 1, m.cap, m.cand, sp, dsp, m.sf, m.dsf, m.tris,
                                       m.edges, ccd_s, accd_max_iters, (float)slack, m.scal + 1);
  count_launch(2);
}

void launch_barrier_pairs(cudaStream_t st, const DevMesh& m, int64_t np, const double* sp,
                          double dhat, double kappa, int precision) {
  np = np < m.cap_act ? np : m.cap_act;
  if (np <= 0) return;
  ProfScope ps(PROF_BARRIER, st);
  const int64_t want = (np + kPairWarps - 1) / kPairWarps;      // one warp per pair
  const unsigned grid = (unsigned)(want < 8 * 152 ? want : 8 * 152);
  const unsigned mgrid = grid;
  if (m.barrier_lanes) {                                          // one lane per pair
    const int64_t lw = (np + kPairLanes - 1) / kPairLanes;
    const unsigned lgrid = (unsigned)(lw < 8 * 152 ? lw : 8 * 152);
    if (precision == 0)
      k_barrier_pairs_lanes<double><<<lgrid, kPairLanes, 0, st>>>(
          m.counters, m.cap_act, m.pairs, sp, m.tris, m.edges, m.Wptr, m.Wcol, m.x2of, dhat, kappa,
          m.pair_grad, m.pair_hess, m.x2mark);
    else
      k_barrier_pairs_lanes<float><<<lgrid, kPairLanes, 0, st>>>(
          m.counters, m.cap_act, m.pairs, sp, m.tris, m.edges, m.Wptr, m.Wcol, m.x2of, dhat, kappa,
          m.pair_grad, m.pair_hess, m.x2mark);
  } else if (precision == 0)
    k_barrier_pairs<double><<<grid, 32 * kPairWarps, 0, st>>>(
        m.counters, m.cap_act, m.pairs, sp, m.tris, m.edges, m.Wptr, m.Wcol, m.x2of, dhat, kappa,
        m.pair_grad, m.pair_hess, m.x2mark);
  else
    k_barrier_pairs<float><<<grid, 32 * kPairWarps, 0, st>>>(
        m.counters, m.cap_act, m.pairs, sp, m.tris, m.edges, m.Wptr, m.Wcol, m.x2of, dhat, kappa,
        m.pair_grad, m.pair_hess, m.x2mark);
  count_launch();
  if (m.ee_moll) {
    k_mollify_ee<<<mgrid, 32, 0, st>>>(m.counters, m.cap_act, m.pairs, sp, m.edges, m.elen2, dhat,
                                      kappa, m.pair_grad, m.pair_hess);
    count_launch();
  }
}

void launch_mark_scan(cudaStream_t st, const DevMesh& m) {
  k_mark_scan<<<1, 1024, 0, st>>>(m.n2, m.x2mark, m.clist, m.counters);
  count_launch();
}

__device__ __forceinline__ void k_ccd_reset_body(int* counters, double* scal) {
  counters[1] = 0;
  counters[9] = 0;
  scal[1] = 1.0;
}
__global__ void k_ccd_reset(int* counters, double* scal) {
  k_ccd_reset_body(counters, scal);
}

void launch_ccd_reset(cudaStream_t st, const DevMesh& m) {
  k_ccd_reset<<<1, 1, 0, st>>>(m.counters, m.scal);
  count_launch();
}

void launch_barrier_scatter(cudaStream_t st, const DevMesh& m, int64_t np, int nc_cap, int mode,
                            double* g) {
  np = np < m.cap_act ? np : m.cap_act;
  if (np <= 0) return;
  const int64_t threads = 16 * np;
  k_barrier_scatter<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(
      np, m.pairs, m.tris, m.edges, m.Wptr, m.Wcol, m.Wval, m.x2of, m.x2mark, m.pair_grad,
      m.pair_hess, m.counters + 3, nc_cap, mode, g, m.Bc, m.bocc);
  count_launch();
}

void launch_zero_reduced(cudaStream_t st, const DevMesh& m, int nc_cap) {
  if (nc_cap <= 0 || m.Bc == nullptr) return;
  k_zero_reduced<<<2 * 152, 256, 0, st>>>(m.counters + 3, nc_cap, m.Bc, m.bocc);
  count_launch();
}

// ---------------------------------------------------------------------------
// Lock-step batches: one launch serves every frame of a batch table (one
// DevMesh per frame, all of one mesh).  The frame is blockIdx.y (blockIdx.z
// for the 2-D tile sweeps); a frame whose `active` flag is clear returns at
// once, uniformly for its blocks.  AT selects the evaluation point: 0 the
// iterate (x, s), 1 the line-search trial (xt, st).  Per-frame scalars
// (kappa of the frame) come from the table, mesh-wide ones are arguments.
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ const DevMesh* bframe_c(const DevMesh* __restrict__ tab, int f) {
  const DevMesh* m = tab + f;
  return m->active ? m : nullptr;
}
}  // namespace

// counters [0] |C|, [1] candidates, [2] overflow, [5] touching, [8] near
// list and scal[0] (barrier energy) of every active frame to zero
__global__ void k_eval_reset_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m || threadIdx.x != 0) return;
  m->counters[0] = 0; m->counters[1] = 0; m->counters[2] = 0;
  m->counters[5] = 0; m->counters[8] = 0;
  m->scal[0] = 0.0;
}

// AT 0: s = W x, 1: st = W xt, 2: ds = W dx
template <int AT>
__global__ void k_proxy_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  const double* x = AT == 0 ? m->x : (AT == 1 ? m->xt : m->dx);
  double* sp = AT == 0 ? m->s : (AT == 1 ? m->st : m->ds);
  k_proxy_body(m->Ns, m->Wptr, m->Wcol, m->Wval, x, sp);
}

// detection (CCD = 0) at s / st, or the CCD step s -> s + ds (CCD = 1)
template <int AT, int CCD>
__global__ void k_prim_prep_b(const DevMesh* __restrict__ tab, double pad) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  k_prim_prep_body(m->Ns, m->Nt, m->Ne, AT ? m->st : m->s, CCD ? m->ds : nullptr, m->tris, m->edges,
                   pad, m->pbox, m->pkey, m->sf, CCD ? m->dsf : nullptr);
}

template <int AT, int CCD>
__global__ void k_skin_check_b(const DevMesh* __restrict__ tab, double margin) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  k_skin_check_body(m->Ns, AT ? m->st : m->s, m->sb, CCD ? m->ds : nullptr, m->skin, margin,
                    m->counters, m->scal);
}

__device__ __forceinline__ SweepArgs sweep_args_b(const DevMesh* m, int mode, float nearf) {
  if (mode == 0)
    return SweepArgs{m->Ns, m->Nt, m->Ne, m->pbox, m->pkey, m->sf, m->tris, m->edges, nearf,
                     m->vlist, m->counters + 10, m->counters + 14, m->cap, m->counters + 11};
  return SweepArgs{m->Ns, m->Nt, m->Ne, m->pbox, m->pkey, m->sf, m->tris, m->edges, nearf,
                   m->cand, m->counters + 1, m->counters + 9, m->cap, m->counters + 13};
}

template <int MODE>
__global__ void __launch_bounds__(kTile) k_sweep_pt_b(const DevMesh* __restrict__ tab, float nearf) {
  const DevMesh* m = bframe_c(tab, blockIdx.z);
  if (!m) return;
  k_sweep_pt_body<MODE>(sweep_args_b(m, MODE, nearf));
}

template <int MODE>
__global__ void __launch_bounds__(kTile) k_sweep_ee_b(const DevMesh* __restrict__ tab, float nearf) {
  const DevMesh* m = bframe_c(tab, blockIdx.z);
  if (!m) return;
  k_sweep_ee_body<MODE>(sweep_args_b(m, MODE, nearf));
}

__global__ void k_skin_near_b(const DevMesh* __restrict__ tab, float near2) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  k_skin_near_body(m->counters, m->cap, m->vlist, m->sf, m->tris, m->edges, near2, m->nearl,
                   m->counters + 8, m->counters + 2);
}

template <int AT>
__global__ void k_near_pairs_b(const DevMesh* __restrict__ tab, double dhat) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  k_near_pairs_body(m->counters + 8, m->cap, m->cap_act, m->nearl, AT ? m->st : m->s, m->tris,
                    m->edges, dhat, m->kappa_f, m->ee_moll ? m->elen2 : nullptr, m->pairs,
                    m->counters, m->scal);
}

__global__ void __launch_bounds__(kPairLanes) k_barrier_pairs_b(const DevMesh* __restrict__ tab,
                                                                     double dhat) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  if (m->bar64)       // a frame switched to float64 contact Hessians
    k_barrier_pairs_body<double>(m->counters, m->cap_act, m->pairs, m->s, m->tris, m->edges,
                                 m->Wptr, m->Wcol, m->x2of, dhat, m->kappa_f, m->pair_grad,
                                 m->pair_hess, m->x2mark);
  else
    k_barrier_pairs_body<float>(m->counters, m->cap_act, m->pairs, m->s, m->tris, m->edges,
                                m->Wptr, m->Wcol, m->x2of, dhat, m->kappa_f, m->pair_grad,
                                m->pair_hess, m->x2mark);
}

__global__ void __launch_bounds__(32) k_mollify_ee_b(const DevMesh* __restrict__ tab, double dhat) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  k_mollify_ee_body(m->counters, m->cap_act, m->pairs, m->s, m->edges, m->elen2, dhat, m->kappa_f,
                    m->pair_grad, m->pair_hess);
}

__global__ void k_zero_x2mark_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m->n2; q += gridDim.x * blockDim.x)
    m->x2mark[q] = 0;
}

__global__ void k_mark_scan_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  k_mark_scan_body(m->n2, m->x2mark, m->clist, m->counters);
}

// B-check and its occupancy zeroed for the frame's n_c when they fit its
// reduced buffers
__global__ void k_zero_reduced_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m || m->Bc == nullptr) return;
  k_zero_reduced_body(m->counters + 3, m->nc_cap, m->Bc, m->bocc);
}

// gradient (mode 1) and B-check (mode 2) scatter; the pair count is read on
// the device (the grid covers the largest count of the batch)
__global__ void k_barrier_scatter_b(const DevMesh* __restrict__ tab, int mode) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  int64_t np = m->counters[0];
  np = np < m->cap_act ? np : m->cap_act;
  k_barrier_scatter_body(np, m->pairs, m->tris, m->edges, m->Wptr, m->Wcol, m->Wval, m->x2of,
                         m->x2mark, m->pair_grad, m->pair_hess, m->counters + 3,
                         m->Bc != nullptr ? m->nc_cap : 0, mode, m->g, m->Bc, m->bocc);
}

__global__ void k_ccd_reset_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m || threadIdx.x != 0) return;
  k_ccd_reset_body(m->counters, m->scal);
}

__global__ void k_skin_cand_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  k_skin_cand_body(m->counters, m->cap, m->vlist, m->pkey, m->Ns, m->Nt, m->cand);
}

__global__ void k_accd_list_b(const DevMesh* __restrict__ tab, double ccd_s, int accd_max_iters,
                              float slack) {
  const DevMesh* m = bframe_c(tab, blockIdx.y);
  if (!m) return;
  k_accd_list_body(m->counters + 1, m->cap, m->cand, m->s, m->ds, m->sf, m->dsf, m->tris, m->edges,
                   ccd_s, accd_max_iters, slack, m->scal + 1);
}

namespace {
void launch_sweeps_b(cudaStream_t st, const DevMesh* tab, int nb, const DevMesh& m0, int mode,
                     float nearf) {
  if (m0.Ns > 0 && m0.Nt > 0) {
    dim3 gpt((m0.Ns + kTile - 1) / kTile, (m0.Nt + kTile - 1) / kTile, nb);
    if (mode == 0) k_sweep_pt_b<0><<<gpt, kTile, 0, st>>>(tab, nearf);
    else k_sweep_pt_b<1><<<gpt, kTile, 0, st>>>(tab, nearf);
    count_launch();
  }
  if (m0.Ne > 1) {
    const int ne = (m0.Ne + kTile - 1) / kTile;
    if (mode == 0) k_sweep_ee_b<0><<<dim3(ne, ne, nb), kTile, 0, st>>>(tab, nearf);
    else k_sweep_ee_b<1><<<dim3(ne, ne, nb), kTile, 0, st>>>(tab, nearf);
    count_launch();
  }
}
}  // namespace

void launch_eval_reset_b(cudaStream_t st, const DevMesh* tab, int nb) {
  k_eval_reset_b<<<dim3(1, nb), 32, 0, st>>>(tab);
  count_launch();
}

void launch_proxy_b(cudaStream_t st, const DevMesh* tab, int nb, const DevMesh& m0, int at) {
  const dim3 g((m0.Ns + 255) / 256, nb);
  if (at == 0) k_proxy_b<0><<<g, 256, 0, st>>>(tab);
  else if (at == 1) k_proxy_b<1><<<g, 256, 0, st>>>(tab);
  else k_proxy_b<2><<<g, 256, 0, st>>>(tab);
  count_launch();
}

void launch_detect_b(cudaStream_t st, const DevMesh* tab, int nb, const DevMesh& m0, int at,
                     double dhat) {
  ProfScope ps(PROF_DETECT, st);
  const int np = nprim(m0);
  if (np == 0) return;
  const double pad = dhat + m0.skin;
  const float margin = (float)skin_margin(m0, dhat);
  const dim3 gp((np + 255) / 256, nb);
  if (at) {
    k_prim_prep_b<1, 0><<<gp, 256, 0, st>>>(tab, pad);
    k_skin_check_b<1, 0><<<dim3(1, nb), 512, 0, st>>>(tab, margin);
  } else {
    k_prim_prep_b<0, 0><<<gp, 256, 0, st>>>(tab, pad);
    k_skin_check_b<0, 0><<<dim3(1, nb), 512, 0, st>>>(tab, margin);
  }
  count_launch(2);
  launch_sweeps_b(st, tab, nb, m0, 0, (float)pad + margin);
  k_skin_near_b<<<dim3(2 * 152, nb), 128, 0, st>>>(tab, 2.0f * (float)dhat);
  if (at) k_near_pairs_b<1><<<dim3(2 * 152, nb), 128, 0, st>>>(tab, dhat);
  else k_near_pairs_b<0><<<dim3(2 * 152, nb), 128, 0, st>>>(tab, dhat);
  count_launch(2);
}

void launch_barrier_b(cudaStream_t st, const DevMesh* tab, int nb, const DevMesh& m0,
                      int64_t np_max, double dhat) {
  k_zero_x2mark_b<<<dim3((std::max(m0.n2, 1) + 255) / 256, nb), 256, 0, st>>>(tab);
  count_launch();
  np_max = np_max < m0.cap_act ? np_max : m0.cap_act;
  if (np_max > 0) {
    ProfScope ps(PROF_BARRIER, st);
    const int64_t want = (np_max + kPairLanes - 1) / kPairLanes;    // one lane per pair
    const unsigned grid = (unsigned)(want < 8 * 152 ? want : 8 * 152);
    const unsigned mgrid = (unsigned)(np_max < 8 * 152 ? np_max : 8 * 152);
    k_barrier_pairs_b<<<dim3(grid, nb), kPairLanes, 0, st>>>(tab, dhat);
    count_launch();
    if (m0.ee_moll) {
      k_mollify_ee_b<<<dim3(mgrid, nb), 32, 0, st>>>(tab, dhat);
      count_launch();
    }
  }
  k_mark_scan_b<<<dim3(1, nb), 1024, 0, st>>>(tab);
  k_zero_reduced_b<<<dim3(2 * 152, nb), 256, 0, st>>>(tab);
  count_launch(2);
  if (np_max > 0) {
    const int64_t threads = 16 * np_max;
    k_barrier_scatter_b<<<dim3((unsigned)((threads + 127) / 128), nb), 128, 0, st>>>(tab, 3);
    count_launch();
  }
}

void launch_ccd_b(cudaStream_t st, const DevMesh* tab, int nb, const DevMesh& m0, double dhat,
                  double ccd_s, int accd_max_iters) {
  launch_proxy_b(st, tab, nb, m0, 2);
  k_ccd_reset_b<<<dim3(1, nb), 32, 0, st>>>(tab);
  count_launch();
  ProfScope ps(PROF_CCD, st);
  const int np = nprim(m0);
  if (np == 0) return;
  k_prim_prep_b<0, 1><<<dim3((np + 255) / 256, nb), 256, 0, st>>>(tab, dhat);
  k_skin_check_b<0, 1><<<dim3(1, nb), 512, 0, st>>>(tab, 0.0);
  k_skin_cand_b<<<dim3(2 * 152, nb), 128, 0, st>>>(tab);
  count_launch(3);
  launch_sweeps_b(st, tab, nb, m0, 1, 0.0f);
  const double slack = fmax(0.01 * dhat, 1e-5 * m0.coord_scale);
  k_accd_list_b<<<dim3(4 * 152, nb), 128, 0, st>>>(tab, ccd_s, accd_max_iters, (float)slack);
  count_launch();
}

}  // namespace fsim

// ===========================================================================
// CCD step bound without any device allocation.
//
// Some callers cannot let a library allocate GPU memory: an animation or game
// engine that reserves all device memory up front in its own pool, or a host
// application that must stay inside a fixed memory budget.  For them,
// fsim_ccd_noalloc computes the same additive-CCD step bound as the solver's
// CCD stage, with every input and output owned by the caller and its only
// scratch (the candidate-pair list and its counters) in the fixed array below.
// Each call reads its status words back and synchronises the caller's stream
// before it returns.  The candidate search is brute force over all
// point-triangle and edge-edge pairs (O(Ns Nt + Ne^2) box tests), meant for
// the few thousand primitives of a contact region.
// ===========================================================================
namespace fsim {
namespace {

// Largest candidate list the static scratch holds (8 MiB of keys).
constexpr int64_t kNoallocCandidates = int64_t(1) << 20;
// Words [0, 2): four int counters ([1] candidates, [2] overflow flag, [3] an
// index outside [0, Ns) in the caller's triangles or edges), as the pair
// kernels use them; words [2, 2 + kNoallocCandidates): candidate keys.
// Every GPU that loads the library keeps this array until the process exits.
constexpr int kNoallocHeaderWords = 2;
static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[kNoallocHeaderWords + kNoallocCandidates];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;          // guards the per-device address table

// ACCD over a candidate list whose length is read on the device (so the host
// never has to read it back); fixed grid, grid-stride loop.
__global__ void k_accd_count(const int* __restrict__ counters, int64_t cap,
                             const unsigned long long* __restrict__ cand,
                             const double* __restrict__ s, const double* __restrict__ ds,
                             const int* __restrict__ tris, const int* __restrict__ edges,
                             double s_ratio, int max_iters, double* __restrict__ alpha) {
  int64_t n = counters[1];
  n = n < cap ? n : cap;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int type, i, j;
    unpack_key(cand[p], type, i, j);
    int V[4];
    load_pair(type, i, j, tris, edges, V);
    double X[4][3], dX[4][3];
    gather_X(s, V, X);
    gather_X(ds, V, dX);
    const double toi = accd_toi(type, X, dX, s_ratio, max_iters);
    if (toi < 1.0)
      atomicMin(reinterpret_cast<unsigned long long*>(alpha),
                (unsigned long long)__double_as_longlong(toi));
  }
}

__global__ void k_set_one(double* a) { *a = 1.0; }

}  // namespace
}  // namespace fsim

extern "C" fsim_status fsim_ccd_noalloc(const double* s_dev, const double* ds_dev, int64_t Ns,
                                        const int32_t* tris_dev, int64_t Nt,
                                        const int32_t* edges_dev, int64_t Ne, double dhat,
                                        double ccd_s, int32_t accd_max_iters, double* alpha_dev,
                                        void* stream) {
  using namespace fsim;
  if (!alpha_dev || Ns < 0 || Nt < 0 || Ne < 0 || Ns >= (1LL << 31) || Nt >= (1LL << 31) ||
      Ne >= (1LL << 31) || !(dhat > 0.0) || !(ccd_s > 0.0 && ccd_s < 1.0) || accd_max_iters <= 0)
    return FSIM_EINVAL;
  if (Ns > 0 && (!s_dev || !ds_dev)) return FSIM_EINVAL;
  if ((Nt > 0 && !tris_dev) || (Ne > 0 && !edges_dev)) return FSIM_EINVAL;
  // the candidate kernels tile triangles and edges along gridDim.y
  if ((Nt + kTile - 1) / kTile > 65535 || (Ne + kTile - 1) / kTile > 65535) return FSIM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSIM_ECUDA;
  // one-time set-up per device: the host-side name of the array is not a
  // device address, so ask the runtime for the address on this device
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return FSIM_ECUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* base = (unsigned long long*)scratch;
  int* counters = reinterpret_cast<int*>(base);          // header: 4 ints
  unsigned long long* keys = base + kNoallocHeaderWords;
  // the array keeps the previous call's contents: reset the counters
  if (cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * kNoallocHeaderWords, st) !=
      cudaSuccess)
    return FSIM_ECUDA;
  k_set_one<<<1, 1, 0, st>>>(alpha_dev);
  if (Ns > 0 && Nt > 0) {
    dim3 gpt((unsigned)((Ns + kTile - 1) / kTile), (unsigned)((Nt + kTile - 1) / kTile));
    k_cand_pt<<<gpt, kTile, 0, st>>>((int)Ns, (int)Nt, s_dev, ds_dev, tris_dev, dhat, keys, counters,
                                     kNoallocCandidates);
  }
  if (Ne > 1) {
    const unsigned ne = (unsigned)((Ne + kTile - 1) / kTile);
    k_cand_ee<<<dim3(ne, ne), kTile, 0, st>>>((int)Ns, (int)Ne, s_dev, ds_dev, edges_dev, dhat, keys, counters,
                                              kNoallocCandidates);
  }
  k_accd_count<<<256, 128, 0, st>>>(counters, kNoallocCandidates, keys, s_dev, ds_dev, tris_dev,
                                    edges_dev, ccd_s, accd_max_iters, alpha_dev);
  if (cudaGetLastError() != cudaSuccess) return FSIM_ECUDA;
  int host_counters[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(host_counters, counters, sizeof(host_counters), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FSIM_ECUDA;
  if (host_counters[3]) return FSIM_EINVAL;      // an index outside [0, Ns)
  return host_counters[2] ? FSIM_ECONTACT_OVERFLOW : FSIM_OK;
}
