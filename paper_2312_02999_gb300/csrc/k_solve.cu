// Global step of Eq. 4 through the Schur complement (Eq. 8-9) and the
// low-rank update of Sigma^-1 (Eq. 10-11), on the GPU.
//
// With H = K (x) I_3, solver positions [x1 ; x2] and r = -g-hat:
//   t1 = K11^-1 r1                      (forward + backward supernodal solves)
//   y2 = r2 - K21 t1                    (lower block step of Eq. 8)
//   u  = Sigma^-1 y2                    (explicit Sigma^-1, Sec. 3.2)
//   z2 = Sigma-hat^-1 y2 = u - Sigma^-1 Q^T v  with the reduced system below
//   dx2 = z2,  dx1 = K11^-1 (r1 - K12 dx2)      (upper block step of Eq. 8)
// Reduced system on the n_c contact-affected vertices (push-through form of
// Eq. 11; B-check is PSD and usually singular, so it is never inverted):
//   v = (I + B S)^-1 B u_c,  S = Sigma^-1[c,c] (x) I_3.
// It is solved in the symmetric form v = L^-T (I + L^T B L)^-1 L^T B u_c with
// S = L L^T; I + L^T B L is SPD with eigenvalues >= 1 (Cholesky, no pivots).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace fsim {

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// gathers / scatters between vertex order and solver positions
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gather_rhs(int nf, const int* __restrict__ perm, const double* __restrict__ g,
                             T* __restrict__ r) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nf) return;
  const int v = perm[p];
#pragma unroll
  for (int d = 0; d < 3; ++d) r[3 * (size_t)p + d] = (T)(-g[3 * (size_t)v + d]);
}

__global__ void k_scatter_dx(int nf, const int* __restrict__ perm, const double* __restrict__ z,
                             double* __restrict__ dx) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nf) return;
  const int v = perm[p];
#pragma unroll
  for (int d = 0; d < 3; ++d) dx[3 * (size_t)v + d] = z[3 * (size_t)p + d];
}

template <typename S, typename T>
__global__ void k_convert(int n, const S* __restrict__ a, T* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

// ---------------------------------------------------------------------------
// supernodal triangular solves with Z_J = [L_JJ^-1 ; L_RJ L_JJ^-1]
// ---------------------------------------------------------------------------
// Chunked forms: a level is a list of work items (J, first row/column, count)
// so that one large supernode spreads over many CTAs.  A level's work is a
// handful of dependent GEMV chunks, so the serial chain per lane sets its
// time: a solve that has the GPU to itself uses 32 warps per item (NT =
// 1024); solves that share the GPU with others, and the float64 form (bound
// by the float64 pipe), use 8 warps per item (NT = 256) so that more items fit
// on an SM.
constexpr int kBwdCols = 8;                       // columns per backward item

// Forward item: rows [r0, r0+32) of Z_J times b_J; lanes own rows (coalesced
// column-major reads), the 32 warps split the inner index and reduce through
// shared memory.
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_fwd_chunk(const int4* __restrict__ items, const int* __restrict__ c0a, const int* __restrict__ nsa,
            const int* __restrict__ nra, const int64_t* __restrict__ roff,
            const int64_t* __restrict__ zoff, const int* __restrict__ rows,
            const T* __restrict__ Z, T* __restrict__ b, T* __restrict__ y) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int kSolveWarps = NT / 32;
  T* bj = reinterpret_cast<T*>(smem_raw);
  __shared__ T part[kSolveWarps][32][3];
  const int4 it = items[blockIdx.x];
  const int J = it.x, r0 = it.y, rn = it.z;
  const int c0 = c0a[J], ns = nsa[J], nr = nra[J], ld = ns + nr;
  const T* Zj = Z + zoff[J];
  for (int k = threadIdx.x; k < 3 * ns; k += blockDim.x) bj[k] = b[3 * (size_t)c0 + k];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int r = r0 + lane;
  T a0 = 0, a1 = 0, a2 = 0;
  if (lane < rn) {
    const int kmax = r < ns ? r + 1 : ns;
    // two independent loads and accumulators in flight per lane
    T q0 = 0, q1 = 0, q2 = 0;
    int k = wid;
    for (; k + kSolveWarps < kmax; k += 2 * kSolveWarps) {
      const T z0 = Zj[(size_t)k * ld + r], z1 = Zj[(size_t)(k + kSolveWarps) * ld + r];
      const int k1 = k + kSolveWarps;
      a0 += z0 * bj[3 * k]; a1 += z0 * bj[3 * k + 1]; a2 += z0 * bj[3 * k + 2];
      q0 += z1 * bj[3 * k1]; q1 += z1 * bj[3 * k1 + 1]; q2 += z1 * bj[3 * k1 + 2];
    }
    if (k < kmax) {
      const T z = Zj[(size_t)k * ld + r];
      a0 += z * bj[3 * k]; a1 += z * bj[3 * k + 1]; a2 += z * bj[3 * k + 2];
    }
    a0 += q0; a1 += q1; a2 += q2;
  }
  part[wid][lane][0] = a0; part[wid][lane][1] = a1; part[wid][lane][2] = a2;
  __syncthreads();
  if (threadIdx.x < 96) {
    const int rl = threadIdx.x / 3, d = threadIdx.x % 3;
    if (rl < rn) {
      T acc = 0;
#pragma unroll 8
      for (int w = 0; w < kSolveWarps; ++w) acc += part[w][rl][d];
      const int rr = r0 + rl;
      if (rr < ns) y[3 * (size_t)(c0 + rr) + d] = acc;
      else atomicAdd(b + 3 * (size_t)rows[roff[J] + rr - ns] + d, -acc);
    }
  }
}

// Backward item: columns [k0, k0+kn) (kn <= 8) of Z_J^T [y_J ; -x_R]; NT/256
// warps per column split its rows.  Reads y (forward result) and the
// ancestors' x, writes x_J (x may alias b).
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_bwd_chunk(const int4* __restrict__ items, const int* __restrict__ c0a, const int* __restrict__ nsa,
            const int* __restrict__ nra, const int64_t* __restrict__ roff,
            const int64_t* __restrict__ zoff, const int* __restrict__ rows,
            const T* __restrict__ Z, const T* __restrict__ y, T* __restrict__ x) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int kBwdWarpsPerCol = NT / 32 / kBwdCols;
  T* wv = reinterpret_cast<T*>(smem_raw);
  __shared__ T part[kBwdCols][kBwdWarpsPerCol][3];
  const int4 it = items[blockIdx.x];
  const int J = it.x, k0 = it.y, kn = it.z;
  const int c0 = c0a[J], ns = nsa[J], nr = nra[J], ld = ns + nr;
  const T* Zj = Z + zoff[J];
  const int* Rj = rows + roff[J];
  // only rows >= k0 of w are used by these columns
  for (int k = 3 * k0 + threadIdx.x; k < 3 * ns; k += blockDim.x) wv[k] = y[3 * (size_t)c0 + k];
  for (int k = threadIdx.x; k < 3 * nr; k += blockDim.x)
    wv[3 * ns + k] = -x[3 * (size_t)Rj[k / 3] + (k % 3)];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int c = wid / kBwdWarpsPerCol, qw = wid % kBwdWarpsPerCol;
  constexpr int kStride = 32 * kBwdWarpsPerCol;
  T a0 = 0, a1 = 0, a2 = 0;
  if (c < kn) {
    const int k = k0 + c;
    const T* zc = Zj + (size_t)k * ld;
    T q0 = 0, q1 = 0, q2 = 0;
    int r = k + qw * 32 + lane;
    for (; r + kStride < ld; r += 2 * kStride) {
      const T z0 = zc[r], z1 = zc[r + kStride];
      const int s1 = r + kStride;
      a0 += z0 * wv[3 * r]; a1 += z0 * wv[3 * r + 1]; a2 += z0 * wv[3 * r + 2];
      q0 += z1 * wv[3 * s1]; q1 += z1 * wv[3 * s1 + 1]; q2 += z1 * wv[3 * s1 + 2];
    }
    if (r < ld) {
      const T z = zc[r];
      a0 += z * wv[3 * r]; a1 += z * wv[3 * r + 1]; a2 += z * wv[3 * r + 2];
    }
    a0 += q0; a1 += q1; a2 += q2;
  }
  a0 = warp_sum_t(a0); a1 = warp_sum_t(a1); a2 = warp_sum_t(a2);
  if (lane == 0) { part[c][qw][0] = a0; part[c][qw][1] = a1; part[c][qw][2] = a2; }
  __syncthreads();
  if (threadIdx.x < 3 * kBwdCols) {
    const int cc = threadIdx.x / 3, d = threadIdx.x % 3;
    if (cc < kn) {
      T acc = 0;
#pragma unroll
      for (int w = 0; w < kBwdWarpsPerCol; ++w) acc += part[cc][w][d];
      x[3 * (size_t)(c0 + k0 + cc) + d] = acc;
    }
  }
}

// u = Sinv y (n2 x n2 dense, 3 right-hand sides), one warp per row
template <typename T>
__global__ void k_gemv3(int n2, const T* __restrict__ A, const T* __restrict__ y, T* __restrict__ u) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n2) return;
  const T* a = A + (size_t)row * n2;
  T a0 = 0, a1 = 0, a2 = 0;
  for (int j = lane; j < n2; j += 32) {
    const T s = a[j];
    a0 += s * y[3 * j]; a1 += s * y[3 * j + 1]; a2 += s * y[3 * j + 2];
  }
  a0 = warp_sum_t(a0); a1 = warp_sum_t(a1); a2 = warp_sum_t(a2);
  if (lane == 0) { u[3 * row] = a0; u[3 * row + 1] = a1; u[3 * row + 2] = a2; }
}

// ---------------------------------------------------------------------------
// Lock-step batches: the triangular solves and the Sigma^-1 product for the
// right-hand sides of all frames at once.  A multi-right-hand-side buffer
// holds, per solver position p, a row of nr floats; frame f's three columns
// start at column 3 col_f.  The factor is read once per pass for all frames.
// A CTA takes one work item (as in the single-frame solves) and 32 columns
// (blockIdx.y); lane = column, each warp 4 rows (forward, GEMM) or one factor
// column (backward); the factor tile is staged in shared memory so that every
// factor entry is one broadcast shared-memory load for 32 columns.
// ---------------------------------------------------------------------------
constexpr int kMrCols = 32;
constexpr int kMrK = 64;           // factor rows / columns staged per step

// The staged tiles are loaded with every load of a thread in flight at once
// (register staging, fixed trip counts) and the next tile is fetched while
// the current one is used: a staging loop that waited for one load per
// iteration cost a memory latency per element row, which set the time of the
// levels with the largest supernodes.
__global__ void __launch_bounds__(256)
k_fwd_mr(const int4* __restrict__ items, const int* __restrict__ c0a, const int* __restrict__ nsa,
         const int* __restrict__ nra, const int64_t* __restrict__ roff,
         const int64_t* __restrict__ zoff, const int* __restrict__ rows,
         const float* __restrict__ Z, float* __restrict__ b, float* __restrict__ y, int nr,
         int nf) {
  extern __shared__ float bj[];                    // ns x 32
  __shared__ __align__(16) float Zs[2][kMrK][32];
  __shared__ float part[8][32][32];                // warp partial sums (no padding needed:
                                                   // lanes always index the last dimension)
  const int4 it = items[blockIdx.x];
  const int J = it.x, r0 = it.y, rn = it.z;
  const int cc = blockIdx.y * kMrCols;
  const int c0 = c0a[J], ns = nsa[J], ld = ns + nra[J];
  const float* Zj = Z + zoff[J];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // rows of the diagonal block only need k <= row (L_JJ^-1 is lower triangular)
  const int kend = r0 < ns ? min(ns, r0 + rn) : ns;
  constexpr int kPer = kMrK * 32 / 256;            // Z elements per thread per tile
  float zr[kPer];
  auto load_z = [&](int k0) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = tid + 256 * i, kk = e >> 5, rr = e & 31, k = k0 + kk, r = r0 + rr;
      zr[i] = (k < kend && rr < rn && (r >= ns || k <= r)) ? __ldg(Zj + (size_t)k * ld + r) : 0.f;
    }
  };
  auto store_z = [&](int buf) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = tid + 256 * i;
      Zs[buf][e >> 5][e & 31] = zr[i];
    }
  };
  load_z(0);
  {   // right-hand sides of the supernode's columns, 8 loads in flight per thread
    const int tot = ns * kMrCols;
    for (int e0 = 0; e0 < tot; e0 += 8 * 256) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int e = e0 + tid + 256 * i;
        v[i] = e < tot ? b[(size_t)(c0 + e / kMrCols) * nr + cc + (e % kMrCols)] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int e = e0 + tid + 256 * i;
        if (e < tot) bj[e] = v[i];
      }
    }
  }
  store_z(0);
  __syncthreads();
  // warp w sums the terms k = w (mod 8) for all 32 rows (lane = column), so
  // each thread keeps 32 independent accumulators
  float acc[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) acc[q] = 0.f;
  int buf = 0;
  for (int k0 = 0; k0 < kend; k0 += kMrK) {
    const bool more = k0 + kMrK < kend;
    if (more) load_z(k0 + kMrK);                   // next tile in flight
    const int kn = min(kMrK, kend - k0);
    for (int kk = wid; kk < kn; kk += 8) {
      const float bk = bj[(k0 + kk) * kMrCols + lane];
      const float4* zp = reinterpret_cast<const float4*>(&Zs[buf][kk][0]);
#pragma unroll
      for (int q4 = 0; q4 < 8; ++q4) {
        const float4 z = zp[q4];
        acc[4 * q4] += z.x * bk; acc[4 * q4 + 1] += z.y * bk;
        acc[4 * q4 + 2] += z.z * bk; acc[4 * q4 + 3] += z.w * bk;
      }
    }
    if (more) store_z(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int q = 0; q < 32; ++q) part[wid][q][lane] = acc[q];
  __syncthreads();
  for (int e = tid; e < 32 * kMrCols; e += blockDim.x) {
    const int rr = e >> 5, j = e & 31;
    if (rr >= rn) continue;
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += part[w][rr][j];
    const int r = r0 + rr;
    if (r < ns) {
      y[(size_t)(c0 + r) * nr + cc + j] = t;
    } else {
      const int row = rows[roff[J] + r - ns];
      if (FSIM_CHECK_IDX(row, nf, CHECK_TRSV_ROW)) atomicAdd(b + (size_t)row * nr + cc + j, -t);
    }
  }
}

// x_J[k] += sum_r Z_J[r][k] w[r] over the item's rows r in [max(k0, rb0),
// rb0 + kBwdRowSplit) (r >= k), w = [y_J ; -x_R], for up to 32 columns
// k0 .. k0 + kn of Z_J and 32 right-hand-side columns; x_J is zeroed before
// the pass and the row ranges of a column group add their partial sums
// atomically.  w and the Z tile are staged in 64-row tiles (w once for all
// kn columns, the next tile in flight while the current one is used); warp w
// sums the rows r = w (mod 8) with 32 independent accumulators (one per
// factor column, lane = right-hand-side column), then the 8 partial sums are
// added
__global__ void __launch_bounds__(256)
k_bwd_mr(const int4* __restrict__ items, const int* __restrict__ c0a, const int* __restrict__ nsa,
         const int* __restrict__ nra, const int64_t* __restrict__ roff,
         const int64_t* __restrict__ zoff, const int* __restrict__ rows,
         const float* __restrict__ Z, const float* __restrict__ y, float* __restrict__ x, int nr,
         int nf) {
  constexpr int kRows = 64;
  constexpr int kPer = kRows * 32 / 256;           // elements per thread per tile
  __shared__ __align__(16) float buf[2 * 2 * kRows * 32 + 64];   // [2][ws | Zs]
  const int4 it = items[blockIdx.x];
  const int J = it.x, k0 = it.y, kn = it.z;
  const int cc = blockIdx.y * kMrCols;
  const int c0 = c0a[J], ns = nsa[J];
  const int ld = min(ns + nra[J], it.w + kBwdRowSplit);   // end of this item's rows
  const int ldz = ns + nra[J];                             // column stride of Z_J
  const float* Zj = Z + zoff[J];
  const int* Rj = rows + roff[J];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // the item's off-diagonal row positions (at most kBwdRowSplit), fetched
  // once, so that each staged tile needs one dependent global load, not two
  __shared__ int ridx[kBwdRowSplit];
  const int r_first = max(k0, it.w);
  for (int q = tid; q < ld - r_first; q += blockDim.x) {
    const int r = r_first + q;
    ridx[q] = r >= ns ? __ldg(Rj + r - ns) : -1;
  }
  __syncthreads();
  float wr[kPer], zr[kPer];
  auto load = [&](int rb) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = tid + 256 * i, rr = e >> 5, j = e & 31, r = rb + rr;
      float w = 0.f;
      if (r < ld) {
        if (r < ns) {
          w = y[(size_t)(c0 + r) * nr + cc + j];
        } else {
          const int row = ridx[r - r_first];
          if (FSIM_CHECK_IDX(row, nf, CHECK_TRSV_ROW)) w = -x[(size_t)row * nr + cc + j];
        }
      }
      wr[i] = w;
      // Z_J[r][k0 + j] (lower triangle of the diagonal block)
      zr[i] = (r < ld && j < kn && r >= k0 + j) ? __ldg(Zj + (size_t)(k0 + j) * ldz + r) : 0.f;
    }
  };
  auto store = [&](int bsel) {
    float* ws = buf + bsel * 2 * kRows * 32;
    float* zs = ws + kRows * 32;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = tid + 256 * i;
      ws[e] = wr[i];
      zs[e] = zr[i];
    }
  };
  float acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0.f;
  load(r_first);
  store(0);
  __syncthreads();
  int bsel = 0;
  for (int rb = r_first; rb < ld; rb += kRows) {
    const bool more = rb + kRows < ld;
    if (more) load(rb + kRows);
    const int rn = min(kRows, ld - rb);
    const float* ws = buf + bsel * 2 * kRows * 32;
    const float* zs = ws + kRows * 32;
    for (int rr = wid; rr < rn; rr += 8) {
      const float wv = ws[rr * 32 + lane];
      const float4* zp = reinterpret_cast<const float4*>(zs + rr * 32);
#pragma unroll
      for (int q4 = 0; q4 < 8; ++q4) {
        const float4 z = zp[q4];
        acc[4 * q4] += z.x * wv; acc[4 * q4 + 1] += z.y * wv;
        acc[4 * q4 + 2] += z.z * wv; acc[4 * q4 + 3] += z.w * wv;
      }
    }
    if (more) store(bsel ^ 1);
    __syncthreads();
    bsel ^= 1;
  }
  // the warps' partial sums reuse the tiles: 8 x 32 x 32 floats fit the
  // 2 x 2 x 64 x 32 of buf (lanes index the last dimension, no padding needed)
  static_assert(8 * 32 * 32 <= 2 * 2 * kRows * 32, "partial sums must fit the tile buffer");
  float (*part)[32][32] = reinterpret_cast<float (*)[32][32]>(buf);
#pragma unroll
  for (int c = 0; c < 32; ++c) part[wid][c][lane] = acc[c];
  __syncthreads();
  for (int e = tid; e < 32 * 32; e += blockDim.x) {
    const int c = e >> 5, j = e & 31;
    if (c >= kn) continue;
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += part[w][c][j];
    atomicAdd(x + (size_t)(c0 + k0 + c) * nr + cc + j, t);
  }
}

// u = Sigma^-1 y2 for all columns: rows [32 blockIdx.x, +32), columns chunk
// blockIdx.y; A and y2 tiles register-staged, the next tile in flight
__global__ void __launch_bounds__(256)
k_gemm_mr(int n2, const float* __restrict__ A, const float* __restrict__ yv, float* __restrict__ u,
          int nr) {
  __shared__ __align__(16) float As[2][kMrK][32];
  __shared__ float Ys[2][kMrK][32];
  constexpr int kPer = kMrK * 32 / 256;
  const int i0 = blockIdx.x * 32, cc = blockIdx.y * kMrCols;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float ar[kPer], yr[kPer];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = tid + 256 * q;
      const int rr = e / kMrK, kk = e % kMrK, i = i0 + rr, k = k0 + kk;   // coalesced along k
      ar[q] = (i < n2 && k < n2) ? __ldg(A + (size_t)i * n2 + k) : 0.f;
      const int kk2 = e >> 5, j = e & 31, k2 = k0 + kk2;
      yr[q] = k2 < n2 ? yv[(size_t)k2 * nr + cc + j] : 0.f;
    }
  };
  auto store = [&](int bsel) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = tid + 256 * q;
      As[bsel][e % kMrK][e / kMrK] = ar[q];
      Ys[bsel][e >> 5][e & 31] = yr[q];
    }
  };
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  load(0);
  store(0);
  __syncthreads();
  int bsel = 0;
  for (int k0 = 0; k0 < n2; k0 += kMrK) {
    const bool more = k0 + kMrK < n2;
    if (more) load(k0 + kMrK);
    const int kn = min(kMrK, n2 - k0);
    for (int kk = 0; kk < kn; ++kk) {
      const float yk = Ys[bsel][kk][lane];
      const float4 a = *reinterpret_cast<const float4*>(&As[bsel][kk][4 * wid]);
      acc[0] += a.x * yk; acc[1] += a.y * yk; acc[2] += a.z * yk; acc[3] += a.w * yk;
    }
    if (more) store(bsel ^ 1);
    __syncthreads();
    bsel ^= 1;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + 4 * wid + q;
    if (i < n2) u[(size_t)i * nr + cc + lane] = acc[q];
  }
}

// right-hand sides r = -g of every frame into the multi-RHS buffer (zero
// columns for inactive frames, so that stale columns never grow)
__global__ void k_gather_rhs_mr(const DevMesh* __restrict__ tab, float* __restrict__ rb, int nr) {
  const DevMesh& m = tab[blockIdx.y];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m.nf) return;
  float* dst = rb + (size_t)p * nr + 3 * m.col;
  if (!m.active) { dst[0] = 0.f; dst[1] = 0.f; dst[2] = 0.f; return; }
  const int v = m.perm[p];
#pragma unroll
  for (int d = 0; d < 3; ++d) dst[d] = (float)(-m.g[3 * (size_t)v + d]);
}

// per frame: u (float64) and y2 (float) in the frame's own buffers for the
// reduced system (the x2 rows of the contact-free backward solve get u by one
// contiguous copy)
__global__ void k_unpack_mr(const DevMesh* __restrict__ tab, const float* __restrict__ ub,
                            const float* __restrict__ rb, int nr) {
  const DevMesh& m = tab[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.n2) return;
  if (!m.active) return;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    m.u[3 * (size_t)i + d] = (double)ub[(size_t)i * nr + 3 * m.col + d];
    m.rf[3 * (size_t)(m.n1 + i) + d] = rb[(size_t)(m.n1 + i) * nr + 3 * m.col + d];
  }
}

// dx of every active frame from its float64 solution r (solver order); zero
// on pinned vertices
__global__ void k_scatter_dx_b(const DevMesh* __restrict__ tab) {
  const DevMesh& m = tab[blockIdx.y];
  if (!m.active) return;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= m.n) return;
  const int p = m.pos[v];
#pragma unroll
  for (int d = 0; d < 3; ++d) m.dx[3 * (size_t)v + d] = p >= 0 ? m.r[3 * (size_t)p + d] : 0.0;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Forward pass over the levels (leaves to root): y_J = L_JJ^-1 b_J on the
// x1 positions, b_R -= L_RJ y_J on every off-diagonal row (x1 and x2).
template <typename T>
void trisolve_fwd(cudaStream_t s, const DevMesh& m, const T* Z, T* b, T* y, bool wide) {
  for (int l = 0; l < m.n_levels; ++l) {
    const int a = m.h_fwd_ptr[l], e = m.h_fwd_ptr[l + 1];
    if (e <= a) continue;
    const size_t sm = sizeof(T) * 3 * (size_t)m.h_level_maxns[l];
    ProfScope ps(PROF_TRSV_FWD, s);
    if (wide)
      k_fwd_chunk<T, 1024><<<e - a, 1024, sm, s>>>(m.fwd_items + a, m.sn_c0, m.sn_ns, m.sn_nr1,
                                                   m.sn_roff, m.sn_zoff, m.sn_rows, Z, b, y);
    else
      k_fwd_chunk<T, 256><<<e - a, 256, sm, s>>>(m.fwd_items + a, m.sn_c0, m.sn_ns, m.sn_nr1,
                                                 m.sn_roff, m.sn_zoff, m.sn_rows, Z, b, y);
    count_launch();
  }
}

// Backward pass (root to leaves): x_J = L_JJ^-T (y_J - L_RJ^T x_R), reading
// x_R from b (x1 ancestors solved earlier, x2 rows = dx2), writing b on x1.
template <typename T>
void trisolve_bwd(cudaStream_t s, const DevMesh& m, const T* Z, const T* y, T* b, bool wide) {
  for (int l = m.n_levels - 1; l >= 0; --l) {
    const int a = m.h_bwd_ptr[l], e = m.h_bwd_ptr[l + 1];
    if (e <= a) continue;
    const size_t sm = sizeof(T) * 3 * (size_t)m.h_level_maxld[l];
    ProfScope ps(PROF_TRSV_BWD, s);
    if (wide)
      k_bwd_chunk<T, 1024><<<e - a, 1024, sm, s>>>(m.bwd_items + a, m.sn_c0, m.sn_ns, m.sn_nr1,
                                                   m.sn_roff, m.sn_zoff, m.sn_rows, Z, y, b);
    else
      k_bwd_chunk<T, 256><<<e - a, 256, sm, s>>>(m.bwd_items + a, m.sn_c0, m.sn_ns, m.sn_nr1,
                                                 m.sn_roff, m.sn_zoff, m.sn_rows, Z, y, b);
    count_launch();
  }
}

// Columns j0 .. j0+2 of Phi = K11^-1 K12 Sigma^-1 come from one backward
// pass with y1 = 0 and x2 = Sigma^-1 e_j (one column per right-hand side):
// x1 = L1^-T (0 - L21^T Sigma^-1 e_j) = -Phi e_j.
__global__ void k_phi_rhs(int n1, int n2, int j0, const double* __restrict__ Sinv,
                          double* __restrict__ y1, double* __restrict__ b) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 3 * n1) y1[e] = 0.0;
  if (e < 3 * n2) {
    const int q = e / 3, d = e % 3;
    b[3 * (size_t)n1 + e] = (j0 + d < n2) ? Sinv[(size_t)q * n2 + j0 + d] : 0.0;
  }
}

__global__ void k_phi_store(int n1, int n2, int j0, const double* __restrict__ b,
                            float* __restrict__ phi_t) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * n1) return;
  const int p = e / 3, d = e % 3;
  if (j0 + d < n2) phi_t[(size_t)(j0 + d) * n1 + p] = (float)(-b[e]);
}

// Eq. 8 with H = K (x) I_3 in solver positions [x1 ; x2], r = -g-hat:
//   lower:    z1 = L1^-1 r1,  y2 = r2 - L21 z1        (one forward pass; the
//             x2 rows of the supernodes hold L21 = H21 L1^-T)
//   diagonal: dx2 = Sigma-hat^-1 y2 = u - Sigma^-1 Q^T v,  u = Sigma^-1 y2
//   upper:    dx1 = L1^-T (z1 - L21^T dx2)             (one backward pass)
template <typename T>
cudaError_t global_step_t(cudaStream_t s, const DevMesh& m, const double* g, double* dx, int* info,
                          int num_sms, bool wide, bool dense_schur, int nc_host) {
  const int nf = m.nf, n1 = m.n1, n2 = m.n2;
  const bool f64 = std::is_same<T, double>::value;
  double* r = m.r;                                  // float64 work (nf * 3)
  T* b = f64 ? (T*)m.r : (T*)m.rf;                  // solve vector (nf * 3)
  T* y = f64 ? (T*)m.y1 : (T*)m.y1f;                // forward result on x1 (n1 * 3)
  const T* Z = f64 ? (const T*)m.Z : (const T*)m.Zf;
  k_gather_rhs<T><<<nblk(nf, 256), 256, 0, s>>>(nf, m.perm, g, b);
  count_launch();
  // the reduced system's factorisation needs only B-check and Sigma^-1: in
  // mixed precision it starts on the side stream and overlaps the forward solve
  const bool prepared = !f64 && !dense_schur && n2 > 0 &&
                        reduced_prepare(s, m, m.u, b + 3 * (size_t)n1, r + 3 * (size_t)n1, info,
                                        num_sms, nc_host);
  if (n1 > 0) trisolve_fwd<T>(s, m, Z, b, y, wide);
  if (n2 > 0) {
    T* y2 = b + 3 * (size_t)n1;
    double* u = m.u;
    double* z2 = r + 3 * (size_t)n1;                // float64 dx2
    // With Phi available the x1 block is split: x1 = L1^-T (y1 - L21^T u)
    // (contact-free, on the side stream while the reduced system is solved)
    // + Phi[:, c] v after it, instead of a backward pass after z2.
    const bool phi = prepared && m.Phi_t && m.bx && n1 > 0;
    if (phi) {
      {
        ProfScope psg(PROF_GEMV, s);
        k_gemv3<float><<<nblk(n2, 8), 256, 0, s>>>(n2, m.Sinvf, (const float*)y2, m.uf);
        k_convert<float, double><<<nblk(3 * (int64_t)n2, 256), 256, 0, s>>>(3 * n2, m.uf, u);
        count_launch(2);
      }
      cudaStream_t s2 = m.aux_stream;
      if (cudaEventRecord(m.ev_fork2, s) != cudaSuccess || cudaStreamWaitEvent(s2, m.ev_fork2, 0) != cudaSuccess)
        return cudaGetLastError();
      k_convert<float, float><<<nblk(3 * (int64_t)n2, 256), 256, 0, s2>>>(3 * n2, m.uf, m.bx + 3 * (size_t)n1);
      count_launch();
      trisolve_bwd<float>(s2, m, m.Zf, m.y1f, m.bx, false);
      if (cudaEventRecord(m.ev_join2, s2) != cudaSuccess) return cudaGetLastError();
      {
        ProfScope psr(PROF_REDUCED, s);
        const cudaError_t e = reduced_solve(s, m, u, y2, z2, info, num_sms, 1, nc_host, true);
        if (e != cudaSuccess) return e;
      }
      if (cudaStreamWaitEvent(s, m.ev_join2, 0) != cudaSuccess) return cudaGetLastError();
      const cudaError_t e = phi_apply(s, m, u, y2, z2, info, m.bx, r);
      if (e != cudaSuccess) return e;
      cudaMemsetAsync(dx, 0, sizeof(double) * 3 * (size_t)m.n, s);
      k_scatter_dx<<<nblk(nf, 256), 256, 0, s>>>(nf, m.perm, r, dx);
      count_launch();
      return cudaGetLastError();
    }
    if (dense_schur) {
      // Schur-only configuration: Sigma-hat factored densely (k_schur.cu)
      const cudaError_t e = sigma_hat_solve(s, m, y2, z2, info, f64 ? 0 : 1);
      if (e != cudaSuccess) return e;
    } else {
      {
        ProfScope psg(PROF_GEMV, s);
        if (f64) {
          k_gemv3<double><<<nblk(n2, 8), 256, 0, s>>>(n2, m.Sinv, (const double*)y2, u);
          count_launch();
        } else {
          float* uf = m.uf;
          k_gemv3<float><<<nblk(n2, 8), 256, 0, s>>>(n2, m.Sinvf, (const float*)y2, uf);
          k_convert<float, double><<<nblk(3 * (int64_t)n2, 256), 256, 0, s>>>(3 * n2, uf, u);
          count_launch(2);
        }
      }
      // The reduced system carries the barrier stiffness (cond ~ kappa b''):
      // float64 factors, or float32 factors refined with float64 residuals.
      // n_c is read on the device (z2 = u when it is 0).
      ProfScope psr(PROF_REDUCED, s);
      const cudaError_t e = reduced_solve(s, m, u, y2, z2, info, num_sms, f64 ? 0 : 1, nc_host,
                                          prepared);
      if (e != cudaSuccess) return e;
    }
    if (!f64) {
      k_convert<double, T><<<nblk(3 * (int64_t)n2, 256), 256, 0, s>>>(3 * n2, z2, y2);
      count_launch();
    }
  }
  if (n1 > 0) trisolve_bwd<T>(s, m, Z, y, b, wide);
  if (!f64) {
    k_convert<T, double><<<nblk(3 * (int64_t)n1, 256), 256, 0, s>>>(3 * n1, b, r);
    count_launch();
  }
  cudaMemsetAsync(dx, 0, sizeof(double) * 3 * (size_t)m.n, s);
  k_scatter_dx<<<nblk(nf, 256), 256, 0, s>>>(nf, m.perm, r, dx);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t global_step_b(const BatchStep& bs) {
  const DevMesh& m = *bs.m0;
  cudaStream_t s = bs.s, s2 = bs.s2;
  const int nb = bs.nb, nr = bs.nr, n1 = m.n1, n2 = m.n2, nf = m.nf;
  const int chunks = nr / kMrCols;
  k_gather_rhs_mr<<<dim3((nf + 255) / 256, nb), 256, 0, s>>>(bs.tab, bs.rb, nr);
  count_launch();
  // S, L_s, block lists, X, N of every frame need only B-check and Sigma^-1:
  // on the side stream, overlapping the forward solve
  if (cudaEventRecord(bs.ev[0], s) != cudaSuccess || cudaStreamWaitEvent(s2, bs.ev[0], 0) != cudaSuccess)
    return cudaGetLastError();
  cudaError_t e = reduced_prepare_b(s2, bs.args_dev, nb, bs.num_sms);
  if (e != cudaSuccess) return e;
  if (cudaEventRecord(bs.ev[1], s2) != cudaSuccess) return cudaGetLastError();
  for (int l = 0; l < m.n_levels && n1 > 0; ++l) {
    const int a = m.h_fwd_ptr[l], z = m.h_fwd_ptr[l + 1];
    if (z <= a) continue;
    ProfScope ps(PROF_TRSV_FWD, s);
    const size_t sm = sizeof(float) * kMrCols * (size_t)m.h_level_maxns[l];
    k_fwd_mr<<<dim3(z - a, chunks), 256, sm, s>>>(m.fwd_items + a, m.sn_c0, m.sn_ns, m.sn_nr1,
                                                   m.sn_roff, m.sn_zoff, m.sn_rows, m.Zf, bs.rb,
                                                   bs.yb, nr, nf);
    count_launch();
  }
  {
    ProfScope ps(PROF_GEMV, s);
    // u = Sigma^-1 y2 on the tensor cores (3xTF32); the SIMT product where
    // the descriptors could not be made
    if (bs.use_tc && tc_sinv_supported(m, nr)) {
      e = launch_sinv_tc(s, m, bs.rb + (size_t)n1 * nr, nr, bs.ub, bs.num_sms, m.counters + 15);
      if (e != cudaSuccess) return e;
    } else {
      k_gemm_mr<<<dim3((n2 + 31) / 32, chunks), 256, 0, s>>>(n2, m.Sinvf, bs.rb + (size_t)n1 * nr,
                                                             bs.ub, nr);
      count_launch();
    }
    k_unpack_mr<<<dim3((n2 + 255) / 256, nb), 256, 0, s>>>(bs.tab, bs.ub, bs.rb, nr);
    count_launch();
    // x2 rows of the contact-free backward solve = u, all columns (same row stride)
    e = cudaMemcpyAsync(bs.bx + (size_t)n1 * nr, bs.ub, sizeof(float) * (size_t)n2 * nr,
                        cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  // the contact-free backward solve x1 = L1^-T (y1 - L21^T u) on the side
  // stream while the reduced systems are solved
  // x1 rows of the backward solution accumulate atomically: zeroed first
  if (n1 > 0 && cudaMemsetAsync(bs.bx, 0, sizeof(float) * (size_t)n1 * nr, s2) != cudaSuccess)
    return cudaGetLastError();
  if (cudaEventRecord(bs.ev[2], s) != cudaSuccess || cudaStreamWaitEvent(s2, bs.ev[2], 0) != cudaSuccess)
    return cudaGetLastError();
  for (int l = m.n_levels - 1; l >= 0 && n1 > 0; --l) {
    const int a = m.h_bwd32_ptr[l], z = m.h_bwd32_ptr[l + 1];
    if (z <= a) continue;
    ProfScope ps(PROF_TRSV_BWD, s2);
    k_bwd_mr<<<dim3(z - a, chunks), 256, 0, s2>>>(m.bwd_items32 + a, m.sn_c0, m.sn_ns, m.sn_nr1,
                                                  m.sn_roff, m.sn_zoff, m.sn_rows, m.Zf, bs.yb,
                                                  bs.bx, nr, nf);
    count_launch();
  }
  if (cudaEventRecord(bs.ev[3], s2) != cudaSuccess) return cudaGetLastError();
  if (cudaStreamWaitEvent(s, bs.ev[1], 0) != cudaSuccess) return cudaGetLastError();
  {
    ProfScope ps(PROF_REDUCED, s);
    e = reduced_solve_b(s, bs.args_dev, bs.args_host, nb, bs.nc_host, bs.num_sms);
    if (e != cudaSuccess) return e;
  }
  if (cudaStreamWaitEvent(s, bs.ev[3], 0) != cudaSuccess) return cudaGetLastError();
  e = phi_apply_b(s, bs.args_dev, bs.cols_dev, nb, n1, m.Phi_t, bs.bx, nr, bs.x1s_dev);
  if (e != cudaSuccess) return e;
  k_scatter_dx_b<<<dim3((m.n + 255) / 256, nb), 256, 0, s>>>(bs.tab);
  count_launch();
  return cudaGetLastError();
}

FSIM_CHECK_READER(check_word_solve)

cudaError_t launch_sinv_simt(cudaStream_t s, const DevMesh& m, const float* Y, int nr, float* U) {
  k_gemm_mr<<<dim3((m.n2 + 31) / 32, nr / kMrCols), 256, 0, s>>>(m.n2, m.Sinvf, Y, U, nr);
  count_launch();
  return cudaGetLastError();
}

bool batch_supported(const DevMesh& m, int nr) {
  if (!m.Zf || !m.Phi_t || !m.Sinvf || m.n1 <= 0 || m.n2 <= 0 || nr % kMrCols != 0) return false;
  int maxns = 0;
  for (int l = 0; l < m.n_levels; ++l) maxns = std::max(maxns, m.h_level_maxns[l]);
  return sizeof(float) * kMrCols * (size_t)maxns <= 160 * 1024;
}

void set_solver_smem_limits(int max_bytes) {
  // k_fwd_mr: its staged right-hand sides (ns x 32 floats) beside 48 KB of
  // static shared memory; batch_supported keeps ns x 128 B within 160 KB
  cudaFuncSetAttribute(k_fwd_mr, cudaFuncAttributeMaxDynamicSharedMemorySize, 170 * 1024);
  tc_set_smem_limits();
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaFuncSetAttribute(k_fwd_chunk<double, 256>, a, max_bytes);
  cudaFuncSetAttribute(k_bwd_chunk<double, 256>, a, max_bytes);
  cudaFuncSetAttribute(k_fwd_chunk<float, 256>, a, max_bytes);
  cudaFuncSetAttribute(k_bwd_chunk<float, 256>, a, max_bytes);
  cudaFuncSetAttribute(k_fwd_chunk<double, 1024>, a, max_bytes);
  cudaFuncSetAttribute(k_bwd_chunk<double, 1024>, a, max_bytes);
  cudaFuncSetAttribute(k_fwd_chunk<float, 1024>, a, max_bytes);
  cudaFuncSetAttribute(k_bwd_chunk<float, 1024>, a, max_bytes);
}

cudaError_t compute_phi(cudaStream_t s, const DevMesh& m, float* phi_t) {
  const int n1 = m.n1, n2 = m.n2;
  const int nb = nblk(3 * (int64_t)std::max(n1, n2), 256);
  for (int j0 = 0; j0 < n2; j0 += 3) {
    k_phi_rhs<<<nb, 256, 0, s>>>(n1, n2, j0, m.Sinv, m.y1, m.r);
    trisolve_bwd<double>(s, m, m.Z, m.y1, m.r, false);
    k_phi_store<<<nblk(3 * (int64_t)n1, 256), 256, 0, s>>>(n1, n2, j0, m.r, phi_t);
    count_launch(2);
  }
  return cudaGetLastError();
}

cudaError_t global_step(cudaStream_t s, const DevMesh& m, const double* g, double* dx, int precision,
                        int* info_dev, int num_sms, bool alone, bool dense_schur, int nc_host) {
  // 32-warp solve items only for a float32 solve that has the GPU to itself
  if (precision == 0)
    return global_step_t<double>(s, m, g, dx, info_dev, num_sms, false, dense_schur, nc_host);
  return global_step_t<float>(s, m, g, dx, info_dev, num_sms, alone, dense_schur, nc_host);
}

}  // namespace fsim
