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
// so that one large supernode spreads over many CTAs.  Forward item: rows
// [r0, r0+32) of Z_J times b_J; lanes own rows (coalesced column-major reads),
// the 8 warps split the inner index and reduce through shared memory.
template <typename T>
__global__ void __launch_bounds__(256)
k_fwd_chunk(const int4* __restrict__ items, const int* __restrict__ c0a, const int* __restrict__ nsa,
            const int* __restrict__ nra, const int64_t* __restrict__ roff,
            const int64_t* __restrict__ zoff, const int* __restrict__ rows,
            const T* __restrict__ Z, T* __restrict__ b, T* __restrict__ y) {
  extern __shared__ unsigned char smem_raw[];
  T* bj = reinterpret_cast<T*>(smem_raw);
  __shared__ T part[8][32][3];
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
    for (int k = wid; k < kmax; k += 8) {
      const T z = Zj[(size_t)k * ld + r];
      a0 += z * bj[3 * k]; a1 += z * bj[3 * k + 1]; a2 += z * bj[3 * k + 2];
    }
  }
  part[wid][lane][0] = a0; part[wid][lane][1] = a1; part[wid][lane][2] = a2;
  __syncthreads();
  if (wid == 0 && lane < rn) {
#pragma unroll
    for (int w = 1; w < 8; ++w) { a0 += part[w][lane][0]; a1 += part[w][lane][1]; a2 += part[w][lane][2]; }
    if (r < ns) {
      T* o = y + 3 * (size_t)(c0 + r);
      o[0] = a0; o[1] = a1; o[2] = a2;
    } else {
      T* o = b + 3 * (size_t)rows[roff[J] + r - ns];
      atomicAdd(o, -a0); atomicAdd(o + 1, -a1); atomicAdd(o + 2, -a2);
    }
  }
}

// Backward item: columns [k0, k0+kn) of Z_J^T [y_J ; -x_R]; one warp per column.
// Reads y (forward result) and the ancestors' x, writes x_J (x may alias b).
template <typename T>
__global__ void __launch_bounds__(256)
k_bwd_chunk(const int4* __restrict__ items, const int* __restrict__ c0a, const int* __restrict__ nsa,
            const int* __restrict__ nra, const int64_t* __restrict__ roff,
            const int64_t* __restrict__ zoff, const int* __restrict__ rows,
            const T* __restrict__ Z, const T* __restrict__ y, T* __restrict__ x) {
  extern __shared__ unsigned char smem_raw[];
  T* wv = reinterpret_cast<T*>(smem_raw);
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
  T res[3] = {0, 0, 0};
  for (int kk = wid; kk < kn; kk += 8) {
    const int k = k0 + kk;
    const T* zc = Zj + (size_t)k * ld;
    T a0 = 0, a1 = 0, a2 = 0;
    for (int r = k + lane; r < ld; r += 32) {
      const T z = zc[r];
      a0 += z * wv[3 * r]; a1 += z * wv[3 * r + 1]; a2 += z * wv[3 * r + 2];
    }
    a0 = warp_sum_t(a0); a1 = warp_sum_t(a1); a2 = warp_sum_t(a2);
    res[0] = a0; res[1] = a1; res[2] = a2;
    __syncwarp();
    if (lane == 0) {
      T* o = x + 3 * (size_t)(c0 + k);
      o[0] = res[0]; o[1] = res[1]; o[2] = res[2];
    }
  }
}

// y[i] -= sum_e val[e] * x[col[e]]   (3-vectors; K (x) I_3 applied blockwise)
template <typename T>
__global__ void k_spmv3_sub(int nrows, const int* __restrict__ ptr, const int* __restrict__ col,
                            const double* __restrict__ val, const T* __restrict__ x,
                            T* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  T a0 = 0, a1 = 0, a2 = 0;
  for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
    const T v = (T)val[e];
    const T* xs = x + 3 * (size_t)col[e];
    a0 += v * xs[0]; a1 += v * xs[1]; a2 += v * xs[2];
  }
  y[3 * (size_t)i] -= a0; y[3 * (size_t)i + 1] -= a1; y[3 * (size_t)i + 2] -= a2;
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
// reduced system kernels (row-major dense, T = double or float)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gather_S(int nc, const int* __restrict__ clist, const T* __restrict__ Sinv,
                           int n2, T* __restrict__ S) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nc * nc) return;
  const int i = idx / nc, j = idx % nc;
  S[idx] = Sinv[(size_t)clist[i] * n2 + clist[j]];
}

// per-row compaction of the block occupancy: list[i*nc + k], cnt[i]
__global__ void k_block_lists(int nc, const int* __restrict__ bocc, int* __restrict__ list,
                              int* __restrict__ cnt) {
  const int i = blockIdx.x;
  if (i >= nc) return;
  const int lane = threadIdx.x;   // one warp
  int base = 0;
  for (int j0 = 0; j0 < nc; j0 += 32) {
    const int j = j0 + lane;
    const bool f = j < nc && bocc[(size_t)i * nc + j] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (f) list[(size_t)i * nc + base + __popc(m & ((1u << lane) - 1u))] = j;
    base += __popc(m);
  }
  if (lane == 0) cnt[i] = base;
}

// X = B (L (x) I_3): X[(i,a),(k,b)] = sum_{j in occ(i), j >= k} B[(i,a),(j,b)] L[j][k]
template <typename T>
__global__ void k_form_X(int nc, const double* __restrict__ Bc, const T* __restrict__ L,
                         const int* __restrict__ list, const int* __restrict__ cnt, T* __restrict__ X) {
  const int n3 = 3 * nc;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n3 * n3) return;
  const int row = (int)(idx / n3), colx = (int)(idx % n3);
  const int i = row / 3, k = colx / 3, b = colx % 3;
  const double* brow = Bc + (size_t)row * n3;
  T acc = 0;
  const int c = cnt[i];
  for (int e = 0; e < c; ++e) {
    const int j = list[(size_t)i * nc + e];
    if (j < k) continue;
    acc += (T)brow[3 * j + b] * L[(size_t)j * nc + k];
  }
  X[idx] = acc;
}

// y = B u_c (over occupied blocks), y[(i,a)]
__global__ void k_bmv(int nc, const double* __restrict__ Bc, const int* __restrict__ list,
                      const int* __restrict__ cnt, const int* __restrict__ clist,
                      const double* __restrict__ u, double* __restrict__ y) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int n3 = 3 * nc;
  if (row >= n3) return;
  const int i = row / 3;
  const double* brow = Bc + (size_t)row * n3;
  double acc = 0.0;
  for (int e = 0; e < cnt[i]; ++e) {
    const int j = list[(size_t)i * nc + e];
    const double* uj = u + 3 * (size_t)clist[j];
    acc += brow[3 * j] * uj[0] + brow[3 * j + 1] * uj[1] + brow[3 * j + 2] * uj[2];
  }
  y[row] = acc;
}

// N = I + (L (x) I_3)^T X (full), and the augmented last row t0 = (L (x) I_3)^T y
// N[(i,a),(k,b)] = delta + sum_{j >= i} L[j][i] X[(j,a),(k,b)]
template <typename T>
__global__ void k_form_N(int nc, const T* __restrict__ L, const T* __restrict__ X,
                         const double* __restrict__ y, T* __restrict__ N) {
  const int n3 = 3 * nc;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)(n3 + 1) * n3) return;
  const int row = (int)(idx / n3), col = (int)(idx % n3);
  if (row < n3) {
    const int i = row / 3, a = row % 3;
    T acc = (row == col) ? T(1) : T(0);
    for (int j = i; j < nc; ++j) acc += L[(size_t)j * nc + i] * X[(size_t)(3 * j + a) * n3 + col];
    N[idx] = acc;
  } else {
    const int i = col / 3, a = col % 3;
    T acc = 0;
    for (int j = i; j < nc; ++j) acc += L[(size_t)j * nc + i] * (T)y[3 * j + a];
    N[idx] = acc;
  }
}

__device__ __forceinline__ double sqrt_any(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_any(float v) { return sqrtf(v); }

// Right-looking blocked Cholesky (lower, row-major, ld) of the leading N x N
// block of an (N + extra) x N matrix, in one cooperative launch.  The extra
// rows receive L_extra = A_extra L^-T.  CTA 0 factors each diagonal block
// right after updating it (look-ahead) while the other CTAs update the rest.
template <typename T>
__global__ void __launch_bounds__(256) k_chol_coop(T* __restrict__ A, int N, int extra, int ld,
                                                   int* __restrict__ info) {
  cg::grid_group grid = cg::this_grid();
  __shared__ T D[32][33];
  __shared__ T Pi[32][33];
  __shared__ T Pj[32][33];
  const int M = N + extra;
  const int tid = threadIdx.x, nthr = blockDim.x;

  auto factor_diag = [&](int k0) {
    const int kb = min(32, N - k0);
    for (int e = tid; e < kb * kb; e += nthr) {
      const int i = e / kb, j = e % kb;
      D[i][j] = (j <= i) ? A[(size_t)(k0 + i) * ld + k0 + j] : T(0);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
      if (tid == 0) {
        T d = D[j][j];
        if (!(d > T(0))) { atomicOr(info, 1); d = T(1); }
        D[j][j] = sqrt_any(d);
      }
      __syncthreads();
      for (int i = j + 1 + tid; i < kb; i += nthr) D[i][j] /= D[j][j];
      __syncthreads();
      const int m = kb - j - 1;
      for (int e = tid; e < m * m; e += nthr) {
        const int i = j + 1 + e / m, c = j + 1 + e % m;
        if (c <= i) D[i][c] -= D[i][j] * D[c][j];
      }
      __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += nthr) {
      const int i = e / kb, j = e % kb;
      A[(size_t)(k0 + i) * ld + k0 + j] = (j <= i) ? D[i][j] : T(0);
    }
    __syncthreads();
  };

  if (blockIdx.x == 0) factor_diag(0);
  grid.sync();
  for (int k0 = 0; k0 < N; k0 += 32) {
    const int kb = min(32, N - k0);
    const int k1 = k0 + kb;
    // (1) panel: rows [k1, M) of columns [k0, k1) := A L_kk^-T, 8 rows per CTA step
    for (int e = tid; e < kb * kb; e += nthr) {
      const int i = e / kb, j = e % kb;
      D[i][j] = A[(size_t)(k0 + i) * ld + k0 + j];
    }
    __syncthreads();
    {
      const int nrow = M - k1;
      const int lane = tid & 31, wid = tid >> 5;
      // one warp per row: lanes hold the row's kb entries; forward substitution
      for (int r = blockIdx.x * (nthr >> 5) + wid; r < nrow; r += gridDim.x * (nthr >> 5)) {
        T* arow = A + (size_t)(k1 + r) * ld + k0;
        T xv = (lane < kb) ? arow[lane] : T(0);
        for (int j = 0; j < kb; ++j) {
          const T xj = __shfl_sync(0xffffffffu, xv, j) / D[j][j];
          if (lane == j) xv = xj;
          if (lane > j && lane < kb) xv -= xj * D[lane][j];
        }
        if (lane < kb) arow[lane] = xv;
      }
    }
    grid.sync();
    // (2) trailing update of rows [k1, M) x cols [k1, N), lower part (tiles)
    if (k1 < N) {
      const int nrb = (M - k1 + 31) / 32;
      const int ncb = (N - k1 + 31) / 32;
      // enumerate tiles (rb, cb) with cb <= rb (cb < ncb); tile 0 = next diagonal
      int ntiles = 0;
      for (int rb = 0; rb < nrb; ++rb) ntiles += min(rb + 1, ncb);
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int rb = 0, rem = tile;
        while (rem >= min(rb + 1, ncb)) { rem -= min(rb + 1, ncb); ++rb; }
        const int cb = rem;
        const int r0 = k1 + rb * 32, c0 = k1 + cb * 32;
        const int rn = min(32, M - r0), cn = min(32, N - c0);
        for (int e = tid; e < 32 * kb; e += nthr) {
          const int i = e / kb, l = e % kb;
          Pi[i][l] = (i < rn) ? A[(size_t)(r0 + i) * ld + k0 + l] : T(0);
          Pj[i][l] = (i < cn) ? A[(size_t)(c0 + i) * ld + k0 + l] : T(0);
        }
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += nthr) {
          const int i = e >> 5, j = e & 31;
          if (i < rn && j < cn && (r0 + i >= c0 + j || r0 + i >= N)) {
            T acc = 0;
            for (int l = 0; l < kb; ++l) acc += Pi[i][l] * Pj[j][l];
            A[(size_t)(r0 + i) * ld + c0 + j] -= acc;
          }
        }
        __syncthreads();
        if (tile == 0) factor_diag(k1);   // look-ahead: next diagonal block is final
      }
    }
    grid.sync();
  }
}

// Single-CTA backward solve L^T x = b (L lower, row-major ld, n x n) for nrhs
// right-hand sides stored x[i*nrhs + r]; b is overwritten by x.
template <typename T>
__global__ void k_trsv_lt(const T* __restrict__ L, int n, int ld, T* __restrict__ b, int nrhs) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  __shared__ T xs[32][4];
  for (int i1 = n; i1 > 0; i1 -= 32) {
    const int i0 = max(0, i1 - 32), nb = i1 - i0;
    // solve the diagonal block (rows i0..i1) by warp 0, lanes = rhs*? (sequential over rows)
    if (tid < 32) {
      for (int r = 0; r < nrhs; ++r) {
        T xv = (tid < nb) ? b[(size_t)(i0 + tid) * nrhs + r] : T(0);
        for (int j = nb - 1; j >= 0; --j) {
          const T xj = __shfl_sync(0xffffffffu, xv, j) / L[(size_t)(i0 + j) * ld + i0 + j];
          if (tid == j) xv = xj;
          if (tid < j) xv -= L[(size_t)(i0 + j) * ld + i0 + tid] * xj;
        }
        if (tid < nb) { b[(size_t)(i0 + tid) * nrhs + r] = xv; xs[tid][r] = xv; }
      }
    }
    __syncthreads();
    // update rows above: b[i] -= sum_{j in block} L[j][i] x[j]
    for (int e = tid; e < i0 * nrhs; e += nthr) {
      const int i = e / nrhs, r = e % nrhs;
      T acc = 0;
      for (int j = 0; j < nb; ++j) acc += L[(size_t)(i0 + j) * ld + i] * xs[j][r];
      b[(size_t)i * nrhs + r] -= acc;
    }
    __syncthreads();
  }
}

// z2[q] = u[q] - sum_m Sinv[q, c_m] v[m]   (3-vectors), one warp per row q
template <typename T>
__global__ void k_z2(int n2, int nc, const T* __restrict__ Sinv, const int* __restrict__ clist,
                     const T* __restrict__ v, const double* __restrict__ u, double* __restrict__ z) {
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= n2) return;
  const T* a = Sinv + (size_t)q * n2;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int m = lane; m < nc; m += 32) {
    const double s = (double)a[clist[m]];
    a0 += s * (double)v[3 * m]; a1 += s * (double)v[3 * m + 1]; a2 += s * (double)v[3 * m + 2];
  }
  a0 = warp_sum_t(a0); a1 = warp_sum_t(a1); a2 = warp_sum_t(a2);
  if (lane == 0) {
    z[3 * q] = u[3 * q] - a0; z[3 * q + 1] = u[3 * q + 1] - a1; z[3 * q + 2] = u[3 * q + 2] - a2;
  }
}

__global__ void k_zero_upper(int n, int ld, double* A) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (j > i) A[(size_t)i * ld + j] = 0.0;
}

template <typename T>
__global__ void k_zero_upper_t(int n, int ld, T* A) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (j > i) A[(size_t)i * ld + j] = T(0);
}

// gather (augmented row -> vector) helper: x[i] = A[row*ld + i]
template <typename T>
__global__ void k_copy_row(int n, const T* __restrict__ A, int row, int ld, T* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = A[(size_t)row * ld + i];
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Forward pass over the levels (leaves to root): y_J = L_JJ^-1 b_J on the
// x1 positions, b_R -= L_RJ y_J on every off-diagonal row (x1 and x2).
template <typename T>
void trisolve_fwd(cudaStream_t s, const DevMesh& m, const T* Z, T* b, T* y) {
  for (int l = 0; l < m.n_levels; ++l) {
    const int a = m.h_fwd_ptr[l], e = m.h_fwd_ptr[l + 1];
    if (e <= a) continue;
    const size_t sm = sizeof(T) * 3 * (size_t)m.h_level_maxns[l];
    ProfScope ps(PROF_TRSV_FWD, s);
    k_fwd_chunk<T><<<e - a, 256, sm, s>>>(m.fwd_items + a, m.sn_c0, m.sn_ns, m.sn_nr1, m.sn_roff,
                                          m.sn_zoff, m.sn_rows, Z, b, y);
    count_launch();
  }
}

// Backward pass (root to leaves): x_J = L_JJ^-T (y_J - L_RJ^T x_R), reading
// x_R from b (x1 ancestors solved earlier, x2 rows = dx2), writing b on x1.
template <typename T>
void trisolve_bwd(cudaStream_t s, const DevMesh& m, const T* Z, const T* y, T* b) {
  for (int l = m.n_levels - 1; l >= 0; --l) {
    const int a = m.h_bwd_ptr[l], e = m.h_bwd_ptr[l + 1];
    if (e <= a) continue;
    const size_t sm = sizeof(T) * 3 * (size_t)m.h_level_maxld[l];
    ProfScope ps(PROF_TRSV_BWD, s);
    k_bwd_chunk<T><<<e - a, 256, sm, s>>>(m.bwd_items + a, m.sn_c0, m.sn_ns, m.sn_nr1, m.sn_roff,
                                          m.sn_zoff, m.sn_rows, Z, y, b);
    count_launch();
  }
}

template <typename T>
void launch_chol(cudaStream_t s, T* A, int N, int extra, int ld, int* info, int num_sms) {
  if (N <= 0) return;
  int tiles = (N + 31) / 32;
  int grid = std::max(1, std::min(num_sms, tiles * (tiles + 1) / 2));
  void* args[] = {&A, &N, &extra, &ld, &info};
  ProfScope ps(PROF_CHOL, s);
  cudaLaunchCooperativeKernel((void*)k_chol_coop<T>, dim3(grid), dim3(256), args, 0, s);
  count_launch();
}

// Reduced push-through system (Eq. 11 reading): z2 = u - Sinv[:,c] v.
template <typename T>
void reduced_solve(cudaStream_t s, const DevMesh& m, const T* Sinv, int nc, const double* u,
                   double* z2, int* info, int num_sms) {
  const int n3 = 3 * nc;
  // workspace layout inside m.red / m.redf (capacity red_cap elements)
  T* base = std::is_same<T, double>::value ? (T*)m.red : (T*)m.redf;
  T* S = base;                                  // nc*nc (-> L_s)
  T* X = S + (size_t)nc * nc;                   // n3*n3
  T* N = X + (size_t)n3 * n3;                   // (n3+1)*n3
  T* tv = N + (size_t)(n3 + 1) * n3;            // n3 (t, then v)
  double* y = m.red + m.red_cap - (size_t)n3 - 8;  // float64 B u_c (tail of m.red)
  int* list = m.bocc + (size_t)nc * nc;         // nc*nc block lists (after bocc)
  int* cnt = list + (size_t)nc * nc;
  k_gather_S<T><<<nblk((int64_t)nc * nc, 256), 256, 0, s>>>(nc, m.clist, Sinv, m.n2, S);
  launch_chol<T>(s, S, nc, 0, nc, info, num_sms);
  k_zero_upper_t<T><<<nblk((int64_t)nc * nc, 256), 256, 0, s>>>(nc, nc, S);
  k_block_lists<<<nc, 32, 0, s>>>(nc, m.bocc, list, cnt);
  k_form_X<T><<<nblk((int64_t)n3 * n3, 256), 256, 0, s>>>(nc, m.Bc, S, list, cnt, X);
  k_bmv<<<nblk(n3, 128), 128, 0, s>>>(nc, m.Bc, list, cnt, m.clist, u, y);
  k_form_N<T><<<nblk((int64_t)(n3 + 1) * n3, 256), 256, 0, s>>>(nc, S, X, y, N);
  launch_chol<T>(s, N, n3, 1, n3, info, num_sms);
  k_copy_row<T><<<nblk(n3, 256), 256, 0, s>>>(n3, N, n3, n3, tv);
  k_trsv_lt<T><<<1, 1024, 0, s>>>(N, n3, n3, tv, 1);       // t = L_N^-T l
  k_trsv_lt<T><<<1, 1024, 0, s>>>(S, nc, nc, tv, 3);       // v = (L_s (x) I)^-T t
  k_z2<T><<<nblk(m.n2, 8), 256, 0, s>>>(m.n2, nc, Sinv, m.clist, tv, u, z2);
  count_launch(9);
}

// Eq. 8 with H = K (x) I_3 in solver positions [x1 ; x2], r = -g-hat:
//   lower:    z1 = L1^-1 r1,  y2 = r2 - L21 z1        (one forward pass; the
//             x2 rows of the supernodes hold L21 = H21 L1^-T)
//   diagonal: dx2 = Sigma-hat^-1 y2 = u - Sigma^-1 Q^T v,  u = Sigma^-1 y2
//   upper:    dx1 = L1^-T (z1 - L21^T dx2)             (one backward pass)
template <typename T>
void global_step_t(cudaStream_t s, const DevMesh& m, const double* g, double* dx, int nc, int* info,
                   int num_sms) {
  const int nf = m.nf, n1 = m.n1, n2 = m.n2;
  const bool f64 = std::is_same<T, double>::value;
  double* r = m.r;                                  // float64 work (nf * 3)
  T* b = f64 ? (T*)m.r : (T*)m.rf;                  // solve vector (nf * 3)
  T* y = f64 ? (T*)m.y1 : (T*)m.y1f;                // forward result on x1 (n1 * 3)
  const T* Z = f64 ? (const T*)m.Z : (const T*)m.Zf;
  k_gather_rhs<T><<<nblk(nf, 256), 256, 0, s>>>(nf, m.perm, g, b);
  count_launch();
  if (n1 > 0) trisolve_fwd<T>(s, m, Z, b, y);
  if (n2 > 0) {
    T* y2 = b + 3 * (size_t)n1;
    double* u = m.u;
    double* z2 = r + 3 * (size_t)n1;                // float64 dx2
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
    if (nc > 0) {
      // The reduced system carries the barrier stiffness (cond ~ kappa b''),
      // so it is factored in float64 in both precisions.
      ProfScope psr(PROF_REDUCED, s);
      reduced_solve<double>(s, m, m.Sinv, nc, u, z2, info, num_sms);
    } else {
      cudaMemcpyAsync(z2, u, sizeof(double) * 3 * (size_t)n2, cudaMemcpyDeviceToDevice, s);
    }
    if (!f64) {
      k_convert<double, T><<<nblk(3 * (int64_t)n2, 256), 256, 0, s>>>(3 * n2, z2, y2);
      count_launch();
    }
  }
  if (n1 > 0) trisolve_bwd<T>(s, m, Z, y, b);
  if (!f64) {
    k_convert<T, double><<<nblk(3 * (int64_t)n1, 256), 256, 0, s>>>(3 * n1, b, r);
    count_launch();
  }
  cudaMemsetAsync(dx, 0, sizeof(double) * 3 * (size_t)m.n, s);
  k_scatter_dx<<<nblk(nf, 256), 256, 0, s>>>(nf, m.perm, r, dx);
  count_launch();
}

}  // namespace

int64_t reduced_workspace_elems(int nc) {
  const int64_t n3 = 3 * (int64_t)nc;
  return (int64_t)nc * nc + n3 * n3 + (n3 + 1) * n3 + 2 * n3 + 16;
}

void set_solver_smem_limits(int max_bytes) {
  cudaFuncSetAttribute(k_fwd_chunk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
  cudaFuncSetAttribute(k_bwd_chunk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
  cudaFuncSetAttribute(k_fwd_chunk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
  cudaFuncSetAttribute(k_bwd_chunk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
}

void global_step(cudaStream_t s, const DevMesh& m, const double* g, double* dx, int nc,
                 int precision, int* info_dev, int num_sms) {
  if (precision == 0) global_step_t<double>(s, m, g, dx, nc, info_dev, num_sms);
  else global_step_t<float>(s, m, g, dx, nc, info_dev, num_sms);
}

}  // namespace fsim
