// Reduced contact system of Sec. 3.2.  The cooperative kernel k_reduced
// (float64, or n_c above the cluster path) runs the phases below in one
// launch; the float32 paths for small n_c (k_small_s/x/n/v, the 4-CTA
// cluster k_clus_v) run the same phases as separate kernels, the first ones
// on a side stream.
//
// Eq. 10-11: Sigma-hat^-1 y2 = u - Sigma^-1 Q^T v with u = Sigma^-1 y2 and,
// in the push-through form (B-check is PSD and usually singular, so it is
// never inverted), v = (I + B S)^-1 B u_c, S = Sigma^-1[c, c] (x) I_3.  With
// S = L L^T (L = L_s (x) I_3) this is v = L^-T (I + L^T B L)^-1 L^T B u_c and
// I + L^T B L is SPD with eigenvalues >= 1, so both factorisations are plain
// Cholesky.  Phases, separated by grid-wide barriers:
//   1 gather S = Sigma^-1[c,c], the block-row lists of B, y = B u_c
//   2 S = L_s L_s^T                         (right-looking, 32-wide panels)
//   3 X = B (L_s (x) I_3)
//   4 N = I + (L_s (x) I_3)^T X, and the extra row t0 = (L_s (x) I_3)^T y
//   5 N = L_N L_N^T; the extra row becomes l = L_N^-1 t0
//   6 v = (L_s (x) I_3)^-T L_N^-T l           (one CTA)
//   7 float32 factors only: refinement, rho = y - v - B (S v) in float64,
//     v += L^-T N^-1 L^T rho.  The error of v reaches the global residual as
//     Q^T rho itself, so the stopping test compares |rho| with |y2| (the
//     Schur right-hand side), not with |y| = |B u_c|, which carries the
//     barrier stiffness and can be many orders larger.  At most
//     kMixedRefineSteps steps: where cond(N) nears 1 / u32 (a pair at
//     ~1e-3 d0 with every vertex of the reduced set in contact) a float32
//     factor gains only 4-10x per step, and 4 steps left |rho| near
//     1e-3 |y2|; the stopping rule ends well-conditioned solves after 1-2.
//   8 z2 = u - (Sigma^-1[:, c] (x) I_3) v
// Pivots use a float32 reciprocal square root refined by two float64 Newton
// steps (float64-accurate, a far shorter dependent chain than sqrt and a
// division on GB300's float64 pipe).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace fsim {

namespace {

constexpr int kRT = 256;   // threads per CTA

template <typename FT>
struct RedArgs {
  int nc, n2, refine;
  const int* nc_dev;    // n_c on the device (set by the contact-marking scan)
  FT* base;             // FT workspace: S, X, N, 1/diag, FT vectors (offsets from n_c)
  double* dtail_end;    // end of the float64 workspace; float64 vectors sit before it
  int* ibase;           // int workspace after the block occupancy: lists, counts
  const int* clist;
  const double* Sinv;   // n2 x n2
  const double* Bc;     // (3nc)^2, row-major
  const int* bocc;      // nc x nc block occupancy
  int* list;            // nc x nc block-row lists
  int* cnt;             // nc
  const double* u;      // n2 * 3
  const FT* y2;         // n2 * 3: right-hand side of the Schur system (u = Sigma^-1 y2)
  double* z2;           // n2 * 3 (out)
  FT* S;                // nc x nc  -> L_s
  FT* X;                // n3 x n3
  FT* N;                // (n3 + 1) x n3 -> L_N and l
  FT* dinv_s;           // nc: 1 / L_s[j][j]
  FT* dinv_n;           // n3
  FT* fv;               // 2 * n3 scratch in FT
  double* y;            // n3: B u_c
  double* v;            // n3
  double* rho;          // n3
  double* w;            // n3
  double* nrm;          // 3: |rho|^2 of a refinement step, unused, |y2|^2
  double* S64;          // one-CTA path: Sigma^-1[c, c] in float64 (n_c x n_c)
  int* info;
  int small_lim;        // n_c handled by the one-CTA path (0: none)
  int active;           // lock-step batches: the frame takes part in the launch
  int one_cta_max;      // largest n_c of the one-CTA path (float32 factors); the
                        // 4-CTA cluster takes n_c up to kClusNc above it
  FT* spk;              // one-CTA path: L_s packed, diagonal blocks inverted
};

// Offsets of the workspace for a given n_c (every kernel of the reduced solve
// derives them from the n_c it reads on the device).
template <typename FT>
__device__ __forceinline__ void red_layout(RedArgs<FT>& a, int nc) {
  const int n3 = 3 * nc;
  // every segment starts on a 16-byte boundary (vector loads)
  constexpr size_t q = 16 / sizeof(FT);
  auto al = [](size_t x) { return (x + q - 1) / q * q; };
  a.nc = nc;
  a.S = a.base;
  a.X = a.S + al((size_t)nc * nc);
  a.N = a.X + al((size_t)n3 * n3);
  a.dinv_s = a.N + al((size_t)(n3 + 1) * n3);
  a.dinv_n = a.dinv_s + al(nc);
  a.fv = a.dinv_n + al(n3);
  a.spk = a.fv + al(2 * (size_t)n3);
  a.y = a.dtail_end - 4 * (size_t)n3 - 8;
  a.v = a.y + n3; a.rho = a.v + n3; a.w = a.rho + n3; a.nrm = a.w + n3;
  a.S64 = a.y - (size_t)nc * nc;
  a.list = a.ibase;
  a.cnt = a.list + (size_t)nc * nc;
}

__device__ __forceinline__ double rsqrt_refined(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double r = (double)rsqrtf((float)d);
  r = r * (1.5 - 0.5 * d * r * r);
  r = r * (1.5 - 0.5 * d * r * r);
  return r;
}
__device__ __forceinline__ float rsqrt_refined(float d) { return rsqrtf(d); }

template <typename FT>
struct Smem {
  FT D[32][33];
  FT Pi[32][33];
  FT Pj[32][33];
  FT dv[32];
};

// CTA-level factorisation of the kb x kb diagonal block at (k0, k0).
template <typename FT>
__device__ void factor_diag(FT* A, int k0, int kb, int ld, FT* dinv, int* info, Smem<FT>& sm) {
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += kRT) {
    const int i = e / kb, j = e % kb;
    sm.D[i][j] = (j <= i) ? A[(size_t)(k0 + i) * ld + k0 + j] : FT(0);
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      FT d = sm.D[j][j];
      if (!(d > FT(0))) { atomicOr(info, 1); d = FT(1); }
      const FT r = rsqrt_refined(d);
      sm.D[j][j] = d * r;
      sm.dv[j] = r;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < kb; i += kRT) sm.D[i][j] *= sm.dv[j];
    __syncthreads();
    const int m = kb - j - 1;
    for (int e = tid; e < m * m; e += kRT) {
      const int i = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= i) sm.D[i][c] -= sm.D[i][j] * sm.D[c][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += kRT) {
    const int i = e / kb, j = e % kb;
    A[(size_t)(k0 + i) * ld + k0 + j] = (j <= i) ? sm.D[i][j] : FT(0);
  }
  for (int j = tid; j < kb; j += kRT) dinv[k0 + j] = sm.dv[j];
  __syncthreads();
}

// Right-looking blocked Cholesky of the leading N x N block of an
// (N + extra) x N row-major matrix (extra rows get A L^-T), by all CTAs.
template <typename FT>
__device__ void coop_chol(cg::grid_group& grid, FT* A, int N, int extra, int ld, FT* dinv,
                          int* info, Smem<FT>& sm) {
  const int M = N + extra;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (blockIdx.x == 0 && N > 0) factor_diag(A, 0, min(32, N), ld, dinv, info, sm);
  grid.sync();
  for (int k0 = 0; k0 < N; k0 += 32) {
    const int kb = min(32, N - k0);
    const int k1 = k0 + kb;
    for (int e = tid; e < kb * kb; e += kRT) {
      const int i = e / kb, j = e % kb;
      sm.D[i][j] = A[(size_t)(k0 + i) * ld + k0 + j];
    }
    for (int j = tid; j < kb; j += kRT) sm.dv[j] = dinv[k0 + j];
    __syncthreads();
    // panel: rows [k1, M) := A L_kk^-T, one warp per row (forward substitution)
    for (int r = blockIdx.x * (kRT / 32) + wid; r < M - k1; r += gridDim.x * (kRT / 32)) {
      FT* arow = A + (size_t)(k1 + r) * ld + k0;
      FT xv = (lane < kb) ? arow[lane] : FT(0);
      for (int j = 0; j < kb; ++j) {
        const FT xj = __shfl_sync(0xffffffffu, xv, j) * sm.dv[j];
        if (lane == j) xv = xj;
        if (lane > j && lane < kb) xv -= xj * sm.D[lane][j];
      }
      if (lane < kb) arow[lane] = xv;
    }
    grid.sync();
    if (k1 < N) {
      const int nrb = (M - k1 + 31) / 32, ncb = (N - k1 + 31) / 32;
      int ntiles = 0;
      for (int rb = 0; rb < nrb; ++rb) ntiles += min(rb + 1, ncb);
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int rb = 0, rem = tile;
        while (rem >= min(rb + 1, ncb)) { rem -= min(rb + 1, ncb); ++rb; }
        const int cb = rem;
        const int r0 = k1 + rb * 32, c0 = k1 + cb * 32;
        const int rn = min(32, M - r0), cn = min(32, N - c0);
        for (int e = tid; e < 32 * kb; e += kRT) {
          const int i = e / kb, l = e % kb;
          sm.Pi[i][l] = (i < rn) ? A[(size_t)(r0 + i) * ld + k0 + l] : FT(0);
          sm.Pj[i][l] = (i < cn) ? A[(size_t)(c0 + i) * ld + k0 + l] : FT(0);
        }
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += kRT) {
          const int i = e >> 5, j = e & 31;
          if (i < rn && j < cn && (r0 + i >= c0 + j || r0 + i >= N)) {
            FT acc = 0;
            for (int l = 0; l < kb; ++l) acc += sm.Pi[i][l] * sm.Pj[j][l];
            A[(size_t)(r0 + i) * ld + c0 + j] -= acc;
          }
        }
        __syncthreads();
        if (tile == 0) factor_diag(A, k1, min(32, N - k1), ld, dinv, info, sm);   // look-ahead
      }
    }
    grid.sync();
  }
}

// One CTA: solve L x = b (lower) or L^T x = b in place for n unknowns and
// nrhs right-hand sides (b[i * nrhs + r]); dinv holds 1 / L[j][j].
template <typename FT, bool TRANS>
__device__ void cta_trsv(const FT* L, const FT* dinv, int n, int ld, FT* b, int nrhs, Smem<FT>& sm) {
  const int tid = threadIdx.x;
  const int nblk = (n + 31) / 32;
  for (int bi = 0; bi < nblk; ++bi) {
    const int blk = TRANS ? nblk - 1 - bi : bi;
    const int i0 = blk * 32, nb = min(32, n - i0);
    // stage the diagonal block and 1/diag in shared memory: the sequential
    // substitution below then never waits on global memory
    for (int e = tid; e < nb * nb; e += kRT) {
      const int i = e / nb, j = e % nb;
      sm.D[i][j] = (j <= i) ? L[(size_t)(i0 + i) * ld + i0 + j] : FT(0);
    }
    for (int j = tid; j < nb; j += kRT) sm.dv[j] = dinv[i0 + j];
    __syncthreads();
    if (tid < 32) {
      for (int r = 0; r < nrhs; ++r) {
        FT xv = (tid < nb) ? b[(size_t)(i0 + tid) * nrhs + r] : FT(0);
        for (int s = 0; s < nb; ++s) {
          const int j = TRANS ? nb - 1 - s : s;
          const FT xj = __shfl_sync(0xffffffffu, xv, j) * sm.dv[j];
          if (tid == j) xv = xj;
          if (TRANS) {
            if (tid < j) xv -= sm.D[j][tid] * xj;
          } else {
            if (tid > j && tid < nb) xv -= sm.D[tid][j] * xj;
          }
        }
        if (tid < nb) { b[(size_t)(i0 + tid) * nrhs + r] = xv; sm.Pi[tid][r] = xv; }
      }
    }
    __syncthreads();
    if (TRANS) {   // rows above: b[i] -= sum_j L[i0+j][i] x[j]
      for (int e = tid; e < i0 * nrhs; e += kRT) {
        const int i = e / nrhs, r = e % nrhs;
        FT acc = 0;
        for (int j = 0; j < nb; ++j) acc += L[(size_t)(i0 + j) * ld + i] * sm.Pi[j][r];
        b[(size_t)i * nrhs + r] -= acc;
      }
    } else {       // rows below: b[i] -= sum_j L[i][i0+j] x[j]
      const int below = n - (i0 + nb);
      for (int e = tid; e < below * nrhs; e += kRT) {
        const int i = i0 + nb + e / nrhs, r = e % nrhs;
        FT acc = 0;
        for (int j = 0; j < nb; ++j) acc += L[(size_t)i * ld + i0 + j] * sm.Pi[j][r];
        b[(size_t)i * nrhs + r] -= acc;
      }
    }
    __syncthreads();
  }
}

// q = (L_s (x) I_3)^T p for vectors laid out q[(i, a)] = q[3 i + a] (one CTA)
template <typename FT, typename VT>
__device__ void cta_lt_apply(const FT* L, int nc, const VT* p, FT* q) {
  for (int e = threadIdx.x; e < 3 * nc; e += kRT) {
    const int i = e / 3, a = e % 3;
    double acc = 0.0;
    for (int j = i; j < nc; ++j) acc += (double)L[(size_t)j * nc + i] * (double)p[3 * j + a];
    q[e] = (FT)acc;
  }
}

// z2 = u - (Sigma^-1[:, c] (x) I_3) v, one warp per row (warp w of nw): the
// form for a single frame, which has few rows to spread over the GPU
template <typename FT>
__device__ void z2_update(const RedArgs<FT>& a, int nc, int w, int nw) {
  const int lane = threadIdx.x & 31;
  for (int q = w; q < a.n2; q += nw) {
    const double* srow = a.Sinv + (size_t)q * a.n2;
    double a0 = 0, a1 = 0, a2 = 0;
    for (int m = lane; m < nc; m += 32) {
      if (!FSIM_CHECK_IDX(a.clist[m], a.n2, CHECK_CLIST)) continue;
      const double sv = srow[a.clist[m]];
      a0 += sv * a.v[3 * m]; a1 += sv * a.v[3 * m + 1]; a2 += sv * a.v[3 * m + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
      a.z2[3 * q] = a.u[3 * q] - a0;
      a.z2[3 * q + 1] = a.u[3 * q + 1] - a1;
      a.z2[3 * q + 2] = a.u[3 * q + 2] - a2;
    }
  }
}

// The same with one row per lane (warp w of nw takes rows 32 w .. 32 w + 31,
// then strides by 32 nw): the form for batches, whose frames together give
// enough warps.  Sigma^-1 is stored exactly symmetric (both triangles from
// one product), so row q's entries at the contact columns are read as
// Sigma^-1[c_m][q]: consecutive lanes read consecutive addresses and no
// cross-lane reduction is needed (each float64 warp instruction costs about
// 64 cycles of its SM sub-partition on GB300, so this halves the cost)
template <typename FT>
__device__ void z2_update_rows(const RedArgs<FT>& a, int nc, int w, int nw) {
  const int lane = threadIdx.x & 31;
  for (int q0 = 32 * w; q0 < a.n2; q0 += 32 * nw) {
    const int q = q0 + lane;
    if (q >= a.n2) continue;
    double a0 = 0, a1 = 0, a2 = 0;
    for (int m = 0; m < nc; ++m) {
      const int c = a.clist[m];
      if (!FSIM_CHECK_IDX(c, a.n2, CHECK_CLIST)) continue;
      const double sv = a.Sinv[(size_t)c * a.n2 + q];
      a0 += sv * a.v[3 * m]; a1 += sv * a.v[3 * m + 1]; a2 += sv * a.v[3 * m + 2];
    }
    a.z2[3 * q] = a.u[3 * q] - a0;
    a.z2[3 * q + 1] = a.u[3 * q + 1] - a1;
    a.z2[3 * q + 2] = a.u[3 * q + 2] - a2;
  }
}

// The z2 update alone (plain launch) after the one-CTA or cluster path; with
// n_c = 0 it copies z2 = u.
__device__ __forceinline__ void k_z2_update_body(RedArgs<float> a, bool rows) {
  const int nc = *a.nc_dev;
  if (nc == 0) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * a.n2; e += gridDim.x * blockDim.x)
      a.z2[e] = a.u[e];
    return;
  }
  if (nc > a.small_lim) return;         // the cooperative kernel owns larger n_c
  red_layout(a, nc);
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  if (rows) z2_update_rows(a, nc, w, nw);
  else z2_update(a, nc, w, nw);
}
__global__ void __launch_bounds__(256) k_z2_update(RedArgs<float> a) {
  k_z2_update_body(a, false);
}

template <typename FT>
__global__ void __launch_bounds__(kRT) k_reduced(RedArgs<FT> a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ Smem<FT> sm;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int gtid = blockIdx.x * kRT + tid, gsz = gridDim.x * kRT;
  const int gwarp = blockIdx.x * (kRT / 32) + wid, nwarps = gridDim.x * (kRT / 32);
  // n_c is read on the device, so the launch (and a captured graph) does not
  // depend on it; every thread reads the same value
  const int nc = *a.nc_dev, n3 = 3 * nc;
  if (nc == 0) {          // no contact: Sigma-hat = Sigma, z2 = u
    for (int e = gtid; e < 3 * a.n2; e += gsz) a.z2[e] = a.u[e];
    return;
  }
  red_layout(a, nc);
  if (nc > a.small_lim) {   // otherwise phases 1-7 ran in the one-CTA path
    // 1. S, block lists, y = B u_c
    if (gtid == 0) a.nrm[2] = 0.0;
    for (int e = gtid; e < nc * nc; e += gsz) {
      const int i = e / nc, j = e % nc;
      a.S[e] = (FT)a.Sinv[(size_t)a.clist[i] * a.n2 + a.clist[j]];
    }
    for (int i = gwarp; i < nc; i += nwarps) {
      int base = 0;
      for (int j0 = 0; j0 < nc; j0 += 32) {
        const int j = j0 + lane;
        const bool f = j < nc && a.bocc[(size_t)i * nc + j] != 0;
        const unsigned msk = __ballot_sync(0xffffffffu, f);
        if (f) a.list[(size_t)i * nc + base + __popc(msk & ((1u << lane) - 1u))] = j;
        base += __popc(msk);
      }
      if (lane == 0) a.cnt[i] = base;
    }
    grid.sync();
    for (int row = gtid; row < n3; row += gsz) {
      const int i = row / 3;
      const double* brow = a.Bc + (size_t)row * n3;
      double acc = 0.0;
      for (int e = 0; e < a.cnt[i]; ++e) {
        const int j = a.list[(size_t)i * nc + e];
        const double* uj = a.u + 3 * (size_t)a.clist[j];
        acc += brow[3 * j] * uj[0] + brow[3 * j + 1] * uj[1] + brow[3 * j + 2] * uj[2];
      }
      a.y[row] = acc;
    }
    if (a.refine > 0) {
      double q = 0.0;
      for (int e = gtid; e < 3 * a.n2; e += gsz) q += (double)a.y2[e] * (double)a.y2[e];
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if (lane == 0 && q != 0.0) atomicAdd(&a.nrm[2], q);
    }
    // 2. L_s
    coop_chol<FT>(grid, a.S, nc, 0, nc, a.dinv_s, a.info, sm);
    // 3. X[(i,a),(k,b)] = sum_{j in row i, j >= k} B[(i,a),(j,b)] L_s[j][k]
    for (int64_t e = gtid; e < (int64_t)n3 * n3; e += gsz) {
      const int row = (int)(e / n3), colx = (int)(e % n3);
      const int i = row / 3, k = colx / 3, b = colx % 3;
      const double* brow = a.Bc + (size_t)row * n3;
      double acc = 0.0;
      for (int q = 0; q < a.cnt[i]; ++q) {
        const int j = a.list[(size_t)i * nc + q];
        if (j >= k) acc += brow[3 * j + b] * (double)a.S[(size_t)j * nc + k];
      }
      a.X[e] = (FT)acc;
    }
    grid.sync();
    // 4. N = I + (L_s (x) I)^T X (lower part suffices) and t0
    for (int64_t e = gtid; e < (int64_t)(n3 + 1) * n3; e += gsz) {
      const int row = (int)(e / n3), col = (int)(e % n3);
      double acc;
      if (row < n3) {
        if (col > row) continue;
        const int i = row / 3, ax = row % 3;
        acc = (row == col) ? 1.0 : 0.0;
        for (int j = i; j < nc; ++j)
          acc += (double)a.S[(size_t)j * nc + i] * (double)a.X[(size_t)(3 * j + ax) * n3 + col];
      } else {
        const int i = col / 3, ax = col % 3;
        acc = 0.0;
        for (int j = i; j < nc; ++j) acc += (double)a.S[(size_t)j * nc + i] * a.y[3 * j + ax];
      }
      a.N[e] = (FT)acc;
    }
    grid.sync();
    // 5. L_N (the extra row becomes l = L_N^-1 t0)
    coop_chol<FT>(grid, a.N, n3, 1, n3, a.dinv_n, a.info, sm);
    // 6. v = (L_s (x) I)^-T L_N^-T l
    FT* t = a.fv;
    if (blockIdx.x == 0) {
      for (int e = tid; e < n3; e += kRT) t[e] = a.N[(size_t)n3 * n3 + e];
      __syncthreads();
      cta_trsv<FT, true>(a.N, a.dinv_n, n3, n3, t, 1, sm);
      cta_trsv<FT, true>(a.S, a.dinv_s, nc, nc, t, 3, sm);
      for (int e = tid; e < n3; e += kRT) a.v[e] = (double)t[e];
    }
    grid.sync();
    // 7. refinement with float64 residuals (float32 factors), until
    //    |rho| <= 1e-7 |y2|, until a step fails to halve |rho|, or after
    //    a.refine steps
    double prev = -1.0;
    for (int it = 0; it < a.refine; ++it) {
      if (gtid == 0) a.nrm[0] = 0.0;
      grid.sync();
      // w = S v with S = Sigma^-1[c, c] (x) I_3 in float64
      for (int e = gtid; e < n3; e += gsz) {
        const int i = e / 3, ax = e % 3;
        const double* srow = a.Sinv + (size_t)a.clist[i] * a.n2;
        double acc = 0.0;
        for (int j = 0; j < nc; ++j) acc += srow[a.clist[j]] * a.v[3 * j + ax];
        a.w[e] = acc;
      }
      grid.sync();
      for (int row = gtid; row < n3; row += gsz) {
        const int i = row / 3;
        const double* brow = a.Bc + (size_t)row * n3;
        double acc = 0.0;
        for (int e = 0; e < a.cnt[i]; ++e) {
          const int j = a.list[(size_t)i * nc + e];
          acc += brow[3 * j] * a.w[3 * j] + brow[3 * j + 1] * a.w[3 * j + 1] +
                 brow[3 * j + 2] * a.w[3 * j + 2];
        }
        const double rr = a.y[row] - a.v[row] - acc;
        a.rho[row] = rr;
        atomicAdd(&a.nrm[0], rr * rr);
      }
      grid.sync();
      {   // the same values for every thread of the grid: a uniform decision
        const double r2 = __ldcg(a.nrm), ys = __ldcg(a.nrm + 2);
        if (!(r2 > 1e-14 * ys)) break;
        if (prev >= 0.0 && !(r2 < 0.25 * prev)) break;
        prev = r2;
      }
      if (blockIdx.x == 0) {
        cta_lt_apply<FT, double>(a.S, nc, a.rho, t);
        __syncthreads();
        cta_trsv<FT, false>(a.N, a.dinv_n, n3, n3, t, 1, sm);
        cta_trsv<FT, true>(a.N, a.dinv_n, n3, n3, t, 1, sm);
        cta_trsv<FT, true>(a.S, a.dinv_s, nc, nc, t, 3, sm);
        for (int e = tid; e < n3; e += kRT) a.v[e] += (double)t[e];
      }
      grid.sync();
    }
  }
  // 8. z2 = u - (Sigma^-1[:, c] (x) I_3) v
  z2_update(a, nc, gwarp, nwarps);
}

// ---------------------------------------------------------------------------
// One-CTA path for small n_c (float32 factors): the two factorisations and
// all triangular solves run inside one CTA with the matrix in shared memory,
// so no grid-wide barrier is needed; only the data-parallel products run
// over the grid.  Launch sequence (all read n_c on the device and return
// when 0 < n_c <= kSmallNc does not hold):
//   k_small_s   (1 CTA)  S = Sigma^-1[c,c], L_s, block lists of B
//   k_small_x   (grid)   y = B u_c (float64), |y2|^2, X = B (L_s (x) I_3)
//   k_small_n   (grid)   N = I + (L_s (x) I_3)^T X  (lower part)
//   k_small_v   (1 CTA)  L_N, v = L^-T N^-1 L^T y and its float64 refinement
// then the cooperative kernel runs only its z2 update.
// ---------------------------------------------------------------------------
constexpr int kSmallNc = 96;               // 3 n_c <= 288 fits in one CTA's shared memory
constexpr int kSmallN3 = 3 * kSmallNc;
constexpr int kClusNc = 128;               // 3 n_c <= 384 fits in a 4-CTA cluster
constexpr int kClusN3 = 3 * kClusNc;
constexpr int kCl = 4;                     // CTAs per cluster
constexpr int kST = 512;                   // threads of the one-CTA kernels
constexpr int kSW = kST / 32;

// Padded packed lower storage: row i holds columns 0..i, padded to a
// multiple of 4 floats, so 32-column segments of a row are 16-byte aligned.
__host__ __device__ constexpr int prow(int i) {
  const int q = i >> 2;
  return 8 * q * (q + 1) + (i - 4 * q) * 4 * (q + 1);
}
constexpr int kPtLd = kSmallN3;            // panel scratch: 32 x kPtLd floats

// Outer-product elimination of the unscaled 32 x 32 diagonal block Ds: after
// step j, Ds[i][c] (c > j) holds the Schur complement; Ds[.][j] (j < i) stays
// the unscaled column and Ds[j][j] the pivot.  Thread (r0, c) = (tid / 32,
// tid % 32) owns rows r0 and r0 + 16 of column c; needs 512 threads.  The
// pivot reciprocal is the hardware approximation (within 2 ulp for pivots
// in [2^-126, 2^126]; those of N = I + L^T B L are >= 1, those of
// S = Sigma^-1[c, c] are positive and far from either end): the IEEE
// division sat on the dependent chain of every step, and these float32
// factors are refined in float64 (N) or feed only the float32 products and
// solves of the reduced system (S).  Two columns per barrier measured no
// faster.
__device__ __forceinline__ void eliminate_diag(float (*Ds)[33], int kb) {
  const int tid = threadIdx.x, r0 = tid >> 5, c = tid & 31;
  for (int j = 0; j < kb; ++j) {
    const float inv = __fdividef(1.f, Ds[j][j]);
    if (c > j) {
      const float lcj = Ds[c][j] * inv;
      if (r0 >= c) Ds[r0][c] -= Ds[r0][j] * lcj;
      if (r0 + 16 >= c) Ds[r0 + 16][c] -= Ds[r0 + 16][j] * lcj;
    }
    __syncthreads();
  }
}

// Blocked right-looking Cholesky of the packed n x n matrix A in shared
// memory by one CTA (kST threads); 32-wide panels.  Per panel: the diagonal
// block is factored in shared memory by all threads (outer-product form, one
// barrier per column), every row below solves its own panel segment by
// substitution (one thread per row) while the last warp inverts the
// diagonal block, and the trailing update A -= P P^T runs with 4 x 4
// register tiles from a transposed copy Pt of the panel.  With inv_diag
// the diagonal blocks are left holding L_kk^-1 (for the solves below);
// Lout (row-major, leading dimension ldo), if given, receives the plain
// diagonal blocks.  Loops stay rolled: straight-line code this size would
// run out of the instruction cache.
__device__ void cta_chol_packed(float* A, int n, float* Pt, int* info, bool inv_diag, float* Lout,
                                int ldo, float* DIout) {
  __shared__ float Ds[32][33];
  __shared__ float Li[32][33];
  __shared__ float dv[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int kb = min(32, n - k0), k1 = k0 + kb, m = n - k1;
    for (int e = tid; e < 32 * 32; e += kST) {
      const int i = e >> 5, j = e & 31;
      Ds[i][j] = (i < kb && j <= i) ? A[prow(k0 + i) + k0 + j] : 0.f;
    }
    __syncthreads();
    // outer-product elimination on the unscaled block; Ds[.][j] is scaled below
    eliminate_diag(Ds, kb);
    if (tid < kb) {
      float d = Ds[tid][tid];
      if (!(d > 0.f)) {
        atomicOr(info, 1);
        d = 1.f;
        Ds[tid][tid] = 1.f;
      }
      float rs = rsqrtf(d);
      rs = rs * (1.5f - 0.5f * d * rs * rs);
      dv[tid] = rs;
    } else if (tid < 32) {
      dv[tid] = 1.f;        // padding of a last, narrower block
    }
    __syncthreads();
    for (int e = tid; e < kb * 32; e += kST) {
      const int i = e >> 5, j = e & 31;
      if (j < i) Ds[i][j] *= dv[j];
    }
    __syncthreads();
    if (tid < kb) Ds[tid][tid] = Ds[tid][tid] * dv[tid];    // sqrt(d)
    __syncthreads();
    if (Lout) {
      for (int e = tid; e < kb * 32; e += kST) {
        const int i = e >> 5, j = e & 31;
        if (j <= i) Lout[(size_t)(k0 + i) * ldo + k0 + j] = Ds[i][j];
      }
    }
    if (tid < m) {
      // row k1 + tid: x L_kk^T = a in registers (right-looking, so the
      // dependent chain is one FMA per column), then its transposed copy
      float* row = A + prow(k1 + tid) + k0;
      float x[32];
#pragma unroll
      for (int l = 0; l < 32; ++l) x[l] = row[l];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        x[q] *= dv[q];
#pragma unroll
        for (int l = q + 1; l < 32; ++l) x[l] -= x[q] * Ds[l][q];
      }
#pragma unroll
      for (int l = 0; l < 32; ++l) {
        row[l] = x[l];
        Pt[l * kPtLd + tid] = x[l];
      }
    } else if (wid == kSW - 1) {
      // Li = L_kk^-1, column `lane` in registers (right-looking)
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        x[i] *= dv[i];
#pragma unroll
        for (int l = i + 1; l < 32; ++l) x[l] -= Ds[l][i] * x[i];
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) Li[i][lane] = (i >= lane) ? x[i] : 0.f;
    }
    __syncthreads();
    if (m > 0) {
      // trailing update A -= P P^T, 4 x 4 tiles of the lower triangle
      const int mb = (m + 3) >> 2, nt = mb * (mb + 1) / 2;
      for (int t = tid; t < nt; t += kST) {
        int I = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
        while ((I + 1) * (I + 2) / 2 <= t) ++I;
        while (I * (I + 1) / 2 > t) --I;
        const int J = t - I * (I + 1) / 2;
        float acc[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
          const float4 av = *reinterpret_cast<const float4*>(Pt + l * kPtLd + 4 * I);
          const float4 bv = *reinterpret_cast<const float4*>(Pt + l * kPtLd + 4 * J);
          const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] += ar[p] * br[q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int i = 4 * I + p;
          if (i >= m) break;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int jj = 4 * J + q;
            if (jj <= i) A[prow(k1 + i) + k1 + jj] -= acc[p][q];
          }
        }
      }
    }
    // the diagonal block: plain factor, or its inverse for the solves
    for (int e = tid; e < kb * 32; e += kST) {
      const int i = e >> 5, j = e & 31;
      if (j <= i) A[prow(k0 + i) + k0 + j] = inv_diag ? Li[i][j] : Ds[i][j];
      if (DIout) DIout[(size_t)(k0 >> 5) * 1024 + e] = (j <= i) ? Li[i][j] : 0.f;
    }
    __syncthreads();
  }
}

// Solve L x = t (TRANS = false) or L^T x = t (TRANS = true) in place for a
// packed factor, with nr interleaved right-hand sides t[i * nr + r].  The
// inverted diagonal blocks come from DI (32 x 32 row-major per block) or,
// when DI is null, from the diagonal blocks of A itself (cta_chol_packed
// with inv_diag).  The 32-term dot products are unrolled so that their
// shared-memory loads overlap.
template <bool TRANS>
__device__ void cta_trsv_packed(const float* A, const float* DI, int n, float* t, int nr) {
  __shared__ float xb[32 * 3];
  __shared__ int rp[32];
  const int tid = threadIdx.x;
  const int nblk = (n + 31) / 32;
  for (int bi = 0; bi < nblk; ++bi) {
    const int blk = TRANS ? nblk - 1 - bi : bi;
    const int k0 = blk * 32, kb = min(32, n - k0), k1 = k0 + kb;
    if (tid < 32) rp[tid] = prow(k0 + tid);
    // x_k = Linv_kk t_k (or Linv_kk^T t_k): one thread per (row, rhs)
    if (tid < kb * nr) {
      const int i = tid / nr, r = tid % nr;
      float acc = 0.f;
#pragma unroll
      for (int l = 0; l < 32; ++l) {
        if (l < kb && (TRANS ? l >= i : l <= i)) {
          const int rr = TRANS ? l : i, cc = TRANS ? i : l;
          const float d = DI ? DI[(size_t)blk * 1024 + rr * 32 + cc] : A[prow(k0 + rr) + k0 + cc];
          acc += d * t[(k0 + l) * nr + r];
        }
      }
      xb[i * nr + r] = acc;
    }
    __syncthreads();
    if (tid < kb * nr) t[k0 * nr + tid] = xb[tid];
    if (TRANS) {      // rows above: t[j] -= sum_l L[k0 + l][j] x_l
      for (int e = tid; e < k0 * nr; e += kST) {
        const int j = e / nr, r = e % nr;
        float acc = 0.f;
#pragma unroll
        for (int l = 0; l < 32; ++l)
          if (l < kb) acc += A[rp[l] + j] * xb[l * nr + r];
        t[e] -= acc;
      }
    } else {          // rows below: t[i] -= sum_l L[i][k0 + l] x_l (kb = 32 here)
      for (int e = tid; e < (n - k1) * nr; e += kST) {
        const int i = k1 + e / nr, r = e % nr;
        const float4* arow = reinterpret_cast<const float4*>(A + prow(i) + k0);
        float acc = 0.f;
#pragma unroll
        for (int l4 = 0; l4 < 8; ++l4) {
          const float4 v = arow[l4];
          acc += v.x * xb[(4 * l4) * nr + r] + v.y * xb[(4 * l4 + 1) * nr + r] +
                 v.z * xb[(4 * l4 + 2) * nr + r] + v.w * xb[(4 * l4 + 3) * nr + r];
        }
        t[k1 * nr + e] -= acc;
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  // red holds kSW + 1 doubles; warp 0 adds the warp sums (float64 adds are
  // slow on GB300: one shuffle tree, not a loop in every thread)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < kSW ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[kSW] = t;
  }
  __syncthreads();
  return red[kSW];
}

// k_small_s: S = Sigma^-1[c, c], its factor (plain, row-major into a.S for
// the products; packed with inverted diagonal blocks into a.spk for the
// solves) and the block-row lists of B.
__device__ __forceinline__ void k_small_s_body(RedArgs<float> a) {
  extern __shared__ float smem_f[];
  const int nc = *a.nc_dev;
  if (nc == 0 || nc > a.small_lim) return;
  red_layout(a, nc);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* P = smem_f;                      // prow(kClusNc) floats
  float* Pt = P + prow(kClusNc);          // 32 x kPtLd
  if (tid == 0) a.nrm[2] = 0.0;
  for (int i = wid; i < nc; i += kSW) {
    if (!FSIM_CHECK_IDX(a.clist[i], a.n2, CHECK_CLIST)) continue;
    const double* srow = a.Sinv + (size_t)a.clist[i] * a.n2;
#pragma unroll 4
    for (int j = lane; j < nc; j += 32) {
      if (!FSIM_CHECK_IDX(a.clist[j], a.n2, CHECK_CLIST)) continue;
      const double sv = srow[a.clist[j]];
      a.S64[(size_t)i * nc + j] = sv;
      if (j <= i) P[prow(i) + j] = (float)sv;
    }
  }
  for (int i = wid; i < nc; i += kSW) {
    bool f[kClusNc / 32];                 // all occupancy flags of the row first
#pragma unroll
    for (int q = 0; q < kClusNc / 32; ++q) {
      const int j = 32 * q + lane;
      f[q] = j < nc && a.bocc[(size_t)i * nc + j] != 0;
    }
    int base = 0;
#pragma unroll
    for (int q = 0; q < kClusNc / 32; ++q) {
      const unsigned msk = __ballot_sync(0xffffffffu, f[q]);
      if (f[q]) a.list[(size_t)i * nc + base + __popc(msk & ((1u << lane) - 1u))] = 32 * q + lane;
      base += __popc(msk);
    }
    if (lane == 0) a.cnt[i] = base;
  }
  __syncthreads();
  // L_s: row-major into a.S (for the grid products), packed plain into
  // a.spk followed by its inverted diagonal blocks (for the one-CTA solves)
  cta_chol_packed(P, nc, Pt, a.info, false, nullptr, 0, a.spk + prow(nc));
  for (int e = tid; e < nc * nc; e += kST) {
    const int i = e / nc, j = e % nc;
    a.S[e] = (j <= i) ? P[prow(i) + j] : 0.f;
  }
  for (int e = tid; e < prow(nc); e += kST) a.spk[e] = P[e];
}
__global__ void __launch_bounds__(kST) k_small_s(RedArgs<float> a) {
  k_small_s_body(a);
}

// k_small_x (grid): y = B u_c in float64, |y2|^2 (PARTS & 1: these need the
// right-hand side), X = B (L_s (x) I_3) (PARTS & 2: needs only B and L_s).
constexpr int kXRows = 4;                  // rows of X per staged block
template <int PARTS>
__device__ __forceinline__ void k_small_x_body(RedArgs<float> a) {
  const int nc = *a.nc_dev;
  if (nc == 0 || nc > a.small_lim) return;
  red_layout(a, nc);
  const int n3 = 3 * nc;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  if (PARTS & 1)
  for (int row = gtid; row < n3; row += gsz) {
    const int i = row / 3;
    const double* brow = a.Bc + (size_t)row * n3;
    double acc = 0.0;
    const int ci = a.cnt[i];
#pragma unroll 4
    for (int e = 0; e < ci; ++e) {
      const int j = a.list[(size_t)i * nc + e];
      const double* uj = a.u + 3 * (size_t)a.clist[j];
      acc += brow[3 * j] * uj[0] + brow[3 * j + 1] * uj[1] + brow[3 * j + 2] * uj[2];
    }
    a.y[row] = acc;
  }
  if (PARTS & 1) {
    double q = 0.0;
    for (int e = gtid; e < 3 * a.n2; e += gsz) q += (double)a.y2[e] * (double)a.y2[e];
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0 && q != 0.0) atomicAdd(&a.nrm[2], q);
  }
  if (PARTS & 2) {
    // X by blocks of kXRows rows: the block's rows of B-check are converted
    // to float32 once into shared memory (a float64 conversion costs a
    // float64-pipe issue on GB300), then every thread forms entries of the
    // block from them
    __shared__ float bs[kXRows][3 * kClusNc];
    const int nblk = (n3 + kXRows - 1) / kXRows;
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
      const int r0 = rb * kXRows;
      __syncthreads();
      for (int e = threadIdx.x; e < kXRows * n3; e += blockDim.x) {
        const int rr = e / n3, c = e - rr * n3, row = r0 + rr;
        bs[rr][c] = row < n3 ? (float)a.Bc[(size_t)row * n3 + c] : 0.f;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kXRows * n3; e += blockDim.x) {
        const int rr = e / n3, colx = e - rr * n3, row = r0 + rr;
        if (row >= n3) continue;
        const int i = row / 3, k = colx / 3, b = colx % 3;
        float acc = 0.f;
        const int ci = a.cnt[i];
#pragma unroll 4
        for (int q = 0; q < ci; ++q) {
          const int j = a.list[(size_t)i * nc + q];
          if (j >= k) acc += bs[rr][3 * j + b] * a.S[(size_t)j * nc + k];
        }
        a.X[(size_t)row * n3 + colx] = acc;
      }
    }
  }
}
template <int PARTS>
__global__ void __launch_bounds__(256) k_small_x(RedArgs<float> a) {
  k_small_x_body<PARTS>(a);
}

// k_small_n (grid): N = I + (L_s (x) I_3)^T X, lower part, packed.
// N = I + (L_s (x) I_3)^T X, lower triangle, by 32 x 32 tiles: CTA `tile`
// takes row tile ti and column tile tj <= ti of the lower triangle (tiles
// beyond 3 n_c exit).  Entry (row = 3 i + ax, col) is 1[row == col] plus the
// sum over j >= i of L_s[j][i] X[3 j + ax][col], accumulated in increasing j.
// X rows 3 j + ax and the tile's L_s entries are staged in shared memory
// kNJ values of j at a time; a thread keeps 4 rows of one column.
constexpr int kNJ = 16;
constexpr int kNTiles = (3 * kClusNc + 31) / 32 * ((3 * kClusNc + 31) / 32 + 1) / 2;
__device__ __forceinline__ void k_small_n_body(RedArgs<float> a, int tile) {
  __shared__ float Xs[3 * kNJ][32];
  __shared__ float Ls[kNJ][12];
  const int nc = *a.nc_dev;
  if (nc == 0 || nc > a.small_lim) return;
  const int n3 = 3 * nc, nt = (n3 + 31) / 32;
  if (tile >= nt * (nt + 1) / 2) return;
  int ti = 0;
  while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
  const int tj = tile - ti * (ti + 1) / 2;
  red_layout(a, nc);
  const int R0 = 32 * ti, C0 = 32 * tj, i0 = R0 / 3;
  const int tid = threadIdx.x, col = tid & 31, rw = tid >> 5;
  int iv[4], ax[4];
  float acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int row = R0 + rw + 8 * q;
    iv[q] = row / 3 - i0;            // 0 .. 11
    ax[q] = row % 3;
    acc[q] = (row == C0 + col) ? 1.f : 0.f;
  }
  for (int j0 = i0; j0 < nc; j0 += kNJ) {
    __syncthreads();
    for (int e = tid; e < 3 * kNJ * 32; e += blockDim.x) {
      const int rr = e >> 5, c = e & 31, xr = 3 * j0 + rr;
      Xs[rr][c] = (xr < n3 && C0 + c < n3) ? a.X[(size_t)xr * n3 + C0 + c] : 0.f;
    }
    for (int e = tid; e < kNJ * 12; e += blockDim.x) {
      const int jj = e / 12, ii = e % 12, j = j0 + jj, i = i0 + ii;
      Ls[jj][ii] = (j < nc && i < nc && j >= i) ? a.S[(size_t)j * nc + i] : 0.f;
    }
    __syncthreads();
    const int jn = min(kNJ, nc - j0);
    for (int jj = 0; jj < jn; ++jj)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += Ls[jj][iv[q]] * Xs[3 * jj + ax[q]][col];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int row = R0 + rw + 8 * q, c = C0 + col;
    if (row < n3 && c <= row) a.N[prow(row) + c] = acc[q];   // packed lower (k_small_v's layout)
  }
}
__global__ void __launch_bounds__(256) k_small_n(RedArgs<float> a) {
  k_small_n_body(a, blockIdx.x);
}

// q = (L_s (x) I_3)^T p (float; L_s packed plain, in shared memory)
// (one warp per entry)
__device__ void cta_lt_apply_f(const float* Lp, int nc, const double* p, float* q) {
  const int lane = threadIdx.x & 31;
  for (int e = threadIdx.x >> 5; e < 3 * nc; e += kSW) {
    const int i = e / 3, ax = e % 3;
    float acc = 0.f;
#pragma unroll 4
    for (int j = i + lane; j < nc; j += 32) acc += Lp[prow(j) + i] * (float)p[3 * j + ax];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) q[e] = acc;
  }
}

// Float64 refinement products.  GB300 issues a warp-wide float64 FMA about
// every 64 cycles per SM sub-partition, so these loops are laid out to keep
// the number of float64 warp instructions small: thread (vertex i, part q)
// of kRP parts accumulates the three rows of vertex i over every kRP-th
// term, the kRP parts (consecutive lanes) are summed by shuffles.  t is the
// thread's index among nt threads taking part (nt a multiple of 32, the
// same loop trip count in every lane).
constexpr int kRP = 4;

// w = S v with S = Sigma^-1[c, c] (x) I_3 (S64 gathered by k_small_s)
__device__ void refine_sv(const RedArgs<float>& a, int nc, int t, int nt) {
  const int total = kRP * nc;
  for (int base = 0; base < total; base += nt) {
    const int item = base + t;
    const bool ok = item < total;
    const int i = ok ? item / kRP : 0, q = item % kRP;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (ok) {
      const double* srow = a.S64 + (size_t)i * nc;
      for (int j = q; j < nc; j += kRP) {
        const double sij = srow[j];
        s0 += sij * a.v[3 * j];
        s1 += sij * a.v[3 * j + 1];
        s2 += sij * a.v[3 * j + 2];
      }
    }
#pragma unroll
    for (int o = kRP / 2; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (ok && q == 0) {
      a.w[3 * i] = s0;
      a.w[3 * i + 1] = s1;
      a.w[3 * i + 2] = s2;
    }
  }
}

// rho = y - v - B w over the block-row lists of B; returns this thread's
// share of |rho|^2
__device__ double refine_rho(const RedArgs<float>& a, int nc, int t, int nt) {
  const int total = kRP * nc, n3 = 3 * nc;
  double r2 = 0.0;
  for (int base = 0; base < total; base += nt) {
    const int item = base + t;
    const bool ok = item < total;
    const int i = ok ? item / kRP : 0, q = item % kRP;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (ok) {
      const double* b0 = a.Bc + (size_t)(3 * i) * n3;
      const double* b1 = b0 + n3;
      const double* b2 = b1 + n3;
      const int* li = a.list + (size_t)i * nc;
      const int ci = a.cnt[i];
      for (int e = q; e < ci; e += kRP) {
        const int j3 = 3 * li[e];
        const double w0 = a.w[j3], w1 = a.w[j3 + 1], w2 = a.w[j3 + 2];
        s0 += b0[j3] * w0 + b0[j3 + 1] * w1 + b0[j3 + 2] * w2;
        s1 += b1[j3] * w0 + b1[j3 + 1] * w1 + b1[j3 + 2] * w2;
        s2 += b2[j3] * w0 + b2[j3 + 1] * w1 + b2[j3 + 2] * w2;
      }
    }
#pragma unroll
    for (int o = kRP / 2; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (ok && q == 0) {
      const double acc[3] = {s0, s1, s2};
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const int row = 3 * i + ax;
        const double rr = a.y[row] - a.v[row] - acc[ax];
        a.rho[row] = rr;
        r2 += rr * rr;
      }
    }
  }
  return r2;
}

// k_small_v (1 CTA): L_N in shared memory, v = (L_s (x) I)^-T N^-1 (L_s (x) I)^T y
// and the float64-residual refinement of v (same stopping rule as the
// cooperative kernel).
__device__ __forceinline__ void k_small_v_body(RedArgs<float> a) {
  extern __shared__ float smem_f[];
  __shared__ double red[kSW + 1];
  const int nc = *a.nc_dev;
  if (nc == 0 || nc > a.one_cta_max) return;
  red_layout(a, nc);
  const int n3 = 3 * nc;
  const int tid = threadIdx.x;
  float* A = smem_f;                      // prow(kSmallN3) floats
  float* Pt = A + prow(kSmallN3);         // 32 x kPtLd
  float* t = Pt + 32 * kPtLd;             // n3
  {   // packed N (padding included: prow(n3) is a multiple of 4)
    const float4* src = reinterpret_cast<const float4*>(a.N);
    float4* dst = reinterpret_cast<float4*>(A);
#pragma unroll 4
    for (int e = tid; e < prow(n3) / 4; e += kST) dst[e] = src[e];
  }
  __syncthreads();
  cta_chol_packed(A, n3, Pt, a.info, true, nullptr, 0, nullptr);
  // L_s (packed plain + inverted diagonal blocks) into the panel scratch
  float* Ls = Pt;
  const float* LsDI = Pt + prow(nc);
  {
    const float4* src = reinterpret_cast<const float4*>(a.spk);
    float4* dst = reinterpret_cast<float4*>(Ls);
    const int n4 = (prow(nc) + 1024 * ((nc + 31) / 32)) / 4;
#pragma unroll 4
    for (int e = tid; e < n4; e += kST) dst[e] = src[e];
  }
  __syncthreads();
  cta_lt_apply_f(Ls, nc, a.y, t);
  __syncthreads();
  cta_trsv_packed<false>(A, nullptr, n3, t, 1);
  cta_trsv_packed<true>(A, nullptr, n3, t, 1);
  cta_trsv_packed<true>(Ls, LsDI, nc, t, 3);
  for (int e = tid; e < n3; e += kST) a.v[e] = (double)t[e];
  __syncthreads();
  double prev = -1.0;
  for (int it = 0; it < a.refine; ++it) {
    // w = S v with S = Sigma^-1[c, c] (x) I_3 in float64 (S gathered by k_small_s)
    refine_sv(a, nc, tid, kST);
    __syncthreads();
    double r2 = refine_rho(a, nc, tid, kST);
    r2 = block_sum_d(r2, red);
    const double ys = __ldcg(a.nrm + 2);
    if (!(r2 > 1e-14 * ys)) break;
    if (prev >= 0.0 && !(r2 < 0.25 * prev)) break;
    prev = r2;
    cta_lt_apply_f(Ls, nc, a.rho, t);
    __syncthreads();
    cta_trsv_packed<false>(A, nullptr, n3, t, 1);
    cta_trsv_packed<true>(A, nullptr, n3, t, 1);
    cta_trsv_packed<true>(Ls, LsDI, nc, t, 3);
    for (int e = tid; e < n3; e += kST) a.v[e] += (double)t[e];
    __syncthreads();
  }
}
__global__ void __launch_bounds__(kST) k_small_v(RedArgs<float> a) {
  k_small_v_body(a);
}

// ---------------------------------------------------------------------------
// k_clus_v: the same solve for kSmallNc < n_c <= kClusNc on a cluster of kCl
// CTAs.  32-row blocks of the packed N are spread block-cyclically over the
// CTAs' shared memory.  Per panel the owner factors its diagonal block and the
// others copy it through distributed shared memory; each CTA solves its own
// rows of the panel and stores them into the panel copy of every CTA
// (distributed shared-memory stores, visible after the cluster barrier that
// follows), then updates only its own rows.  The diagonal blocks are
// inverted after the factorisation, one warp per block.  The triangular
// solves pass 32-value blocks through distributed shared memory with one
// cluster barrier per block, and the float64 residuals of the refinement are
// split over the CTAs.
// ---------------------------------------------------------------------------
constexpr int kClusRowsMax = 32 * ((kClusN3 / 32 + kCl - 1) / kCl);   // own rows per CTA
// largest packed storage of the rows one CTA owns (padded row lengths)
constexpr int clus_aloc() {
  int mx = 0;
  for (int rank = 0; rank < kCl; ++rank) {
    int tot = 0;
    for (int b = rank; b < kClusN3 / 32; b += kCl)
      for (int rr = 0; rr < 32; ++rr) tot += 4 * ((32 * b + rr + 4) / 4);
    mx = tot > mx ? tot : mx;
  }
  return mx + 64;
}
constexpr int kClusALoc = clus_aloc();
static_assert(kClusALoc % 4 == 0, "panel scratch must stay 16-byte aligned");
constexpr size_t kClusSmem =
    sizeof(float) * ((size_t)kClusALoc + 32 * (size_t)kClusN3 + (size_t)prow(kClusNc) +
                     1024 * (kClusNc / 32) + 2 * (size_t)kClusN3);

// (__maxnreg__ rather than __launch_bounds__: with the latter ptxas settles
// on 64 registers and spills; 512 threads x 128 registers fill one SM)
__device__ __forceinline__ void k_clus_v_body(RedArgs<float> a) {
  namespace cgx = cooperative_groups;
  cgx::cluster_group cl = cgx::this_cluster();
  extern __shared__ float smem_f[];
  __shared__ float Ds[32][33];
  __shared__ float dv[32];
  __shared__ float dvown[kClusRowsMax];            // 1 / L_ii of own rows
  __shared__ float Dinv[kClusRowsMax / 32][32][33];  // own diagonal blocks, inverted at the end
  __shared__ float xb[2][32];
  __shared__ float part[2][kCl][32];
  __shared__ double nrm_parts[kCl];
  __shared__ float wsum[kSW][32];
  __shared__ int loff[kClusRowsMax];
  __shared__ double red[kSW + 1];
  const int nc = *a.nc_dev;
  if (nc <= a.one_cta_max || nc > kClusNc) return;  // uniform over the cluster
  red_layout(a, nc);
  const int n3 = 3 * nc, nblk = (n3 + 31) / 32;
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* A = smem_f;                               // own rows, packed
  float* Pt = A + kClusALoc;                       // 32 x kClusN3, panel by global row - k1
  float* Ls = Pt + 32 * kClusN3;                   // L_s packed plain, then inverted blocks
  float* LsDI = Ls + prow(nc);
  float* t = Ls + prow(kClusNc) + 1024 * (kClusNc / 32);   // n3: rhs / solution (own rows valid)
  float* xg = t + kClusN3;                         // n3: gathered solution (rank 0)
  // own rows: block b is owned by b % kCl; local row lb * 32 + (r % 32)
  auto lrow = [&](int r) { return ((r >> 5) / kCl) * 32 + (r & 31); };
  if (tid < kClusRowsMax) {
    int off = 0;
    for (int lr = 0; lr < tid; ++lr) {
      const int r = ((lr >> 5) * kCl + rank) * 32 + (lr & 31);
      off += 4 * ((r + 4) / 4);                    // padded length of row r
    }
    loff[tid] = off;
  }
  __syncthreads();
  auto Ael = [&](int r, int c) -> float& { return A[loff[lrow(r)] + c]; };
  // load own rows of the packed N and L_s.  A packed row r is a 16-byte
  // aligned run of 4 (r / 4 + 1) floats in both layouts (padding included,
  // never read), so rows move as float4: warp w takes own rows w, w + 16, ..
  // two rows and all their loads in flight at once (a row has <= 96 float4)
  static_assert(kClusN3 / 4 <= 96, "a packed row must fit three float4 per lane");
  for (int lr0 = wid; lr0 < kClusRowsMax; lr0 += 2 * kSW) {
    float4 v[2][3];
    int len4[2];
    const float4* src[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int lr = lr0 + h * kSW;
      const int r = 32 * (((lr >> 5) * kCl) + rank) + (lr & 31);
      len4[h] = (lr < kClusRowsMax && r < n3) ? (r >> 2) + 1 : 0;
      src[h] = reinterpret_cast<const float4*>(a.N + prow(r < n3 ? r : 0));
#pragma unroll
      for (int u = 0; u < 3; ++u)
        if (lane + 32 * u < len4[h]) v[h][u] = src[h][lane + 32 * u];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (len4[h] == 0) continue;
      float4* dst = reinterpret_cast<float4*>(A + loff[lr0 + h * kSW]);
#pragma unroll
      for (int u = 0; u < 3; ++u)
        if (lane + 32 * u < len4[h]) dst[lane + 32 * u] = v[h][u];
    }
  }
  {
    const float4* src = reinterpret_cast<const float4*>(a.spk);
    float4* dst = reinterpret_cast<float4*>(Ls);
    const int n4 = (prow(nc) + 1024 * ((nc + 31) / 32)) / 4;
#pragma unroll 4
    for (int e = tid; e < n4; e += kST) dst[e] = src[e];
  }
  __syncthreads();

  // ---- Cholesky of N over the cluster --------------------------------------
  for (int k = 0; k < nblk; ++k) {
    const int k0 = 32 * k, kb = min(32, n3 - k0), k1 = k0 + kb, m = n3 - k1;
    const int owner = k % kCl;
    if (rank == owner) {
      for (int e = tid; e < 32 * 32; e += kST) {
        const int i = e >> 5, j = e & 31;
        Ds[i][j] = (i < kb && j <= i) ? Ael(k0 + i, k0 + j) : 0.f;
      }
      __syncthreads();
      eliminate_diag(Ds, kb);
      if (tid < kb) {
        float d = Ds[tid][tid];
        if (!(d > 0.f)) {
          atomicOr(a.info, 1);
          d = 1.f;
          Ds[tid][tid] = 1.f;
        }
        float rs = rsqrtf(d);
        rs = rs * (1.5f - 0.5f * d * rs * rs);
        dv[tid] = rs;
      } else if (tid < 32) {
        dv[tid] = 1.f;
      }
      __syncthreads();
      for (int e = tid; e < kb * 32; e += kST) {
        const int i = e >> 5, j = e & 31;
        if (j < i) Ds[i][j] *= dv[j];
      }
      __syncthreads();
      if (tid < kb) Ds[tid][tid] = Ds[tid][tid] * dv[tid];
      if (tid < 32) dvown[lrow(k0) + tid] = dv[tid];   // kept for the inverse below
      __syncthreads();
    }
    cl.sync();
    if (rank != owner) {     // the owner's diagonal factor and 1/diag
      const float* rD = cl.map_shared_rank(&Ds[0][0], owner);
      const float* rv = cl.map_shared_rank(&dv[0], owner);
#pragma unroll
      for (int e = tid; e < 32 * 33; e += kST) (&Ds[0][0])[e] = rD[e];
      if (tid < 32) dv[tid] = rv[tid];
    }
    __syncthreads();
    // own panel rows: x L_kk^T = a (registers), into A and into the panel
    // copy of every CTA of the cluster (remote stores, made visible by the
    // cluster barrier below); one warp per own block below the panel
    for (int idx = tid; idx < kClusRowsMax; idx += kST) {
      const int b = ((idx >> 5) * kCl) + rank;
      const int r = 32 * b + (idx & 31);
      if (b > k && r < n3) {
        float* row = &Ael(r, k0);
        float x[32];
#pragma unroll
        for (int l = 0; l < 32; ++l) x[l] = row[l];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          x[q] *= dv[q];
#pragma unroll
          for (int l = q + 1; l < 32; ++l) x[l] -= x[q] * Ds[l][q];
        }
#pragma unroll
        for (int l = 0; l < 32; ++l) row[l] = x[l];
#pragma unroll
        for (int l = 0; l < 32; ++l) Pt[l * kClusN3 + (r - k1)] = x[l];
        for (int q = 1; q < kCl; ++q) {
          float* dst = cl.map_shared_rank(Pt, (rank + q) % kCl);
#pragma unroll
          for (int l = 0; l < 32; ++l) dst[l * kClusN3 + (r - k1)] = x[l];
        }
      }
    }
    // the owner keeps the plain diagonal factor (inverted after the loop)
    if (rank == owner)
      for (int e = tid; e < kb * 32; e += kST) {
        const int i = e >> 5, j = e & 31;
        if (j <= i) Ael(k0 + i, k0 + j) = Ds[i][j];
      }
    cl.sync();
    // trailing update of own rows: A(i, j) -= P_i . P_j, 4 x 4 tiles
    if (m > 0) {
      // only this CTA's 4-row tiles (tile I covers rows k1 + 4I ..; a 32-row
      // block b below the panel holds tiles (32b - k1)/4 + 0..7, each with
      // I + 1 column tiles J <= I), numbered consecutively over the threads
      const int mb = (m + 3) >> 2;
      int bfirst = rank;
      while (bfirst <= k) bfirst += kCl;
      int total = 0;
      for (int b = bfirst; 32 * b < n3; b += kCl) {
        const int I0 = (32 * b - k1) >> 2, ns = min(8, mb - I0);
        total += ns * (I0 + 1) + ns * (ns - 1) / 2;
      }
      for (int u = tid; u < total; u += kST) {
        int rem = u, I = 0, J = 0;
        for (int b = bfirst; 32 * b < n3; b += kCl) {
          const int I0 = (32 * b - k1) >> 2, ns = min(8, mb - I0);
          const int cnt = ns * (I0 + 1) + ns * (ns - 1) / 2;
          if (rem < cnt) {
            int s2 = 0;
            while (rem >= I0 + s2 + 1) { rem -= I0 + s2 + 1; ++s2; }
            I = I0 + s2;
            J = rem;
            break;
          }
          rem -= cnt;
        }
        float acc[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
          const float4 av = *reinterpret_cast<const float4*>(Pt + l * kClusN3 + 4 * I);
          const float4 bv = *reinterpret_cast<const float4*>(Pt + l * kClusN3 + 4 * J);
          const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] += ar[p] * br[q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int i = 4 * I + p;
          if (i >= m) break;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int jj = 4 * J + q;
            if (jj <= i) Ael(k1 + i, k1 + jj) -= acc[p][q];
          }
        }
      }
    }
    __syncthreads();
  }
  // L_kk^-1 of every own diagonal block (for the solves), one warp per
  // block, all blocks at once: column `lane` by substitution in registers
  {
    const int b = rank + kCl * wid;
    if (b < nblk) {
      const int k0 = 32 * b, kb = min(32, n3 - k0), lb = lrow(k0);
      float (*D)[33] = Dinv[wid];
      for (int i = 0; i < 32; ++i)
        D[i][lane] = (i < kb && lane <= i) ? A[loff[lb + i] + k0 + lane] : 0.f;
      __syncwarp();
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        x[i] *= dvown[lb + i];
#pragma unroll
        for (int l = i + 1; l < 32; ++l) x[l] -= D[l][i] * x[i];
      }
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i < kb && i >= lane) A[loff[lb + i] + k0 + lane] = x[i];
    }
  }
  cl.sync();

  // ---- distributed solves with L_N (own rows of t hold the values) ---------
  auto solve_n = [&]() {
    // forward: L x = t
    for (int k = 0; k < nblk; ++k) {
      const int k0 = 32 * k, kb = min(32, n3 - k0), owner = k % kCl, buf = k & 1;
      if (rank == owner) {
        {   // x_k = L_kk^-1 t_k: 16 threads per row, two terms each, shuffle sum
          const int rw = tid >> 4, pp = tid & 15;
          float acc = 0.f;
          if (rw < kb) {
            const float* drow = &Ael(k0 + rw, k0);
            if (pp <= rw) acc += drow[pp] * t[k0 + pp];
            if (pp + 16 <= rw) acc += drow[pp + 16] * t[k0 + pp + 16];
          }
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (pp == 0 && rw < kb) xb[buf][rw] = acc;
        }
        __syncthreads();
        if (tid < kb) {
          t[k0 + tid] = xb[buf][tid];
          for (int q = 0; q < kCl; ++q)
            if (q != rank) cl.map_shared_rank(&xb[buf][0], q)[tid] = xb[buf][tid];
        }
      }
      cl.sync();
      for (int idx = tid; idx < kClusRowsMax; idx += kST) {
        const int b = ((idx >> 5) * kCl) + rank;
        const int r = 32 * b + (idx & 31);
        if (b > k && r < n3) {
          const float* row = &Ael(r, k0);
          float acc = 0.f;
#pragma unroll
          for (int l = 0; l < 32; ++l) acc += row[l] * xb[buf][l];
          t[r] -= acc;
        }
      }
      __syncthreads();
    }
    // backward: L^T x = t
    for (int k = nblk - 1; k >= 0; --k) {
      const int k0 = 32 * k, kb = min(32, n3 - k0), owner = k % kCl, buf = k & 1;
      // partial sums over own rows below block k for its columns: warp w
      // takes own rows w, w + 16, ...; lane = column
      {
        float acc = 0.f;
        if (lane < kb)
          for (int idx = wid; idx < kClusRowsMax; idx += kSW) {
            const int b = ((idx >> 5) * kCl) + rank;
            const int r = 32 * b + (idx & 31);
            if (b > k && r < n3) acc += Ael(r, k0 + lane) * t[r];
          }
        wsum[wid][lane] = acc;
        __syncthreads();
        if (tid < 32) {
          float tot = 0.f;
          for (int w = 0; w < kSW; ++w) tot += wsum[w][tid];
          cl.map_shared_rank(&part[buf][0][0], owner)[rank * 32 + tid] = tot;
        }
      }
      cl.sync();
      if (rank == owner) {
        if (tid < kb) {
          float s = t[k0 + tid];
          for (int q = 0; q < kCl; ++q) s -= part[buf][q][tid];
          xb[buf][tid] = s;
        }
        __syncthreads();
        {   // x_k = L_kk^-T s_k: 16 threads per column, two terms each
          const int col = tid >> 4, pp = tid & 15;
          float acc = 0.f;
          if (col < kb) {
            if (pp >= col && pp < kb) acc += Ael(k0 + pp, k0 + col) * xb[buf][pp];
            if (pp + 16 >= col && pp + 16 < kb)
              acc += Ael(k0 + pp + 16, k0 + col) * xb[buf][pp + 16];
          }
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (pp == 0 && col < kb) t[k0 + col] = acc;
        }
        __syncthreads();
      }
    }
    cl.sync();
  };
  // (L_s (x) I)^-T on the gathered solution (rank 0), result into a.v / added to it
  auto finish = [&](bool add) {
    if (rank == 0) {
      // every row from the CTA that owns it, all remote loads in flight at once
      for (int r = tid; r < n3; r += kST) {
        const int q = (r >> 5) % kCl;
        xg[r] = (q == 0) ? t[r] : cl.map_shared_rank(t, q)[r];
      }
      __syncthreads();
      cta_trsv_packed<true>(Ls, LsDI, nc, xg, 3);
      for (int e = tid; e < n3; e += kST) a.v[e] = (add ? a.v[e] : 0.0) + (double)xg[e];
    }
    cl.sync();
  };
  // t = (L_s (x) I_3)^T p on own rows
  auto lt_own = [&](const double* p) {     // one warp per own row
    for (int idx = wid; idx < kClusRowsMax; idx += kSW) {
      const int r = 32 * (((idx >> 5) * kCl) + rank) + (idx & 31);
      if (r >= n3) continue;
      const int i = r / 3, ax = r % 3;
      float acc = 0.f;
#pragma unroll 4
      for (int j = i + lane; j < nc; j += 32) acc += Ls[prow(j) + i] * (float)p[3 * j + ax];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) t[r] = acc;
    }
    __syncthreads();
  };
  lt_own(a.y);
  solve_n();
  finish(false);

  // ---- float64 refinement, rows split over the cluster ----------------------
  double prev = -1.0;
  // refinement threads numbered warp-interleaved over the cluster's CTAs
  const int gt = (wid * kCl + rank) * 32 + lane;
  for (int it = 0; it < a.refine; ++it) {
    refine_sv(a, nc, gt, kCl * kST);
    cl.sync();
    double r2 = refine_rho(a, nc, gt, kCl * kST);
    r2 = block_sum_d(r2, red);
    if (tid < kCl) cl.map_shared_rank(&nrm_parts[0], tid)[rank] = r2;
    cl.sync();
    double tot = 0.0;
    for (int q = 0; q < kCl; ++q) tot += nrm_parts[q];     // same order everywhere
    const double ys = __ldcg(a.nrm + 2);
    if (!(tot > 1e-14 * ys)) break;
    if (prev >= 0.0 && !(tot < 0.25 * prev)) break;
    prev = tot;
    lt_own(a.rho);
    solve_n();
    finish(true);
  }
}
__global__ void __maxnreg__(128) k_clus_v(RedArgs<float> a) {
  k_clus_v_body(a);
}

constexpr size_t kSmallSmemS = sizeof(float) * ((size_t)prow(kClusNc) + 32 * kPtLd);
constexpr size_t kSmallSmemV = sizeof(float) * ((size_t)prow(kSmallN3) + 32 * kPtLd + kSmallN3);

template <typename FT>
RedArgs<FT> make_args(const DevMesh& m, const double* u, const FT* y2, double* z2, int* info,
                      int refine) {
  RedArgs<FT> a{};
  a.n2 = m.n2; a.refine = refine;
  a.nc_dev = m.counters + 3;
  a.base = std::is_same<FT, double>::value ? (FT*)m.red : (FT*)m.redf;
  a.dtail_end = m.red + m.red_cap;      // float64 vectors at the tail of m.red
  a.ibase = m.bocc + (size_t)m.nc_cap * m.nc_cap;
  a.clist = m.clist; a.Sinv = m.Sinv; a.Bc = m.Bc; a.bocc = m.bocc;
  a.u = u; a.y2 = y2; a.z2 = z2;
  a.info = info;
  a.small_lim = std::is_same<FT, float>::value ? kClusNc : 0;
  a.one_cta_max = std::max(0, std::min(m.one_cta_max, kSmallNc));
  return a;
}

// Launch one of the cluster kernels (kCl CTAs per cluster).
cudaError_t launch_clus_v(cudaStream_t s, const RedArgs<float>& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCl);
  cfg.blockDim = dim3(kST);
  cfg.dynamicSmemBytes = kClusSmem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_clus_v, a);
  count_launch();
  return e;
}

template <typename FT>
cudaError_t launch_reduced_t(cudaStream_t s, const DevMesh& m, const double* u, const FT* y2,
                             double* z2, int* info, int num_sms, int refine, int nc_host,
                             bool prepared) {
  RedArgs<FT> a = make_args<FT>(m, u, y2, z2, info, refine);
  if constexpr (std::is_same<FT, float>::value) {
    // one-CTA path for 0 < n_c <= kSmallNc, 4-CTA cluster for n_c <= kClusNc
    // (every kernel reads n_c on the device and exits when it is not its
    // range).  With n_c known on the host (nc_host >= 0) only the kernels of
    // its path are launched and the z2 update runs as a plain launch, so
    // n_c <= kClusNc needs no cooperative launch (whose grid must find all of
    // its SMs free at once when other solves share the GPU).
    ProfScope ps(PROF_CHOL, s);
    const int zgrid = std::max(1, std::min(2 * std::max(1, num_sms), (m.n2 + 7) / 8));
    if (nc_host == 0) {
      k_z2_update<<<zgrid, 256, 0, s>>>(a);
      count_launch();
      return cudaGetLastError();
    }
    const bool known = nc_host > 0 && nc_host <= kClusNc;
    const bool want_small = !known || nc_host <= a.one_cta_max;
    const bool want_clus = !known || nc_host > a.one_cta_max;
    if (prepared) {       // S, L_s, lists, X and N came from reduced_prepare
      if (cudaStreamWaitEvent(s, m.ev_join, 0) != cudaSuccess) return cudaGetLastError();
      k_small_x<1><<<2 * std::max(1, num_sms), 256, 0, s>>>(a);
      count_launch();
    } else {
      k_small_s<<<1, kST, kSmallSmemS, s>>>(a);
      k_small_x<3><<<2 * std::max(1, num_sms), 256, 0, s>>>(a);
      k_small_n<<<kNTiles, 256, 0, s>>>(a);
      count_launch(3);
    }
    if (want_small) {
      k_small_v<<<1, kST, kSmallSmemV, s>>>(a);
      count_launch();
    }
    if (want_clus) {
      const cudaError_t e = launch_clus_v(s, a);
      if (e != cudaSuccess) return e;
    }
    if (known) {
      k_z2_update<<<zgrid, 256, 0, s>>>(a);
      count_launch();
      return cudaGetLastError();
    }
  }
  void* args[] = {&a};
  const int grid = std::max(1, num_sms);
  ProfScope ps(PROF_CHOL, s);
  const cudaError_t e = cudaLaunchCooperativeKernel((void*)k_reduced<FT>, dim3(grid), dim3(kRT), args, 0, s);
  count_launch();
  return e;
}

}  // namespace

int64_t reduced_workspace_elems(int nc) {
  const int64_t n3 = 3 * (int64_t)nc;
  // S, X, N (+1 row), 1/diag of both factors, two FT vectors, packed L_s, and
  // (at the tail of the float64 buffer) four float64 vectors
  return (int64_t)nc * nc + n3 * n3 + (n3 + 1) * n3 + nc + n3 + 2 * n3 +
         (prow(nc) + 1024 * ((int64_t)nc + 31) / 32 + 16) + 4 * n3 + (int64_t)nc * nc + 128;
}

// Most float64 refinement steps of a float32 reduced factor (see step 7).
constexpr int kMixedRefineSteps = 12;

int reduced_path(int nc_host, int precision, int one_cta_max) {
  if (precision == 0 || nc_host < 0 || nc_host > kClusNc) return 0;   // cooperative kernel
  if (nc_host == 0) return 1;
  return nc_host <= std::min(one_cta_max, kSmallNc) ? 2 : 3;
}

cudaError_t reduced_solve(cudaStream_t s, const DevMesh& m, const double* u, const void* y2,
                          double* z2, int* info, int num_sms, int precision, int nc_host,
                          bool prepared) {
  if (precision == 0)
    return launch_reduced_t<double>(s, m, u, (const double*)y2, z2, info, num_sms, 0, nc_host, false);
  return launch_reduced_t<float>(s, m, u, (const float*)y2, z2, info, num_sms, kMixedRefineSteps,
                                 nc_host, prepared);
}

namespace {

// x1 = bx1 + Phi[:, c] v.  A CTA covers 32 consecutive x1 solver positions
// (coalesced reads of the rows of Phi_t) with kPhiSplit warps, each summing
// a strided share of the n_c columns; v (as float) and the c list are staged
// in shared memory.  The work is bound by load latency, hence the split.
constexpr int kPhiSplit = 8;
__global__ void __launch_bounds__(32 * kPhiSplit) k_phi_apply(RedArgs<float> a, int n1,
                                                             const float* __restrict__ phi_t,
                                                             const float* __restrict__ bx1,
                                                             double* __restrict__ x1) {
  __shared__ float vs[3 * kClusNc];
  __shared__ int cs[kClusNc];
  __shared__ float part[kPhiSplit][3][32];
  const int nc = *a.nc_dev;
  const bool have = nc > 0 && nc <= a.small_lim;
  if (have) {
    red_layout(a, nc);
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      const bool okc = FSIM_CHECK_IDX(a.clist[k], a.n2, CHECK_CLIST);
      cs[k] = okc ? a.clist[k] : 0;
      vs[3 * k] = okc ? (float)a.v[3 * k] : 0.f;
      vs[3 * k + 1] = okc ? (float)a.v[3 * k + 1] : 0.f;
      vs[3 * k + 2] = okc ? (float)a.v[3 * k + 2] : 0.f;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f;
  if (have && p < n1) {
#pragma unroll 4
    for (int k = wq; k < nc; k += kPhiSplit) {
      const float f = phi_t[(size_t)cs[k] * n1 + p];
      c0 += f * vs[3 * k];
      c1 += f * vs[3 * k + 1];
      c2 += f * vs[3 * k + 2];
    }
  }
  part[wq][0][lane] = c0;
  part[wq][1][lane] = c1;
  part[wq][2][lane] = c2;
  __syncthreads();
  if (wq < 3 && p < n1) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < kPhiSplit; ++q) t += part[q][wq][lane];
    x1[3 * (size_t)p + wq] = (double)bx1[3 * (size_t)p + wq] + (double)t;
  }
}

// ---- lock-step batches: blockIdx.y = frame, RedArgs per frame on the device
template <int PARTS>
__global__ void __launch_bounds__(256) k_small_x_b(const RedArgs<float>* __restrict__ A) {
  const RedArgs<float> a = A[blockIdx.y];
  if (a.active) k_small_x_body<PARTS>(a);
}
__global__ void __launch_bounds__(kST) k_small_s_b(const RedArgs<float>* __restrict__ A) {
  const RedArgs<float> a = A[blockIdx.y];
  if (a.active) k_small_s_body(a);
}
__global__ void __launch_bounds__(256) k_small_n_b(const RedArgs<float>* __restrict__ A) {
  const RedArgs<float> a = A[blockIdx.y];
  if (a.active) k_small_n_body(a, blockIdx.x);
}
__global__ void __launch_bounds__(kST) k_small_v_b(const RedArgs<float>* __restrict__ A) {
  const RedArgs<float> a = A[blockIdx.y];
  if (a.active) k_small_v_body(a);
}
// one 4-CTA cluster per frame: the cluster spans blockIdx.x, the frame is
// blockIdx.y, so the inactive test is uniform over a cluster
__global__ void __maxnreg__(128) k_clus_v_b(const RedArgs<float>* __restrict__ A) {
  const RedArgs<float> a = A[blockIdx.y];
  if (a.active) k_clus_v_body(a);
}
__global__ void __launch_bounds__(256) k_z2_update_b(const RedArgs<float>* __restrict__ A) {
  const RedArgs<float> a = A[blockIdx.y];
  if (a.active) k_z2_update_body(a, true);
}

// x1 = bx1 + Phi[:, c] v for every frame and any n_c (v from whichever path
// solved the reduced system), with bx1 read from a multi-right-hand-side
// buffer: frame f's three columns start at column col_f of rows of nr floats.
__global__ void __launch_bounds__(32 * kPhiSplit) k_phi_apply_b(const RedArgs<float>* __restrict__ A,
                                                               const int* __restrict__ cols, int n1,
                                                               const float* __restrict__ phi_t,
                                                               const float* __restrict__ bxm, int nr,
                                                               double* const* __restrict__ x1s) {
  RedArgs<float> a = A[blockIdx.y];
  if (!a.active) return;
  __shared__ float vs[3 * kClusNc];
  __shared__ int cs[kClusNc];
  __shared__ float part[kPhiSplit][3][32];
  const int nc = *a.nc_dev;
  const int col = cols[blockIdx.y];
  double* x1 = x1s[blockIdx.y];
  if (nc > 0) red_layout(a, nc);
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f;
  for (int k0 = 0; k0 < nc; k0 += kClusNc) {       // n_c in chunks of the staging size
    const int kn = min(kClusNc, nc - k0);
    __syncthreads();
    for (int k = threadIdx.x; k < kn; k += blockDim.x) {
      const bool okc = FSIM_CHECK_IDX(a.clist[k0 + k], a.n2, CHECK_CLIST);
      cs[k] = okc ? a.clist[k0 + k] : 0;
      vs[3 * k] = okc ? (float)a.v[3 * (k0 + k)] : 0.f;
      vs[3 * k + 1] = okc ? (float)a.v[3 * (k0 + k) + 1] : 0.f;
      vs[3 * k + 2] = okc ? (float)a.v[3 * (k0 + k) + 2] : 0.f;
    }
    __syncthreads();
    if (p < n1) {
#pragma unroll 4
      for (int k = wq; k < kn; k += kPhiSplit) {
        const float f = phi_t[(size_t)cs[k] * n1 + p];
        c0 += f * vs[3 * k];
        c1 += f * vs[3 * k + 1];
        c2 += f * vs[3 * k + 2];
      }
    }
  }
  part[wq][0][lane] = c0;
  part[wq][1][lane] = c1;
  part[wq][2][lane] = c2;
  __syncthreads();
  if (wq < 3 && p < n1)  {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < kPhiSplit; ++q) t += part[q][wq][lane];
    x1[3 * (size_t)p + wq] = (double)bxm[(size_t)p * nr + col + wq] + (double)t;
  }
}

}  // namespace

size_t reduced_args_bytes() { return sizeof(RedArgs<float>); }

void reduced_args_fill(void* dst, const DevMesh& m, int active) {
  RedArgs<float> a = make_args<float>(m, m.u, (const float*)(m.rf + 3 * (size_t)m.n1),
                                      m.r + 3 * (size_t)m.n1, m.counters + 6, kMixedRefineSteps);
  a.active = active;
  std::memcpy(dst, &a, sizeof(a));
}

cudaError_t reduced_prepare_b(cudaStream_t s2, const void* args_dev, int nb, int num_sms) {
  const auto* A = static_cast<const RedArgs<float>*>(args_dev);
  ProfScope ps(PROF_CHOL, s2);
  k_small_s_b<<<dim3(1, nb), kST, kSmallSmemS, s2>>>(A);
  k_small_x_b<2><<<dim3((3 * kClusNc + kXRows - 1) / kXRows, nb), 256, 0, s2>>>(A);
  k_small_n_b<<<dim3(kNTiles, nb), 256, 0, s2>>>(A);
  count_launch(3);
  return cudaGetLastError();
}

cudaError_t reduced_solve_b(cudaStream_t s, const void* args_dev, const void* args_host, int nb,
                            const int* nc_host, int num_sms) {
  const auto* A = static_cast<const RedArgs<float>*>(args_dev);
  const auto* H = static_cast<const RedArgs<float>*>(args_host);
  bool any_small = false, any_clus = false;
  for (int f = 0; f < nb; ++f) {
    if (!H[f].active) continue;
    any_small |= nc_host[f] > 0 && nc_host[f] <= H[f].one_cta_max;
    any_clus |= nc_host[f] > H[f].one_cta_max && nc_host[f] <= kClusNc;
  }
  ProfScope ps(PROF_CHOL, s);
  k_small_x_b<1><<<dim3(std::max(1, 2 * num_sms / nb), nb), 256, 0, s>>>(A);
  count_launch();
  if (any_small) {
    k_small_v_b<<<dim3(1, nb), kST, kSmallSmemV, s>>>(A);
    count_launch();
  }
  if (any_clus) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCl, nb);
    cfg.blockDim = dim3(kST);
    cfg.dynamicSmemBytes = kClusSmem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kCl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_clus_v_b, A);
    count_launch();
    if (e != cudaSuccess) return e;
  }
  // n_c beyond the cluster path: the cooperative kernel, one frame at a time
  for (int f = 0; f < nb; ++f) {
    if (!H[f].active || nc_host[f] <= kClusNc) continue;
    RedArgs<float> a = H[f];
    void* args[] = {&a};
    const cudaError_t e = cudaLaunchCooperativeKernel((void*)k_reduced<float>,
                                                      dim3(std::max(1, num_sms)), dim3(kRT), args,
                                                      0, s);
    count_launch();
    if (e != cudaSuccess) return e;
  }
  // float64 row products, one row per lane: 256 rows per CTA of 8 warps,
  // enough CTAs to cover the rows of every frame (at least 2 per frame, also
  // for the n_c = 0 copy)
  const int zgrid = std::max(2, (H[0].n2 + 255) / 256);
  k_z2_update_b<<<dim3(zgrid, nb), 256, 0, s>>>(A);
  count_launch();
  return cudaGetLastError();
}

cudaError_t phi_apply_b(cudaStream_t s, const void* args_dev, const int* cols_dev, int nb, int n1,
                        const float* phi_t, const float* bxm, int nr, double* const* x1s_dev) {
  const auto* A = static_cast<const RedArgs<float>*>(args_dev);
  k_phi_apply_b<<<dim3((n1 + 31) / 32, nb), 32 * kPhiSplit, 0, s>>>(A, cols_dev, n1, phi_t, bxm, nr,
                                                                    x1s_dev);
  count_launch();
  return cudaGetLastError();
}

cudaError_t phi_apply(cudaStream_t s, const DevMesh& m, const double* u, const void* y2, double* z2,
                      int* info, const float* bx1, double* x1) {
  const RedArgs<float> a = make_args<float>(m, u, (const float*)y2, z2, info, kMixedRefineSteps);
  k_phi_apply<<<(m.n1 + 31) / 32, 32 * kPhiSplit, 0, s>>>(a, m.n1, m.Phi_t, bx1, x1);
  count_launch();
  return cudaGetLastError();
}

bool reduced_prepare(cudaStream_t s, const DevMesh& m, const double* u, const void* y2, double* z2,
                     int* info, int num_sms, int nc_host) {
  if (nc_host <= 0 || nc_host > kClusNc || !m.aux_stream || !m.ev_fork || !m.ev_join) return false;
  const RedArgs<float> a = make_args<float>(m, u, (const float*)y2, z2, info, kMixedRefineSteps);
  cudaStream_t s2 = m.aux_stream;
  if (cudaEventRecord(m.ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(s2, m.ev_fork, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  {
    ProfScope ps(PROF_CHOL, s2);
    k_small_s<<<1, kST, kSmallSmemS, s2>>>(a);
    k_small_x<2><<<2 * std::max(1, num_sms), 256, 0, s2>>>(a);
    k_small_n<<<kNTiles, 256, 0, s2>>>(a);
    count_launch(3);
  }
  // the join is recorded even if a launch failed, so the fork always closes
  cudaEventRecord(m.ev_join, s2);
  return true;
}

}  // namespace fsim

namespace fsim {
void set_reduced_smem_limits() {
  cudaFuncSetAttribute(k_small_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmemS);
  cudaFuncSetAttribute(k_small_v, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmemV);
  cudaFuncSetAttribute(k_clus_v, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusSmem);
  cudaFuncSetAttribute(k_small_s_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmemS);
  cudaFuncSetAttribute(k_small_v_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmemV);
  cudaFuncSetAttribute(k_clus_v_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusSmem);
}
FSIM_CHECK_READER(check_word_reduced)

}  // namespace fsim
