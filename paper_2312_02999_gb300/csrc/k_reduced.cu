// Reduced contact system of Sec. 3.2 in one cooperative launch.
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
//     barrier stiffness and can be many orders larger.
//   8 z2 = u - (Sigma^-1[:, c] (x) I_3) v
// Pivots use a float32 reciprocal square root refined by two float64 Newton
// steps (float64-accurate, a far shorter dependent chain than sqrt and a
// division on GB300's float64 pipe).
#include <cooperative_groups.h>

#include <algorithm>
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
  int* info;
};

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
  a.nc = nc;
  a.S = a.base;
  a.X = a.S + (size_t)nc * nc;
  a.N = a.X + (size_t)n3 * n3;
  a.dinv_s = a.N + (size_t)(n3 + 1) * n3;
  a.dinv_n = a.dinv_s + nc;
  a.fv = a.dinv_n + n3;
  a.y = a.dtail_end - 4 * (size_t)n3 - 8;
  a.v = a.y + n3; a.rho = a.v + n3; a.w = a.rho + n3; a.nrm = a.w + n3;
  a.list = a.ibase;
  a.cnt = a.list + (size_t)nc * nc;

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
  // 8. z2 = u - (Sigma^-1[:, c] (x) I_3) v, one warp per row
  for (int q = gwarp; q < a.n2; q += nwarps) {
    const double* srow = a.Sinv + (size_t)q * a.n2;
    double a0 = 0, a1 = 0, a2 = 0;
    for (int m = lane; m < nc; m += 32) {
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

template <typename FT>
cudaError_t launch_reduced_t(cudaStream_t s, const DevMesh& m, const double* u, const FT* y2,
                             double* z2, int* info, int num_sms, int refine) {
  RedArgs<FT> a{};
  a.n2 = m.n2; a.refine = refine;
  a.nc_dev = m.counters + 3;
  a.base = std::is_same<FT, double>::value ? (FT*)m.red : (FT*)m.redf;
  a.dtail_end = m.red + m.red_cap;      // float64 vectors at the tail of m.red
  a.ibase = m.bocc + (size_t)m.nc_cap * m.nc_cap;
  a.clist = m.clist; a.Sinv = m.Sinv; a.Bc = m.Bc; a.bocc = m.bocc;
  a.u = u; a.y2 = y2; a.z2 = z2;
  a.info = info;
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
  // S, X, N (+1 row), 1/diag of both factors, two FT vectors, and (at the
  // tail of the float64 buffer) four float64 vectors
  return (int64_t)nc * nc + n3 * n3 + (n3 + 1) * n3 + nc + n3 + 2 * n3 + 4 * n3 + 64;
}

cudaError_t reduced_solve(cudaStream_t s, const DevMesh& m, const double* u, const void* y2,
                          double* z2, int* info, int num_sms, int precision) {
  if (precision == 0)
    return launch_reduced_t<double>(s, m, u, (const double*)y2, z2, info, num_sms, 0);
  return launch_reduced_t<float>(s, m, u, (const float*)y2, z2, info, num_sms, 4);
}

}  // namespace fsim
