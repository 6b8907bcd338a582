// Schur-complement-only global step (the paper's Sec. 3.1 configuration,
// before the low-rank update of Sec. 3.2): the x2 block of Eq. 8 is solved
// with the dense matrix Sigma-hat = Sigma (x) I_3 + B-hat_22 (Eq. 9),
// factored afresh every iteration, instead of Sigma^-1 and Eq. 11.
//
//   A  = Sigma (x) I_3  (3 n2 x 3 n2, dense, row-major),  A[c, c] += B-check
//   A  = L L^T          (right-looking blocked Cholesky, 64-wide panels)
//   z2 = L^-T L^-1 y2
//
// Precision 0 factors and solves in float64.  Precision 1 factors a float32
// copy and refines z2 twice with float64 residuals y2 - A z2 against the
// float64 A (each step gains about -log10(cond(A) * 6e-8) digits).
// A non-positive pivot sets info[0] (the matrix is SPD in exact arithmetic;
// the host reports FSIM_ENOT_SPD) and the factorisation continues with 1.
#include <algorithm>

#include "kernels.h"

namespace fsim {

namespace {

constexpr int kNb = 64;          // panel width
constexpr int kTrsmRows = 128;   // rows per CTA in the panel solve

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// A = Sigma (x) I_3 (float64), plus a float32 copy when Af != nullptr
__global__ void k_sigma_kron(int n2, const double* __restrict__ Sig, double* __restrict__ A,
                             float* __restrict__ Af) {
  const int64_t N = 3 * (int64_t)n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / N, c = e - r * N;
    const double v = (r % 3 == c % 3) ? Sig[(r / 3) * n2 + c / 3] : 0.0;
    A[e] = v;
    if (Af) Af[e] = (float)v;
  }
}

// A[3 q_i + a][3 q_j + b] += B-check[3 i + a][3 j + b] over the n_c list
// (n_c read on the device)
__global__ void k_add_bcheck(int n2, const int* __restrict__ ncp, const int* __restrict__ clist,
                             const double* __restrict__ Bc, double* __restrict__ A,
                             float* __restrict__ Af) {
  const int nc = *ncp;
  const int64_t ld = 3 * (int64_t)nc, N = 3 * (int64_t)n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ld * ld;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ld, c = e - r * ld;
    const int64_t R = 3 * (int64_t)clist[r / 3] + r % 3, C = 3 * (int64_t)clist[c / 3] + c % 3;
    const double v = A[R * N + C] + Bc[e];
    A[R * N + C] = v;
    if (Af) Af[R * N + C] = (float)v;
  }
}

// Unblocked Cholesky of the nb x nb diagonal block at (k0, k0), in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_potrf_diag(T* __restrict__ A, int64_t N, int k0, int nb,
                                                    int* __restrict__ info) {
  __shared__ T Ls[kNb][kNb + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    Ls[i][j] = A[(int64_t)(k0 + i) * N + k0 + j];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      T d = Ls[j][j];
      if (!(d > T(0))) {
        atomicExch(info, 1);
        d = T(1);
      }
      Ls[j][j] = sqrt(d);
    }
    __syncthreads();
    const T piv = Ls[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) Ls[i][j] /= piv;
    __syncthreads();
    const int m = nb - j - 1;                 // trailing (m x m) lower update
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, l = j + 1 + e % m;
      if (l <= i) Ls[i][l] -= Ls[i][j] * Ls[l][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    if (j <= i) A[(int64_t)(k0 + i) * N + k0 + j] = Ls[i][j];
  }
}

// Panel solve: rows i >= k0 + nb of columns k0 .. k0 + nb - 1 become
// A[i, panel] L_kk^-T (one thread per row, forward substitution).
template <typename T>
__global__ void __launch_bounds__(kTrsmRows) k_trsm_panel(T* __restrict__ A, int64_t N, int k0,
                                                          int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);              // nb x nb (ld kNb)
  T* Xs = Ls + kNb * kNb;                              // [kNb][kTrsmRows]
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    Ls[i * kNb + j] = A[(int64_t)(k0 + i) * N + k0 + j];
  }
  __syncthreads();
  const int64_t row = (int64_t)k0 + nb + (int64_t)blockIdx.x * kTrsmRows + threadIdx.x;
  if (row >= N) return;
  T* a = A + row * N + k0;
  for (int j = 0; j < nb; ++j) {
    T v = a[j];
    for (int l = 0; l < j; ++l) v -= Ls[j * kNb + l] * Xs[l * kTrsmRows + threadIdx.x];
    v /= Ls[j * kNb + j];
    Xs[j * kTrsmRows + threadIdx.x] = v;
  }
  for (int j = 0; j < nb; ++j) a[j] = Xs[j * kTrsmRows + threadIdx.x];
}

// Trailing update A[I, J] -= A[I, panel] A[J, panel]^T over the 64 x 64 tiles
// with J <= I below the panel (16 x 16 threads, 4 x 4 outputs each).
constexpr int kLdT = kNb + 1;     // padded tile row

template <typename T>
__global__ void __launch_bounds__(256) k_syrk_tiles(T* __restrict__ A, int64_t N, int k0, int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T (*As)[kLdT] = reinterpret_cast<T (*)[kLdT]>(smem_raw);   // As[l][r] = A[i0 + r][k0 + l]
  T (*Bs)[kLdT] = As + kNb;                                    // Bs[l][c] = A[j0 + c][k0 + l]
  const int64_t k1 = (int64_t)k0 + nb;
  // tile t -> (ti, tj), tj <= ti, in row-major order of the lower triangle
  const int64_t t = blockIdx.x;
  int64_t ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int64_t tj = t - ti * (ti + 1) / 2;
  const int64_t i0 = k1 + ti * kNb, j0 = k1 + tj * kNb;
  for (int e = threadIdx.x; e < kNb * kNb; e += blockDim.x) {
    const int r = e / kNb, l = e - r * kNb;
    As[l][r] = (i0 + r < N && l < nb) ? A[(i0 + r) * N + k0 + l] : T(0);
    Bs[l][r] = (j0 + r < N && l < nb) ? A[(j0 + r) * N + k0 + l] : T(0);
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 8
  for (int l = 0; l < kNb; ++l) {
    T x[4], y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = As[l][ty + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = Bs[l][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += x[a] * y[b];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + ty + 16 * a;
    if (i >= N) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = j0 + tx + 16 * b;
      if (j < N && j <= i) A[i * N + j] -= acc[a][b];
    }
  }
}

// Forward block: z[k0 .. k0+nb) = L_kk^-1 z[k0 .. k0+nb) (one warp), in place.
template <typename T>
__global__ void k_trsv_diag_fwd(const T* __restrict__ L, int64_t N, int k0, int nb, T* __restrict__ z) {
  __shared__ T zs[kNb];
  const int lane = threadIdx.x;
  for (int i = lane; i < nb; i += 32) zs[i] = z[k0 + i];
  __syncwarp();
  for (int j = 0; j < nb; ++j) {
    const T zj = zs[j] / L[(int64_t)(k0 + j) * N + k0 + j];
    __syncwarp();
    for (int i = j + 1 + lane; i < nb; i += 32) zs[i] -= L[(int64_t)(k0 + i) * N + k0 + j] * zj;
    if (lane == 0) zs[j] = zj;
    __syncwarp();
  }
  for (int i = lane; i < nb; i += 32) z[k0 + i] = zs[i];
}

// z[i] -= sum_l L[i][k0 + l] z[k0 + l] for rows i >= k0 + nb (one warp per row)
template <typename T>
__global__ void k_trsv_update_fwd(const T* __restrict__ L, int64_t N, int k0, int nb, T* __restrict__ z) {
  const int64_t row = (int64_t)k0 + nb + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  T v = T(0);
  for (int l = lane; l < nb; l += 32) v += L[row * N + k0 + l] * z[k0 + l];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) z[row] -= v;
}

// Backward block: z[k0 .. k0+nb) = L_kk^-T z[k0 .. k0+nb) (one warp), in place.
template <typename T>
__global__ void k_trsv_diag_bwd(const T* __restrict__ L, int64_t N, int k0, int nb, T* __restrict__ z) {
  __shared__ T zs[kNb];
  const int lane = threadIdx.x;
  for (int i = lane; i < nb; i += 32) zs[i] = z[k0 + i];
  __syncwarp();
  for (int j = nb - 1; j >= 0; --j) {
    const T zj = zs[j] / L[(int64_t)(k0 + j) * N + k0 + j];
    __syncwarp();
    for (int i = lane; i < j; i += 32) zs[i] -= L[(int64_t)(k0 + j) * N + k0 + i] * zj;
    if (lane == 0) zs[j] = zj;
    __syncwarp();
  }
  for (int i = lane; i < nb; i += 32) z[k0 + i] = zs[i];
}

// z[j] -= sum_l L[k0 + l][j] z[k0 + l] for columns j < k0 (coalesced over j)
template <typename T>
__global__ void k_trsv_update_bwd(const T* __restrict__ L, int64_t N, int k0, int nb, T* __restrict__ z) {
  __shared__ T zk[kNb];
  for (int l = threadIdx.x; l < nb; l += blockDim.x) zk[l] = z[k0 + l];
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k0) return;
  T v = T(0);
  for (int l = 0; l < nb; ++l) v += L[(int64_t)(k0 + l) * N + j] * zk[l];
  z[j] -= v;
}

// r = y - A z (float64, one warp per row)
__global__ void k_residual(const double* __restrict__ A, int64_t N, const double* __restrict__ y,
                           const double* __restrict__ z, double* __restrict__ r) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  double v = 0.0;
  for (int64_t c = lane; c < N; c += 32) v += A[row * N + c] * z[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) r[row] = y[row] - v;
}

template <typename S, typename T>
__global__ void k_copy_cast(int64_t n, const S* __restrict__ a, T* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

__global__ void k_add_to(int64_t n, const float* __restrict__ d, double* __restrict__ z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] += (double)d[i];
}

template <typename T>
void dense_potrf(cudaStream_t s, T* A, int64_t N, int* info) {
  const size_t trsm_smem = sizeof(T) * (kNb * kNb + kNb * kTrsmRows);
  const size_t syrk_smem = sizeof(T) * 2 * kNb * kLdT;
  for (int k0 = 0; k0 < N; k0 += kNb) {
    const int nb = (int)std::min<int64_t>(kNb, N - k0);
    k_potrf_diag<T><<<1, 256, 0, s>>>(A, N, k0, nb, info);
    const int64_t below = N - k0 - nb;
    count_launch();
    if (below <= 0) break;
    k_trsm_panel<T><<<nblk(below, kTrsmRows), kTrsmRows, trsm_smem, s>>>(A, N, k0, nb);
    const int64_t M = (below + kNb - 1) / kNb;
    k_syrk_tiles<T><<<(unsigned)(M * (M + 1) / 2), 256, syrk_smem, s>>>(A, N, k0, nb);
    count_launch(2);
  }
}

template <typename T>
void dense_solve(cudaStream_t s, const T* L, int64_t N, T* z) {
  for (int k0 = 0; k0 < N; k0 += kNb) {
    const int nb = (int)std::min<int64_t>(kNb, N - k0);
    k_trsv_diag_fwd<T><<<1, 32, 0, s>>>(L, N, k0, nb, z);
    count_launch();
    const int64_t below = N - k0 - nb;
    if (below > 0) {
      k_trsv_update_fwd<T><<<nblk(below * 32, 256), 256, 0, s>>>(L, N, k0, nb, z);
      count_launch();
    }
  }
  const int64_t last = ((N - 1) / kNb) * kNb;
  for (int64_t k0 = last; k0 >= 0; k0 -= kNb) {
    const int nb = (int)std::min<int64_t>(kNb, N - k0);
    k_trsv_diag_bwd<T><<<1, 32, 0, s>>>(L, N, (int)k0, nb, z);
    count_launch();
    if (k0 > 0) {
      k_trsv_update_bwd<T><<<nblk(k0, 256), 256, 0, s>>>(L, N, (int)k0, nb, z);
      count_launch();
    }
  }
}

}  // namespace

void set_schur_smem_limits() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaFuncSetAttribute(k_trsm_panel<double>, a, (int)(sizeof(double) * (kNb * kNb + kNb * kTrsmRows)));
  cudaFuncSetAttribute(k_trsm_panel<float>, a, (int)(sizeof(float) * (kNb * kNb + kNb * kTrsmRows)));
  cudaFuncSetAttribute(k_syrk_tiles<double>, a, (int)(sizeof(double) * 2 * kNb * kLdT));
  cudaFuncSetAttribute(k_syrk_tiles<float>, a, (int)(sizeof(float) * 2 * kNb * kLdT));
}

cudaError_t sigma_hat_solve(cudaStream_t s, const DevMesh& m, const void* y2, double* z2, int* info,
                            int precision) {
  const int n2 = m.n2;
  const int64_t N = 3 * (int64_t)n2;
  if (N == 0) return cudaSuccess;
  const unsigned g = 2 * 152;
  ProfScope ps(PROF_SCHUR, s);
  k_sigma_kron<<<g * 4, 256, 0, s>>>(n2, m.Sig, m.sh_A, precision ? m.sh_Af : nullptr);
  k_add_bcheck<<<g, 256, 0, s>>>(n2, m.counters + 3, m.clist, m.Bc, m.sh_A,
                                 precision ? m.sh_Af : nullptr);
  count_launch(2);
  if (precision == 0) {
    k_copy_cast<double, double><<<nblk(N, 256), 256, 0, s>>>(N, (const double*)y2, z2);
    count_launch();
    dense_potrf<double>(s, m.sh_A, N, info);        // in place
    dense_solve<double>(s, m.sh_A, N, z2);
    return cudaGetLastError();
  }
  // float32 factor, float64 refinement
  const float* y2f = (const float*)y2;
  double* y64 = m.sh_y;       // y2 in float64
  double* r64 = m.sh_r;
  float* df = m.sh_df;
  k_copy_cast<float, double><<<nblk(N, 256), 256, 0, s>>>(N, y2f, y64);
  k_copy_cast<float, float><<<nblk(N, 256), 256, 0, s>>>(N, y2f, df);
  count_launch(2);
  dense_potrf<float>(s, m.sh_Af, N, info);
  dense_solve<float>(s, m.sh_Af, N, df);
  k_copy_cast<float, double><<<nblk(N, 256), 256, 0, s>>>(N, df, z2);
  count_launch();
  for (int it = 0; it < 2; ++it) {
    k_residual<<<nblk(N * 32, 256), 256, 0, s>>>(m.sh_A, N, y64, z2, r64);
    k_copy_cast<double, float><<<nblk(N, 256), 256, 0, s>>>(N, r64, df);
    count_launch(2);
    dense_solve<float>(s, m.sh_Af, N, df);
    k_add_to<<<nblk(N, 256), 256, 0, s>>>(N, df, z2);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace fsim
