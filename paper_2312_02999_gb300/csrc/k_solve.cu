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
    // four independent loads and accumulators in flight per lane: the loop is
    // bound by load and FMA latency, not by bandwidth
    T q0 = 0, q1 = 0, q2 = 0, d0 = 0, d1 = 0, d2 = 0, e0 = 0, e1 = 0, e2 = 0;
    int k = wid;
    for (; k + 24 < kmax; k += 32) {
      const T z0 = Zj[(size_t)k * ld + r], z1 = Zj[(size_t)(k + 8) * ld + r];
      const T z2 = Zj[(size_t)(k + 16) * ld + r], z3 = Zj[(size_t)(k + 24) * ld + r];
      a0 += z0 * bj[3 * k]; a1 += z0 * bj[3 * k + 1]; a2 += z0 * bj[3 * k + 2];
      q0 += z1 * bj[3 * k + 24]; q1 += z1 * bj[3 * k + 25]; q2 += z1 * bj[3 * k + 26];
      d0 += z2 * bj[3 * k + 48]; d1 += z2 * bj[3 * k + 49]; d2 += z2 * bj[3 * k + 50];
      e0 += z3 * bj[3 * k + 72]; e1 += z3 * bj[3 * k + 73]; e2 += z3 * bj[3 * k + 74];
    }
    for (; k < kmax; k += 8) {
      const T z = Zj[(size_t)k * ld + r];
      a0 += z * bj[3 * k]; a1 += z * bj[3 * k + 1]; a2 += z * bj[3 * k + 2];
    }
    a0 += (q0 + d0) + e0; a1 += (q1 + d1) + e1; a2 += (q2 + d2) + e2;
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
    T a0 = 0, a1 = 0, a2 = 0, q0 = 0, q1 = 0, q2 = 0;
    int r = k + lane;
    for (; r + 32 < ld; r += 64) {
      const T z0 = zc[r], z1 = zc[r + 32];
      a0 += z0 * wv[3 * r]; a1 += z0 * wv[3 * r + 1]; a2 += z0 * wv[3 * r + 2];
      q0 += z1 * wv[3 * r + 96]; q1 += z1 * wv[3 * r + 97]; q2 += z1 * wv[3 * r + 98];
    }
    if (r < ld) {
      const T z = zc[r];
      a0 += z * wv[3 * r]; a1 += z * wv[3 * r + 1]; a2 += z * wv[3 * r + 2];
    }
    a0 += q0; a1 += q1; a2 += q2;
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

// Eq. 8 with H = K (x) I_3 in solver positions [x1 ; x2], r = -g-hat:
//   lower:    z1 = L1^-1 r1,  y2 = r2 - L21 z1        (one forward pass; the
//             x2 rows of the supernodes hold L21 = H21 L1^-T)
//   diagonal: dx2 = Sigma-hat^-1 y2 = u - Sigma^-1 Q^T v,  u = Sigma^-1 y2
//   upper:    dx1 = L1^-T (z1 - L21^T dx2)             (one backward pass)
template <typename T>
cudaError_t global_step_t(cudaStream_t s, const DevMesh& m, const double* g, double* dx, int nc,
                          int* info, int num_sms) {
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
      // The reduced system carries the barrier stiffness (cond ~ kappa b''):
      // float64 factors, or float32 factors refined with float64 residuals.
      ProfScope psr(PROF_REDUCED, s);
      const cudaError_t e = reduced_solve(s, m, nc, u, y2, z2, info, num_sms, f64 ? 0 : 1);
      if (e != cudaSuccess) return e;
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
  return cudaGetLastError();
}

}  // namespace

void set_solver_smem_limits(int max_bytes) {
  cudaFuncSetAttribute(k_fwd_chunk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
  cudaFuncSetAttribute(k_bwd_chunk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
  cudaFuncSetAttribute(k_fwd_chunk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
  cudaFuncSetAttribute(k_bwd_chunk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
}

cudaError_t global_step(cudaStream_t s, const DevMesh& m, const double* g, double* dx, int nc,
                        int precision, int* info_dev, int num_sms) {
  if (precision == 0) return global_step_t<double>(s, m, g, dx, nc, info_dev, num_sms);
  return global_step_t<float>(s, m, g, dx, nc, info_dev, num_sms);
}

}  // namespace fsim
