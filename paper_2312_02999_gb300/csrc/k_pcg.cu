// Global step by conjugate gradients preconditioned with the PD matrix: the
// paper's comparison configuration (Sec. 3, Eq. 5; Table 1, "IPC with
// PD-preconditioned CG").  It solves the same system as Eq. 8-11,
// (H + W^T grad^2 B W) dx = -g-hat, iteratively:
//   A p   = (K (x) I_3) p + W^T sum_pairs H_pair (W p)   (sparse K, pair blocks)
//   M^-1 r = H^-1 r   (the prefactored supernodal solves and Sigma^-1, i.e. the
//                      global step of Eq. 8 with the contact term left out)
// All vectors are in vertex order (3 per vertex); pinned vertices stay zero.
#include <cmath>

#include "kernels.h"

namespace fsim {

namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// y = (K (x) I_3) x over the free vertices (CSR in vertex order)
__global__ void k_spmv_k(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                         const double* __restrict__ val, const double* __restrict__ x,
                         double* __restrict__ y) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int e = ptr[v]; e < ptr[v + 1]; ++e) {
    const double k = val[e];
    const double* xc = x + 3 * (size_t)col[e];
    a0 += k * xc[0]; a1 += k * xc[1]; a2 += k * xc[2];
  }
  y[3 * (size_t)v] = a0; y[3 * (size_t)v + 1] = a1; y[3 * (size_t)v + 2] = a2;
}

// y += W^T H_pair W x for every active pair (12 x 12 blocks as 4 x 4 of 3 x 3)
__global__ void k_pair_apply(int64_t np, const int* __restrict__ count, const unsigned long long* __restrict__ pairs,
                             const int* __restrict__ tris, const int* __restrict__ edges,
                             const int64_t* __restrict__ Wptr, const int* __restrict__ Wcol,
                             const double* __restrict__ Wval, const uint8_t* __restrict__ pinned,
                             const double* __restrict__ phess, const double* __restrict__ x,
                             double* __restrict__ y) {
  int64_t n = *count;
  n = n < np ? n : np;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = pairs[p];
    const int type = (int)(key >> 62), i = (int)((key >> 31) & 0x7fffffffULL),
              j = (int)(key & 0x7fffffffULL);
    int V[4];
    if (type == 0) { V[0] = i; V[1] = tris[3 * j]; V[2] = tris[3 * j + 1]; V[3] = tris[3 * j + 2]; }
    else { V[0] = edges[2 * i]; V[1] = edges[2 * i + 1]; V[2] = edges[2 * j]; V[3] = edges[2 * j + 1]; }
    double xs[4][3];
    for (int b = 0; b < 4; ++b) {
      xs[b][0] = xs[b][1] = xs[b][2] = 0.0;
      for (int64_t e = Wptr[V[b]]; e < Wptr[V[b] + 1]; ++e) {
        const int v = Wcol[e];
        if (pinned[v]) continue;
        const double w = Wval[e];
        xs[b][0] += w * x[3 * (size_t)v]; xs[b][1] += w * x[3 * (size_t)v + 1];
        xs[b][2] += w * x[3 * (size_t)v + 2];
      }
    }
    const double* h = phess + p * 144;
    for (int a = 0; a < 4; ++a) {
      double ya[3] = {0.0, 0.0, 0.0};
      for (int b = 0; b < 4; ++b) {
        const double* hb = h + (a * 4 + b) * 9;
        for (int r = 0; r < 3; ++r) ya[r] += hb[3 * r] * xs[b][0] + hb[3 * r + 1] * xs[b][1] + hb[3 * r + 2] * xs[b][2];
      }
      for (int64_t e = Wptr[V[a]]; e < Wptr[V[a] + 1]; ++e) {
        const int v = Wcol[e];
        if (pinned[v]) continue;
        const double w = Wval[e];
        for (int r = 0; r < 3; ++r) atomicAdd(y + 3 * (size_t)v + r, w * ya[r]);
      }
    }
  }
}

// out[0] += a.b, out[1] += c.d (block partial sums, then atomics)
__global__ void k_dot2(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ c, const double* __restrict__ d, double* out) {
  double s0 = 0.0, s1 = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    s0 += a[e] * b[e];
    if (c) s1 += c[e] * d[e];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, s0);
    if (c) atomicAdd(out + 1, s1);
  }
}

// x += alpha p; r -= alpha q
__global__ void k_cg_update(int64_t n, double alpha, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  x[e] += alpha * p[e];
  r[e] -= alpha * q[e];
}

// p = z + beta p ; also used with beta = 0 for p = z
__global__ void k_cg_dir(int64_t n, double beta, const double* __restrict__ z, double* __restrict__ p) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  p[e] = z[e] + beta * p[e];
}

// out = -in
__global__ void k_neg(int64_t n, const double* __restrict__ in, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) out[e] = -in[e];
}

}  // namespace

int pcg_global_step(cudaStream_t s, const DevMesh& m, const double* g, double* dx, double rel_tol,
                    int max_iters, int* info_dev, int num_sms, double* h_scal2, int* iters_out) {
  const int64_t n3 = 3 * (int64_t)m.n;
  const unsigned nb = nblk(n3, 256);
  double* r = m.cg_r;
  double* z = m.cg_z;
  double* p = m.cg_p;
  double* q = m.cg_q;
  double* red = m.cg_red;   // 2 doubles on the device
  // the preconditioner M^-1 r = H^-1 r is the global step without contact:
  // the reduced-system kernels read n_c = 0 from counters[3]
  auto precond = [&](const double* rin, double* zout) -> int {
    k_neg<<<nb, 256, 0, s>>>(n3, rin, m.cg_tmp);
    count_launch();
    if (global_step(s, m, m.cg_tmp, zout, 0, info_dev, num_sms, true) != cudaSuccess) return -1;
    return 0;
  };
  auto dots = [&](const double* a, const double* b, const double* c, const double* d) -> int {
    if (cudaMemsetAsync(red, 0, sizeof(double) * 2, s) != cudaSuccess) return -1;
    k_dot2<<<2 * 152, 256, 0, s>>>(n3, a, b, c, d, red);
    count_launch();
    if (cudaMemcpyAsync(h_scal2, red, sizeof(double) * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return -1;
    return 0;
  };
  ProfScope ps(PROF_PCG, s);
  if (cudaMemsetAsync(m.counters + 3, 0, sizeof(int), s) != cudaSuccess) return -1;
  if (cudaMemsetAsync(dx, 0, sizeof(double) * n3, s) != cudaSuccess) return -1;
  k_neg<<<nb, 256, 0, s>>>(n3, g, r);          // r = -g - A 0
  count_launch();
  if (precond(r, z)) return -1;
  k_cg_dir<<<nb, 256, 0, s>>>(n3, 0.0, z, p);
  count_launch();
  if (dots(r, r, r, z)) return -1;
  const double r0 = std::sqrt(h_scal2[0]);
  double rz = h_scal2[1];
  int it = 0;
  if (r0 > 0.0) {
    for (; it < max_iters; ++it) {
      k_spmv_k<<<nblk(m.n, 128), 128, 0, s>>>(m.n, m.kv_ptr, m.kv_col, m.kv_val, p, q);
      k_pair_apply<<<2 * 152, 64, 0, s>>>(m.cap_act, m.counters, m.pairs, m.tris, m.edges, m.Wptr,
                                           m.Wcol, m.Wval, m.pinned, m.pair_hess, p, q);
      count_launch(2);
      if (dots(p, q, nullptr, nullptr)) return -1;
      const double pq = h_scal2[0];
      if (!(pq > 0.0)) break;                    // A is SPD; a breakdown ends the solve
      const double alpha = rz / pq;
      k_cg_update<<<nb, 256, 0, s>>>(n3, alpha, p, q, dx, r);
      count_launch();
      if (precond(r, z)) return -1;
      if (dots(r, r, r, z)) return -1;
      if (std::sqrt(h_scal2[0]) <= rel_tol * r0) { ++it; break; }
      const double rz_new = h_scal2[1];
      k_cg_dir<<<nb, 256, 0, s>>>(n3, rz_new / rz, z, p);
      count_launch();
      rz = rz_new;
    }
  }
  *iters_out = it;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace fsim
