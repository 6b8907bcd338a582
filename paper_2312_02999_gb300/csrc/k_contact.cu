// IPC work on the proxy surface: s = W x (Sec. 3.1), UpdateConstraintSet,
// barrier energy (Eq. 3), PSD barrier Hessian mapped through W into the
// reduced block B-check (Eq. 10) and the additive-CCD step bound (Algorithm 1).
//
// Broad phase: all point-triangle and edge-edge pairs are swept in tiles;
// each primitive's box is rounded outward to float32 so that the float32
// overlap test keeps every pair the exact float64 test keeps.  The float64
// test (boxes inflated by dhat, closed intervals) then decides CCD candidates
// exactly as the oracle does, and the float64 distance decides d < dhat.
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

__global__ void k_proxy(int Ns, const int64_t* __restrict__ Wptr, const int* __restrict__ Wcol,
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
  if (idx < cap) out[idx] = key;
  else atomicOr(overflow, 1);
}

// MODE 0: constraint set (d < dhat) + barrier energy;  MODE 1: CCD candidates
// (swept boxes, exact float64 overlap test)
template <int MODE>
__global__ void __launch_bounds__(kTile)
k_pairs_pt(int Ns, int Nt, const double* __restrict__ s, const double* __restrict__ ds,
           const int* __restrict__ tris, double dhat, double kappa,
           unsigned long long* __restrict__ out, int* counters, int64_t cap, double* scal) {
  __shared__ Box32 tb[kTile];
  __shared__ int tid3[kTile][3];
  const int t0 = blockIdx.y * kTile;
  for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
    const int t = t0 + k;
    if (t < Nt) {
      int ids[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
      double lo[3], hi[3];
      prim_box<3>(s, MODE == 1 ? ds : nullptr, ids, lo, hi);
      tb[k] = to_box32(lo, hi, 0.0);
      tid3[k][0] = ids[0]; tid3[k][1] = ids[1]; tid3[k][2] = ids[2];
    } else {
      tid3[k][0] = -1;
    }
  }
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= Ns) return;
  double vlo[3], vhi[3];
  prim_box<1>(s, MODE == 1 ? ds : nullptr, &v, vlo, vhi);
  const Box32 vb = to_box32(vlo, vhi, dhat);
  const int nt = min(kTile, Nt - t0);
  double esum = 0.0;
  for (int k = 0; k < nt; ++k) {
    if (!box_overlap32(vb, tb[k])) continue;
    const int a = tid3[k][0], b = tid3[k][1], c = tid3[k][2];
    if (a == v || b == v || c == v) continue;
    const int t = t0 + k;
    if (MODE == 1) {
      double tlo[3], thi[3];
      int ids[3] = {a, b, c};
      prim_box<3>(s, ds, ids, tlo, thi);
      if (box_overlap64(vlo, vhi, tlo, thi, dhat))
        append(pack_key(0, v, t), out, counters + 1, counters + 2, cap);
    } else {
      const int V[4] = {v, a, b, c};
      double X[4][3];
      gather_X(s, V, X);
      float Xf[4][3];
      to_rel_f(X, Xf);
      if (pair_distance_f(0, Xf) > 2.0f * (float)dhat) continue;   // far: skip float64 work
      const double d = pair_distance(0, X);
      if (d < dhat) {
        append(pack_key(0, v, t), out, counters + 0, counters + 2, cap);
        esum += barrier_value(d, dhat);
        if (!(d > 0.0)) atomicOr(counters + 5, 1);
      }
    }
  }
  if (MODE == 0 && esum != 0.0) atomicAdd(scal + 0, kappa * esum);
}

template <int MODE>
__global__ void __launch_bounds__(kTile)
k_pairs_ee(int Ne, const double* __restrict__ s, const double* __restrict__ ds,
           const int* __restrict__ edges, double dhat, double kappa,
           unsigned long long* __restrict__ out, int* counters, int64_t cap, double* scal) {
  if (blockIdx.y < blockIdx.x) return;        // tiles with j-tile >= i-tile
  __shared__ Box32 eb[kTile];
  __shared__ int eid[kTile][2];
  const int j0 = blockIdx.y * kTile;
  for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
    const int e = j0 + k;
    if (e < Ne) {
      int ids[2] = {edges[2 * e], edges[2 * e + 1]};
      double lo[3], hi[3];
      prim_box<2>(s, MODE == 1 ? ds : nullptr, ids, lo, hi);
      eb[k] = to_box32(lo, hi, 0.0);
      eid[k][0] = ids[0]; eid[k][1] = ids[1];
    }
  }
  __syncthreads();
  const int i = blockIdx.x * kTile + threadIdx.x;
  if (i >= Ne) return;
  const int ia[2] = {edges[2 * i], edges[2 * i + 1]};
  double ilo[3], ihi[3];
  prim_box<2>(s, MODE == 1 ? ds : nullptr, ia, ilo, ihi);
  const Box32 ib = to_box32(ilo, ihi, dhat);
  const int ne = min(kTile, Ne - j0);
  double esum = 0.0;
  for (int k = 0; k < ne; ++k) {
    const int j = j0 + k;
    if (j <= i) continue;
    if (!box_overlap32(ib, eb[k])) continue;
    const int b0 = eid[k][0], b1 = eid[k][1];
    if (b0 == ia[0] || b0 == ia[1] || b1 == ia[0] || b1 == ia[1]) continue;
    if (MODE == 1) {
      double jlo[3], jhi[3];
      int ids[2] = {b0, b1};
      prim_box<2>(s, ds, ids, jlo, jhi);
      if (box_overlap64(ilo, ihi, jlo, jhi, dhat))
        append(pack_key(1, i, j), out, counters + 1, counters + 2, cap);
    } else {
      const int V[4] = {ia[0], ia[1], b0, b1};
      double X[4][3];
      gather_X(s, V, X);
      float Xf[4][3];
      to_rel_f(X, Xf);
      if (pair_distance_f(1, Xf) > 2.0f * (float)dhat) continue;   // far: skip float64 work
      const double d = pair_distance(1, X);
      if (d < dhat) {
        append(pack_key(1, i, j), out, counters + 0, counters + 2, cap);
        esum += barrier_value(d, dhat);
        if (!(d > 0.0)) atomicOr(counters + 5, 1);
      }
    }
  }
  if (MODE == 0 && esum != 0.0) atomicAdd(scal + 0, kappa * esum);
}

// Pass A: per-pair gradient and PSD Hessian blocks; mark touched x2 vertices.
__global__ void k_barrier_pairs(int64_t np, const unsigned long long* __restrict__ pairs,
                                const double* __restrict__ s, const int* __restrict__ tris,
                                const int* __restrict__ edges, const int64_t* __restrict__ Wptr,
                                const int* __restrict__ Wcol, const int* __restrict__ x2of,
                                double dhat, double kappa, double* __restrict__ pgrad,
                                double* __restrict__ phess, int* __restrict__ x2mark) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  int type, i, j;
  unpack_key(pairs[p], type, i, j);
  int V[4];
  load_pair(type, i, j, tris, edges, V);
  double X[4][3];
  gather_X(s, V, X);
  double gr[4][3], H[4][4][9];
  pair_barrier_psd(type, X, dhat, kappa, gr, H);
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) pgrad[p * 12 + 3 * k + d] = gr[k][d];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int e = 0; e < 9; ++e) phess[p * 144 + (a * 4 + b) * 9 + e] = H[a][b][e];
  for (int k = 0; k < 4; ++k)
    for (int64_t e = Wptr[V[k]]; e < Wptr[V[k] + 1]; ++e) {
      const int q = x2of[Wcol[e]];
      if (q >= 0) x2mark[q] = 1;
    }
}

// x2mark (0/1 flags) -> x2mark[q] = c position + 1 (0 if untouched); clist; nc.
__global__ void k_mark_scan(int n2, int* __restrict__ x2mark, int* __restrict__ clist,
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

// Pass C: scatter gradients (through W) into g and blocks into B-check.
__global__ void k_barrier_scatter(int64_t np, const unsigned long long* __restrict__ pairs,
                                  const int* __restrict__ tris, const int* __restrict__ edges,
                                  const int64_t* __restrict__ Wptr, const int* __restrict__ Wcol,
                                  const double* __restrict__ Wval, const int* __restrict__ x2of,
                                  const int* __restrict__ x2mark, const double* __restrict__ pgrad,
                                  const double* __restrict__ phess, int nc, double* __restrict__ g,
                                  double* __restrict__ Bc, int* __restrict__ bocc) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  int type, i, j;
  unpack_key(pairs[p], type, i, j);
  int V[4];
  load_pair(type, i, j, tris, edges, V);
  const int ld = 3 * nc;
  for (int a = 0; a < 4; ++a) {
    for (int64_t ea = Wptr[V[a]]; ea < Wptr[V[a] + 1]; ++ea) {
      const int va = Wcol[ea];
      const int qa = x2of[va];
      if (qa < 0) continue;                       // pinned: no DOF
      const double wa = Wval[ea];
      for (int d = 0; d < 3; ++d) atomicAdd(g + 3 * (size_t)va + d, wa * pgrad[p * 12 + 3 * a + d]);
      const int ca = x2mark[qa] - 1;
      if (ca < 0 || ca >= nc) continue;
      for (int b = 0; b < 4; ++b)
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

__global__ void k_accd(int64_t nc, const unsigned long long* __restrict__ cand,
                       const double* __restrict__ s, const double* __restrict__ ds,
                       const int* __restrict__ tris, const int* __restrict__ edges,
                       double s_ratio, int max_iters, double* __restrict__ alpha) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nc) return;
  int type, i, j;
  unpack_key(cand[p], type, i, j);
  int V[4];
  load_pair(type, i, j, tris, edges, V);
  double X[4][3], dX[4][3];
  gather_X(s, V, X);
  gather_X(ds, V, dX);
  const double toi = accd_toi(type, X, dX, s_ratio, max_iters);
  if (toi < 1.0)
    atomicMin(reinterpret_cast<unsigned long long*>(alpha), (unsigned long long)__double_as_longlong(toi));
}

// ---------------------------------------------------------------------------
void launch_proxy(cudaStream_t st, const DevMesh& m, const double* x, double* sp) {
  k_proxy<<<(m.Ns + 255) / 256, 256, 0, st>>>(m.Ns, m.Wptr, m.Wcol, m.Wval, x, sp);
  count_launch();
}

void launch_detect(cudaStream_t st, const DevMesh& m, const double* sp, double dhat, double kappa) {
  ProfScope ps(PROF_DETECT, st);
  if (m.Ns > 0 && m.Nt > 0) {
    dim3 gpt((m.Ns + kTile - 1) / kTile, (m.Nt + kTile - 1) / kTile);
    k_pairs_pt<0><<<gpt, kTile, 0, st>>>(m.Ns, m.Nt, sp, nullptr, m.tris, dhat, kappa, m.pairs,
                                         m.counters, m.cap, m.scal);
    count_launch();
  }
  if (m.Ne > 1) {
    const int ne = (m.Ne + kTile - 1) / kTile;
    dim3 gee(ne, ne);
    k_pairs_ee<0><<<gee, kTile, 0, st>>>(m.Ne, sp, nullptr, m.edges, dhat, kappa, m.pairs,
                                         m.counters, m.cap, m.scal);
    count_launch();
  }
}

void launch_ccd_candidates(cudaStream_t st, const DevMesh& m, const double* sp, const double* dsp,
                           double dhat) {
  ProfScope ps(PROF_CCD, st);
  if (m.Ns > 0 && m.Nt > 0) {
    dim3 gpt((m.Ns + kTile - 1) / kTile, (m.Nt + kTile - 1) / kTile);
    k_pairs_pt<1><<<gpt, kTile, 0, st>>>(m.Ns, m.Nt, sp, dsp, m.tris, dhat, 0.0, m.cand,
                                         m.counters, m.cap, m.scal);
    count_launch();
  }
  if (m.Ne > 1) {
    const int ne = (m.Ne + kTile - 1) / kTile;
    dim3 gee(ne, ne);
    k_pairs_ee<1><<<gee, kTile, 0, st>>>(m.Ne, sp, dsp, m.edges, dhat, 0.0, m.cand, m.counters,
                                         m.cap, m.scal);
    count_launch();
  }
}

void launch_ccd(cudaStream_t st, const DevMesh& m, const double* sp, const double* dsp, double dhat,
                double ccd_s, int accd_max_iters, int64_t ncand) {
  (void)dhat;
  ncand = ncand < m.cap ? ncand : m.cap;   // an overflowed list holds only cap keys
  if (ncand <= 0) return;
  ProfScope ps(PROF_CCD, st);
  k_accd<<<(unsigned)((ncand + 127) / 128), 128, 0, st>>>(ncand, m.cand, sp, dsp, m.tris, m.edges,
                                                         ccd_s, accd_max_iters, m.scal + 1);
  count_launch();
}

void launch_barrier_pairs(cudaStream_t st, const DevMesh& m, int64_t np, const double* sp,
                          double dhat, double kappa) {
  np = np < m.cap ? np : m.cap;
  if (np <= 0) return;
  ProfScope ps(PROF_BARRIER, st);
  k_barrier_pairs<<<(unsigned)((np + 63) / 64), 64, 0, st>>>(np, m.pairs, sp, m.tris, m.edges,
                                                            m.Wptr, m.Wcol, m.x2of, dhat, kappa,
                                                            m.pair_grad, m.pair_hess, m.x2mark);
  count_launch();
}

void launch_mark_scan(cudaStream_t st, const DevMesh& m) {
  k_mark_scan<<<1, 1024, 0, st>>>(m.n2, m.x2mark, m.clist, m.counters);
  count_launch();
}

void launch_barrier_scatter(cudaStream_t st, const DevMesh& m, int64_t np, int nc, double* g) {
  np = np < m.cap ? np : m.cap;
  if (np <= 0) return;
  k_barrier_scatter<<<(unsigned)((np + 63) / 64), 64, 0, st>>>(np, m.pairs, m.tris, m.edges,
                                                              m.Wptr, m.Wcol, m.Wval, m.x2of,
                                                              m.x2mark, m.pair_grad, m.pair_hess,
                                                              nc, g, m.Bc, m.bocc);
  count_launch();
}

}  // namespace fsim

// ===========================================================================
// CCD step bound without any device allocation.
//
// Some callers cannot let a library allocate GPU memory: an animation or game
// engine that reserves all device memory up front in its own pool, a host
// application that must stay inside a fixed memory budget, or code that is
// about to be recorded into someone else's CUDA graph.  For them,
// fsim_ccd_noalloc computes the same additive-CCD step bound as the solver's
// CCD stage, with every input and output owned by the caller and its only
// scratch (the candidate-pair list and two counters) in the fixed array below.
// ===========================================================================
namespace fsim {
namespace {

// Largest candidate list the static scratch holds (8 MiB of keys).
constexpr int64_t kNoallocCandidates = int64_t(1) << 20;
// Words [0, 2): four int counters ([1] candidates, [2] overflow flag), as the
// pair kernels use them; words [2, 2 + kNoallocCandidates): candidate keys.
// Every GPU that loads the library keeps this array until the process exits.
constexpr int kNoallocHeaderWords = 2;
static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[kNoallocHeaderWords + kNoallocCandidates];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSIM_ECUDA;
  // one-time set-up per device: the host-side name of the array is not a
  // device address, so ask the runtime for the address on this device
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return FSIM_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* base = (unsigned long long*)g_noalloc_ptr[dev];
  int* counters = reinterpret_cast<int*>(base);          // header: 4 ints
  unsigned long long* keys = base + kNoallocHeaderWords;
  // the array keeps the previous call's contents: reset the counters
  if (cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * kNoallocHeaderWords, st) !=
      cudaSuccess)
    return FSIM_ECUDA;
  k_set_one<<<1, 1, 0, st>>>(alpha_dev);
  if (Ns > 0 && Nt > 0) {
    dim3 gpt((unsigned)((Ns + kTile - 1) / kTile), (unsigned)((Nt + kTile - 1) / kTile));
    k_pairs_pt<1><<<gpt, kTile, 0, st>>>((int)Ns, (int)Nt, s_dev, ds_dev, tris_dev, dhat, 0.0, keys,
                                         counters, kNoallocCandidates, nullptr);
  }
  if (Ne > 1) {
    const unsigned ne = (unsigned)((Ne + kTile - 1) / kTile);
    k_pairs_ee<1><<<dim3(ne, ne), kTile, 0, st>>>((int)Ne, s_dev, ds_dev, edges_dev, dhat, 0.0, keys,
                                                  counters, kNoallocCandidates, nullptr);
  }
  k_accd_count<<<256, 128, 0, st>>>(counters, kNoallocCandidates, keys, s_dev, ds_dev, tris_dev,
                                    edges_dev, ccd_s, accd_max_iters, alpha_dev);
  if (cudaGetLastError() != cudaSuccess) return FSIM_ECUDA;
  int host_counters[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(host_counters, counters, sizeof(host_counters), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FSIM_ECUDA;
  return host_counters[2] ? FSIM_ECONTACT_OVERFLOW : FSIM_OK;
}
