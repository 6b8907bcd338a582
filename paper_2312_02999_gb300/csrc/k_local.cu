// Local step of Algorithm 1 (GetProjection, Eq. 1 and Sec. 2.1) fused with
// the elastic energy and the per-tet elastic forces of Eq. 4.
//
// Per tet i: F = Ds Dm^-1, M = F A (A symmetric), R = polar rotation of M,
// p = vec(R A), D = F - R A, energy 1/2 w |D|_F^2 and the gradient
// contribution w D gradN_a of each of its four vertices (the row form of
// w_i G_i^T (G_i x - p_i)).  Forces are written per tet and gathered per
// vertex in a fixed order (deterministic sums, no atomics).
#include <nvtx3/nvToolsExt.h>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "df64.cuh"
#include "mat3.cuh"

namespace fsim {

namespace {
std::atomic<std::int64_t> g_launches{0};
// ProfScope may be used from several host threads (server workers)
std::mutex g_prof_mu;

// event-pair pool for ProfScope; resolved (summed per class) in prof_read
struct Prof {
  unsigned mask = 0;
  std::vector<cudaEvent_t> ev0, ev1;
  std::vector<int> cls;
  std::vector<int> free_slots, pending;
  int64_t launches[PROF_NCLASS] = {0};
  double ms[PROF_NCLASS] = {0};
} g_prof;

void prof_resolve() {
  for (int slot : g_prof.pending) {
    cudaEventSynchronize(g_prof.ev1[slot]);
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g_prof.ev0[slot], g_prof.ev1[slot]) == cudaSuccess) {
      g_prof.ms[g_prof.cls[slot]] += t;
      g_prof.launches[g_prof.cls[slot]] += 1;
    }
    g_prof.free_slots.push_back(slot);
  }
  g_prof.pending.clear();
}
}  // namespace

thread_local bool tl_capturing = false;
int64_t launch_counter() { return g_launches.load(); }
void count_launch(int k) {
  if (!tl_capturing) g_launches += k;
}
void set_capturing(bool on) { tl_capturing = on; }

// NVTX range names of the stage classes (a tool such as Nsight Systems shows
// them; without one attached a push/pop is a null check)
static const char* const kProfNames[PROF_NCLASS] = {
    "fsim.local_step", "fsim.constraint_set", "fsim.trisolve_fwd", "fsim.trisolve_bwd",
    "fsim.reduced_factor", "fsim.barrier", "fsim.ccd", "fsim.sigma_product", "fsim.reduced_system",
    "fsim.pcg", "fsim.schur"};

ProfScope::ProfScope(int c, cudaStream_t s) : slot(-1), stream(s) {
  nvtxRangePushA(c >= 0 && c < PROF_NCLASS ? kProfNames[c] : "fsim");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!(g_prof.mask & (1u << c))) return;
  if (g_prof.pending.size() >= 4096) prof_resolve();
  if (g_prof.free_slots.empty()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
    g_prof.ev0.push_back(a); g_prof.ev1.push_back(b); g_prof.cls.push_back(c);
    g_prof.free_slots.push_back((int)g_prof.ev0.size() - 1);
  }
  slot = g_prof.free_slots.back();
  g_prof.free_slots.pop_back();
  g_prof.cls[slot] = c;
  cudaEventRecord(g_prof.ev0[slot], s);
}

FSIM_CHECK_READER(check_word_local)

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

ProfScope::~ProfScope() {
  nvtxRangePop();
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_prof.ev1[slot], stream);
  g_prof.pending.push_back(slot);
}

void prof_set_mask(unsigned mask) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.mask = mask;
}

bool prof_active() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_prof.mask != 0;
}

int prof_read(int c, int64_t* launches, double* total_ms) {
  if (c < 0 || c >= PROF_NCLASS) return -1;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_resolve();
  *launches = g_prof.launches[c];
  *total_ms = g_prof.ms[c];
  return 0;
}

void prof_reset() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_resolve();
  for (int c = 0; c < PROF_NCLASS; ++c) { g_prof.launches[c] = 0; g_prof.ms[c] = 0.0; }
}

constexpr int kElasticThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  __syncthreads();
  return v;   // valid in thread 0
}

__global__ void k_actuation(int T, const double* __restrict__ fiber,
                            const double* __restrict__ stretch, double* __restrict__ act,
                            float2* __restrict__ act_df) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double f0 = fiber[3 * t], f1 = fiber[3 * t + 1], f2 = fiber[3 * t + 2];
  const double nn = sqrt(f0 * f0 + f1 * f1 + f2 * f2);
  f0 /= nn; f1 /= nn; f2 /= nn;
  const double a = stretch[t];
  const double b = 1.0 / sqrt(a);          // transverse stretch a^(-1/2)
  const double k = a - b;
  act[0 * T + t] = b + k * f0 * f0;
  act[1 * T + t] = k * f0 * f1;
  act[2 * T + t] = k * f0 * f2;
  act[3 * T + t] = b + k * f1 * f1;
  act[4 * T + t] = k * f1 * f2;
  act[5 * T + t] = b + k * f2 * f2;
  if (act_df) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double v = act[c * T + t];
      const float h = __double2float_rn(v);
      act_df[(size_t)c * T + t] = make_float2(h, __double2float_rn(v - (double)h));
    }
  }
}

template <int PREC>
__global__ void __launch_bounds__(kElasticThreads)
k_elastic(int T, const int4* __restrict__ tets, const double* __restrict__ dminv,
          const double* __restrict__ w, const double* __restrict__ act,
          const double* __restrict__ x, double* __restrict__ tetf,
          double* __restrict__ proj, double* __restrict__ partials) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (t < T) {
    const int4 tv = tets[t];
    const double* x0 = x + 3 * (size_t)tv.x;
    const double* x1 = x + 3 * (size_t)tv.y;
    const double* x2 = x + 3 * (size_t)tv.z;
    const double* x3 = x + 3 * (size_t)tv.w;
    double Ds[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double o = x0[d];
      Ds[d][0] = x1[d] - o;
      Ds[d][1] = x2[d] - o;
      Ds[d][2] = x3[d] - o;
    }
    double Di[3][3];
#pragma unroll
    for (int k = 0; k < 9; ++k) Di[k / 3][k % 3] = dminv[(size_t)k * T + t];
    double F[3][3];
    matmul(Ds, Di, F);
    double A[3][3];
    A[0][0] = act[0 * (size_t)T + t];
    A[0][1] = A[1][0] = act[1 * (size_t)T + t];
    A[0][2] = A[2][0] = act[2 * (size_t)T + t];
    A[1][1] = act[3 * (size_t)T + t];
    A[1][2] = A[2][1] = act[4 * (size_t)T + t];
    A[2][2] = act[5 * (size_t)T + t];
    double M[3][3], R[3][3];
    matmul(F, A, M);
    if (PREC == 0) {
      polar_rotation<double, 10>(M, R);
    } else {
      float Mf[3][3], Rf[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Mf[i][j] = (float)M[i][j];
      polar_rotation<float, 6>(Mf, Rf);
      double R0[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) R0[i][j] = (double)Rf[i][j];
      polar_refine(M, R0, R);
    }
    double P[3][3];
    matmul(R, A, P);
    const double wt = w[t];
    double Dd[3][3];
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Dd[i][j] = F[i][j] - P[i][j];
        s += Dd[i][j] * Dd[i][j];
      }
    e = 0.5 * wt * s;
    // f_a = w D gradN_a, gradN_a = row a-1 of Dm^-1 (a = 1..3), f_0 = -sum
    double f0[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double fa = wt * (Dd[d][0] * Di[a - 1][0] + Dd[d][1] * Di[a - 1][1] + Dd[d][2] * Di[a - 1][2]);
        tetf[(size_t)(a * 3 + d) * T + t] = fa;
        f0[d] -= fa;
      }
#pragma unroll
    for (int d = 0; d < 3; ++d) tetf[(size_t)d * T + t] = f0[d];
    if (proj != nullptr) {
#pragma unroll
      for (int k = 0; k < 9; ++k) proj[(size_t)9 * t + k] = P[k / 3][k % 3];
    }
  }
  const double bs = block_sum(e);
  if (threadIdx.x == 0) partials[blockIdx.x] = bs;
}

// Mixed-precision local step in double-float arithmetic (df64.cuh), with
// no float64 instruction per tet: GB300 issues float64 (and float64
// conversions) at about 1/64 of the float32 rate, so the float64 loads,
// differences, conversions and products of a per-tet float64 interface cost
// more than the whole float32 SVD.  The kernel reads the vertex
// displacements u = x - X as float pairs (k_disp_df, once per vertex), Dm^-1,
// A and w as float pairs, and works with the displacement gradient:
//   F = Ds Dm^-1 = I + Du Dm^-1,  Du = [u1 - u0, u2 - u0, u3 - u0],
// which keeps F - I (the strain) to double-float accuracy relative to itself.
// Then M = F A, a float32 rotation R0 of M (Jacobi SVD) refined to float64
// accuracy as in polar_refine but with the small terms in float32:
// R1 = R0 + R0 D with D = (I - R0^T R0) / 2 (about 1e-7), the skew part of
// S = R1^T M kept in double-float, w = ((tr S) I - S)^-1 2 a in float32, and
// R = R1 exp([w]) = R0 + C with C = R0 D + R0 (E - I) + R0 D (E - I) (all
// about 1e-7, so float32 products suffice); p = R A, D = F - p, the energy
// 1/2 w |D|^2 and the forces w D gradN_a.  Forces are written as float
// pairs (tetf reinterpreted, the same 8 bytes per entry as float64) and
// summed per vertex by k_gather_forces_df; the energy is summed per block in
// double-float and converted once per block.  Sums of products use Dekker's
// addition (df_add_fast); the strain D = F - p, where F and p agree to a few
// digits, uses the full df_add.
__device__ __forceinline__ void disp_df_body(int n3, const double* __restrict__ x,
                                             const double* __restrict__ rest,
                                             float2* __restrict__ udf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const df u = df_from_double(__dsub_rn(x[i], rest[i]));
  udf[i] = make_float2(u.hi, u.lo);
}
__global__ void k_disp_df(int n3, const double* __restrict__ x, const double* __restrict__ rest,
                          float2* __restrict__ udf) {
  disp_df_body(n3, x, rest, udf);
}

__device__ __forceinline__ df ld_df(const float2* __restrict__ p, size_t i) {
  const float2 v = p[i];
  return {v.x, v.y};
}

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, w);
  }
  return v;
}

__device__ __forceinline__ void elastic_df_body(int T, const int4* __restrict__ tets,
                                                const float2* __restrict__ dminv_df,
                                                const float2* __restrict__ w_df,
                                                const float2* __restrict__ act_df,
                                                const float2* __restrict__ udf,
                                                float2* __restrict__ tetf,
                                                double* __restrict__ proj,
                                                double* __restrict__ partials) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  df e = {0.f, 0.f};
  if (t < T) {
    const int4 tv = tets[t];
    df u0[3], Du[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) u0[d] = ld_df(udf, 3 * (size_t)tv.x + d);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Du[d][0] = df_sub_fast(ld_df(udf, 3 * (size_t)tv.y + d), u0[d]);
      Du[d][1] = df_sub_fast(ld_df(udf, 3 * (size_t)tv.z + d), u0[d]);
      Du[d][2] = df_sub_fast(ld_df(udf, 3 * (size_t)tv.w + d), u0[d]);
    }
    df Di[3][3];
#pragma unroll
    for (int k = 0; k < 9; ++k) Di[k / 3][k % 3] = ld_df(dminv_df, (size_t)k * T + t);
    df A[3][3];
    A[0][0] = ld_df(act_df, 0 * (size_t)T + t);
    A[0][1] = A[1][0] = ld_df(act_df, 1 * (size_t)T + t);
    A[0][2] = A[2][0] = ld_df(act_df, 2 * (size_t)T + t);
    A[1][1] = ld_df(act_df, 3 * (size_t)T + t);
    A[1][2] = A[2][1] = ld_df(act_df, 4 * (size_t)T + t);
    A[2][2] = ld_df(act_df, 5 * (size_t)T + t);
    df F[3][3], M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        F[i][j] = df_dot3(Du[i][0], Di[0][j], Du[i][1], Di[1][j], Du[i][2], Di[2][j]);
        if (i == j) F[i][j] = df_add_fast(F[i][j], df_from_float(1.f));
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        M[i][j] = df_dot3(F[i][0], A[0][j], F[i][1], A[1][j], F[i][2], A[2][j]);
    float R0[3][3];
    {
      float Mf[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Mf[i][j] = M[i][j].hi;
      polar_rotation<float, 6>(Mf, R0);
    }
    // D = (I - R0^T R0) / 2 from exact float products summed in double-float
    float Dm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const df g = df_dot3_ff(R0[0][i], R0[0][j], R0[1][i], R0[1][j], R0[2][i], R0[2][j]);
        // (1 - g.hi) is exact for g.hi near 1 (and 0 - g.hi always)
        Dm[i][j] = Dm[j][i] = 0.5f * ((i == j ? 1.f - g.hi : -g.hi) - g.lo);
      }
    float R1c[3][3];
    matmul(R0, Dm, R1c);
    // S = R1^T M = R0^T M (double-float) + R1c^T M (float)
    df S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        df acc = df_dot3_f(M[0][j], R0[0][i], M[1][j], R0[1][i], M[2][j], R0[2][i]);
        const float c = R1c[0][i] * M[0][j].hi + R1c[1][i] * M[1][j].hi + R1c[2][i] * M[2][j].hi;
        // c is a correction of relative size ~1e-7: it joins the low part
        S[i][j] = df_fast_two_sum(acc.hi, __fadd_rn(acc.lo, c));
      }
    float wv0 = 0.f, wv1 = 0.f, wv2 = 0.f;
    {
      const df d0 = df_sub(S[2][1], S[1][2]), d1 = df_sub(S[0][2], S[2][0]), d2 = df_sub(S[1][0], S[0][1]);
      const float a0 = 0.5f * (d0.hi + d0.lo), a1 = 0.5f * (d1.hi + d1.lo), a2 = 0.5f * (d2.hi + d2.lo);
      const float s00 = S[0][0].hi, s11 = S[1][1].hi, s22 = S[2][2].hi;
      const float s01 = 0.5f * (S[0][1].hi + S[1][0].hi);
      const float s02 = 0.5f * (S[0][2].hi + S[2][0].hi);
      const float s12 = 0.5f * (S[1][2].hi + S[2][1].hi);
      const float tr = s00 + s11 + s22;
      const float A00 = tr - s00, A11 = tr - s11, A22 = tr - s22;
      const float A01 = -s01, A02 = -s02, A12 = -s12;
      const float c00 = A11 * A22 - A12 * A12, c01 = A02 * A12 - A01 * A22, c02 = A01 * A12 - A02 * A11;
      const float c11 = A00 * A22 - A02 * A02, c12 = A01 * A02 - A00 * A12, c22 = A00 * A11 - A01 * A01;
      const float det = A00 * c00 + A01 * c01 + A02 * c02;
      if (fabsf(det) > 1e-30f) {
        const float id = 2.f / det;
        wv0 = id * (c00 * a0 + c01 * a1 + c02 * a2);
        wv1 = id * (c01 * a0 + c11 * a1 + c12 * a2);
        wv2 = id * (c02 * a0 + c12 * a1 + c22 * a2);
      }
    }
    // E - I for exp([w]) to second order
    float Em[3][3];
    Em[0][0] = -0.5f * (wv1 * wv1 + wv2 * wv2);
    Em[1][1] = -0.5f * (wv0 * wv0 + wv2 * wv2);
    Em[2][2] = -0.5f * (wv0 * wv0 + wv1 * wv1);
    Em[0][1] = -wv2 + 0.5f * wv0 * wv1;
    Em[1][0] = wv2 + 0.5f * wv0 * wv1;
    Em[0][2] = wv1 + 0.5f * wv0 * wv2;
    Em[2][0] = -wv1 + 0.5f * wv0 * wv2;
    Em[1][2] = -wv0 + 0.5f * wv1 * wv2;
    Em[2][1] = wv0 + 0.5f * wv1 * wv2;
    // R = (R0 + R1c)(I + Em) = R0 + C
    df R[3][3];
    {
      float T1[3][3], T2[3][3];
      matmul(R0, Em, T1);
      matmul(R1c, Em, T2);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) R[i][j] = df_two_sum(R0[i][j], R1c[i][j] + T1[i][j] + T2[i][j]);
    }
    df P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        P[i][j] = df_dot3(R[i][0], A[0][j], R[i][1], A[1][j], R[i][2], A[2][j]);
    const df wt = ld_df(w_df, t);
    df Dd[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Dd[i][j] = df_sub_fast(F[i][j], P[i][j]);
    // |D|^2 by rows (terms of one sign)
    const df ssum = df_sum3(df_dot3(Dd[0][0], Dd[0][0], Dd[0][1], Dd[0][1], Dd[0][2], Dd[0][2]),
                            df_dot3(Dd[1][0], Dd[1][0], Dd[1][1], Dd[1][1], Dd[1][2], Dd[1][2]),
                            df_dot3(Dd[2][0], Dd[2][0], Dd[2][1], Dd[2][1], Dd[2][2], Dd[2][2]));
    e = df_mul(wt, ssum);
    e.hi *= 0.5f;
    e.lo *= 0.5f;
    // f_a = w D gradN_a, gradN_a = row a-1 of Dm^-1 (a = 1..3), f_0 = -sum
    df fa[3][3];
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const df q = df_dot3(Dd[d][0], Di[a - 1][0], Dd[d][1], Di[a - 1][1], Dd[d][2], Di[a - 1][2]);
        fa[a - 1][d] = df_mul(wt, q);
        tetf[(size_t)(a * 3 + d) * T + t] = make_float2(fa[a - 1][d].hi, fa[a - 1][d].lo);
      }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const df f0 = df_neg(df_sum3(fa[0][d], fa[1][d], fa[2][d]));
      tetf[(size_t)d * T + t] = make_float2(f0.hi, f0.lo);
    }
    if (proj != nullptr) {
#pragma unroll
      for (int k = 0; k < 9; ++k) proj[(size_t)9 * t + k] = df_to_double(P[k / 3][k % 3]);
    }
  }
  // energy: double-float block sum, one float64 conversion per block
  __shared__ df red[kElasticThreads / 32];
  e = warp_sum_df(e);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = e;
  __syncthreads();
  if (wid == 0) {
    df v = lane < kElasticThreads / 32 ? red[lane] : df{0.f, 0.f};
    v = warp_sum_df(v);
    if (lane == 0) partials[blockIdx.x] = df_to_double(v);
  }
}

__global__ void __launch_bounds__(kElasticThreads)
k_elastic_df(int T, const int4* __restrict__ tets, const float2* __restrict__ dminv_df,
             const float2* __restrict__ w_df, const float2* __restrict__ act_df,
             const float2* __restrict__ udf, float2* __restrict__ tetf,
             double* __restrict__ proj, double* __restrict__ partials) {
  elastic_df_body(T, tets, dminv_df, w_df, act_df, udf, tetf, proj, partials);
}

// Per-vertex sum of the double-float per-tet forces (fixed order), one
// float64 conversion per coordinate.
__device__ __forceinline__ void gather_forces_df_body(int n, int T, const int* __restrict__ vptr,
                                                      const int* __restrict__ vslot,
                                                      const float2* __restrict__ tetf,
                                                      const uint8_t* __restrict__ pinned,
                                                      double* __restrict__ g) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  df s0 = {0.f, 0.f}, s1 = {0.f, 0.f}, s2 = {0.f, 0.f};
  if (!pinned[v]) {
    // four slots per step: their index and force loads are all in flight
    // before the (exact-cancellation safe) double-float sums use them
    const int e0 = vptr[v], e1 = vptr[v + 1];
    for (int e = e0; e < e1; e += 4) {
      int slot[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) slot[q] = e + q < e1 ? vslot[e + q] : -1;
      df f[4][3];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = slot[q] >> 2, a = slot[q] & 3;
        const bool ok = slot[q] >= 0 && FSIM_CHECK_IDX(t, T, CHECK_GATHER_TET);
#pragma unroll
        for (int d = 0; d < 3; ++d)
          f[q][d] = ok ? ld_df(tetf, (size_t)(a * 3 + d) * T + t) : df{0.f, 0.f};
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (slot[q] < 0) break;
        s0 = df_add(s0, f[q][0]);
        s1 = df_add(s1, f[q][1]);
        s2 = df_add(s2, f[q][2]);
      }
    }
  }
  g[3 * (size_t)v + 0] = df_to_double(s0);
  g[3 * (size_t)v + 1] = df_to_double(s1);
  g[3 * (size_t)v + 2] = df_to_double(s2);
}
__global__ void k_gather_forces_df(int n, int T, const int* __restrict__ vptr,
                                   const int* __restrict__ vslot, const float2* __restrict__ tetf,
                                   const uint8_t* __restrict__ pinned, double* __restrict__ g) {
  gather_forces_df_body(n, T, vptr, vslot, tetf, pinned, g);
}

__global__ void k_gather_forces(int n, int T, const int* __restrict__ vptr,
                                const int* __restrict__ vslot, const double* __restrict__ tetf,
                                const uint8_t* __restrict__ pinned, double* __restrict__ g) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (!pinned[v]) {
    for (int e = vptr[v]; e < vptr[v + 1]; ++e) {
      const int slot = vslot[e];
      const int t = slot >> 2, a = slot & 3;
      if (!FSIM_CHECK_IDX(t, T, CHECK_GATHER_TET)) continue;
      s0 += tetf[(size_t)(a * 3 + 0) * T + t];
      s1 += tetf[(size_t)(a * 3 + 1) * T + t];
      s2 += tetf[(size_t)(a * 3 + 2) * T + t];
    }
  }
  g[3 * (size_t)v + 0] = s0;
  g[3 * (size_t)v + 1] = s1;
  g[3 * (size_t)v + 2] = s2;
}

// Fixed-order sum of n partials by one block (deterministic).
__device__ __forceinline__ void sum_partials_body(const double* __restrict__ p, int n,
                                                  double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}
__global__ void k_sum_partials(const double* __restrict__ p, int n, double* __restrict__ out) {
  sum_partials_body(p, n, out);
}

__global__ void k_axpy(int n3, const double* __restrict__ x, const double* __restrict__ dx,
                       const double* __restrict__ alpha, double scale, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const double a = alpha[0] * scale;
  out[i] = x[i] + a * dx[i];
}

__device__ __forceinline__ void gnorm2_body(int n, const double* __restrict__ g,
                                            const uint8_t* __restrict__ pinned,
                                            double* __restrict__ partials) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (v < n && !pinned[v]) {
    const double a = g[3 * (size_t)v], b = g[3 * (size_t)v + 1], c = g[3 * (size_t)v + 2];
    s = a * a + b * b + c * c;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}
__global__ void k_gnorm2(int n, const double* __restrict__ g, const uint8_t* __restrict__ pinned,
                         double* __restrict__ partials) {
  gnorm2_body(n, g, pinned, partials);
}

// ---- lock-step batches: one launch for the frames of a batch table ----------
// blockIdx.y selects the frame; a frame whose `active` flag is clear returns
// at once (uniformly for its blocks).  AT selects the evaluation point: 0 =
// the iterate (x, tetf), 1 = the line-search trial (xt, tetf_t).
__device__ __forceinline__ const DevMesh* bframe(const DevMesh* __restrict__ tab) {
  const DevMesh* m = tab + blockIdx.y;
  return m->active ? m : nullptr;
}

template <int AT>
__global__ void k_disp_df_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe(tab);
  if (!m) return;
  disp_df_body(3 * m->n, AT ? m->xt : m->x, m->rest, m->udf);
}

template <int AT>
__global__ void __launch_bounds__(kElasticThreads) k_elastic_df_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe(tab);
  if (!m) return;
  elastic_df_body(m->T, m->tets, m->dminv_df, m->w_df, m->act_df, m->udf,
                  reinterpret_cast<float2*>(AT ? m->tetf_t : m->tetf), nullptr, m->partials);
}

// out = scal[which] of each frame: the fixed-order sum of its nparts partials
__global__ void k_sum_partials_b(const DevMesh* __restrict__ tab, int nparts, int which) {
  const DevMesh* m = bframe(tab);
  if (!m) return;
  sum_partials_body(m->partials, nparts, m->scal + which);
}

__global__ void k_gather_forces_df_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe(tab);
  if (!m) return;
  gather_forces_df_body(m->n, m->T, m->vinc_ptr, m->vinc_slot,
                        reinterpret_cast<const float2*>(m->tetf), m->pinned, m->g);
}

// xt = x + (alpha_m * ls_scale) dx per frame
__global__ void k_axpy_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe(tab);
  if (!m) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * m->n) return;
  const double a = m->scal[1] * m->ls_scale;
  m->xt[i] = m->x[i] + a * m->dx[i];
}

__global__ void k_gnorm2_b(const DevMesh* __restrict__ tab) {
  const DevMesh* m = bframe(tab);
  if (!m) return;
  gnorm2_body(m->n, m->g, m->pinned, m->partials);
}

__global__ void k_reset_pinned(int n, const uint8_t* __restrict__ pinned,
                               const double* __restrict__ rest, double* __restrict__ x) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n || !pinned[v]) return;
  x[3 * (size_t)v] = rest[3 * (size_t)v];
  x[3 * (size_t)v + 1] = rest[3 * (size_t)v + 1];
  x[3 * (size_t)v + 2] = rest[3 * (size_t)v + 2];
}

__global__ void k_check_finite(int n, const double* __restrict__ v, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(v[i])) atomicOr(flag, 1);
}

// ---------------------------------------------------------------------------
void launch_actuation(cudaStream_t s, int T, const double* fiber, const double* stretch, double* act,
                      float2* act_df) {
  k_actuation<<<(T + 255) / 256, 256, 0, s>>>(T, fiber, stretch, act, act_df);
  count_launch();
}

int elastic_blocks(int T) { return (T + kElasticThreads - 1) / kElasticThreads; }

bool elastic_uses_df(const DevMesh& m, int precision) {
  return precision != 0 && m.dminv_df && m.act_df && m.w_df && m.udf;
}

void launch_elastic(cudaStream_t s, const DevMesh& m, const double* x, double* tetf,
                    double* proj, double* partials, int precision) {
  const int nb = elastic_blocks(m.T);
  ProfScope ps(PROF_ELASTIC, s);
  if (precision == 0) {
    k_elastic<0><<<nb, kElasticThreads, 0, s>>>(m.T, m.tets, m.dminv, m.w, m.act, x, tetf, proj, partials);
    count_launch();
  } else if (elastic_uses_df(m, precision)) {
    k_disp_df<<<(3 * m.n + 255) / 256, 256, 0, s>>>(3 * m.n, x, m.rest, m.udf);
    k_elastic_df<<<nb, kElasticThreads, 0, s>>>(m.T, m.tets, m.dminv_df, m.w_df, m.act_df, m.udf,
                                               reinterpret_cast<float2*>(tetf), proj, partials);
    count_launch(2);
  } else {
    k_elastic<1><<<nb, kElasticThreads, 0, s>>>(m.T, m.tets, m.dminv, m.w, m.act, x, tetf, proj, partials);
    count_launch();
  }
}

void launch_gather_forces(cudaStream_t s, const DevMesh& m, const double* tetf, double* g,
                          int precision) {
  if (elastic_uses_df(m, precision))
    k_gather_forces_df<<<(m.n + 255) / 256, 256, 0, s>>>(m.n, m.T, m.vinc_ptr, m.vinc_slot,
                                                         reinterpret_cast<const float2*>(tetf),
                                                         m.pinned, g);
  else
    k_gather_forces<<<(m.n + 255) / 256, 256, 0, s>>>(m.n, m.T, m.vinc_ptr, m.vinc_slot, tetf,
                                                      m.pinned, g);
  count_launch();
}

void launch_sum_partials(cudaStream_t s, const double* partials, int n, double* out) {
  k_sum_partials<<<1, 1024, 0, s>>>(partials, n, out);
  count_launch();
}

void launch_axpy_positions(cudaStream_t s, int n3, const double* x, const double* dx,
                           const double* alpha_dev, double alpha_scale, double* out) {
  k_axpy<<<(n3 + 255) / 256, 256, 0, s>>>(n3, x, dx, alpha_dev, alpha_scale, out);
  count_launch();
}

int gnorm_blocks(int n) { return (n + 255) / 256; }

void launch_local_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0, int at) {
  ProfScope ps(PROF_ELASTIC, s);
  const dim3 gv((3 * m0.n + 255) / 256, nb), gt(elastic_blocks(m0.T), nb);
  if (at) {
    k_disp_df_b<1><<<gv, 256, 0, s>>>(tab);
    k_elastic_df_b<1><<<gt, kElasticThreads, 0, s>>>(tab);
  } else {
    k_disp_df_b<0><<<gv, 256, 0, s>>>(tab);
    k_elastic_df_b<0><<<gt, kElasticThreads, 0, s>>>(tab);
  }
  k_sum_partials_b<<<dim3(1, nb), 1024, 0, s>>>(tab, elastic_blocks(m0.T), 2);
  count_launch(3);
}

void launch_gather_forces_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0) {
  k_gather_forces_df_b<<<dim3((m0.n + 255) / 256, nb), 256, 0, s>>>(tab);
  count_launch();
}

void launch_gnorm2_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0) {
  k_gnorm2_b<<<dim3(gnorm_blocks(m0.n), nb), 256, 0, s>>>(tab);
  k_sum_partials_b<<<dim3(1, nb), 1024, 0, s>>>(tab, gnorm_blocks(m0.n), 3);
  count_launch(2);
}

void launch_axpy_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0) {
  k_axpy_b<<<dim3((3 * m0.n + 255) / 256, nb), 256, 0, s>>>(tab);
  count_launch();
}

void launch_gnorm2(cudaStream_t s, const DevMesh& m, const double* g, double* partials, int nblk) {
  k_gnorm2<<<nblk, 256, 0, s>>>(m.n, g, m.pinned, partials);
  count_launch();
}

void launch_reset_pinned(cudaStream_t s, const DevMesh& m, double* x) {
  k_reset_pinned<<<(m.n + 255) / 256, 256, 0, s>>>(m.n, m.pinned, m.rest, x);
  count_launch();
}

void launch_check_finite(cudaStream_t s, int n, const double* v, int* flag) {
  if (n <= 0) return;
  k_check_finite<<<(n + 255) / 256, 256, 0, s>>>(n, v, flag);
  count_launch();
}

}  // namespace fsim
