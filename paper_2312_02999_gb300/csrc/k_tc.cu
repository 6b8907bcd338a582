// Tensor-core product of the batched global step: u = Sigma^-1 y2 for every
// frame's three right-hand sides at once (Eq. 9's explicit Sigma^-1 applied to
// the lower block step's y2, Sec. 3.2).  Sigma^-1 is dense (n2 x n2) and the
// right-hand sides of a batch form an n2 x nr block, so the product is a
// plain dense contraction: it runs on the 5th-generation tensor cores
// (tcgen05.mma, kind::tf32) with the accumulator in tensor memory and the
// Sigma^-1 tiles brought in by TMA.
//
// Precision: TF32 keeps 11 significant bits, too few for a solve whose
// float32 form is refined only in the reduced system.  Each operand is split
// into a TF32 head and a TF32 tail, a = a_hi + a_lo (a_hi = a with its low 13
// mantissa bits cleared, a_lo = the same of a - a_hi), and the product takes
// three MMAs, a_hi b_hi + a_hi b_lo + a_lo b_hi, which carries about 22
// significant bits (the dropped a_lo b_lo term is below 2^-22 of |a||b|).
// Sigma^-1 is constant, so its split is made once at prefactor time.
//
// One CTA computes a 128-row tile of u over a range of k (split-K); the tiles
// of a row range add their partial sums into u with vector atomics, so u is
// zeroed first.  Per 32-wide k step: TMA loads the Sigma^-1 head and tail
// tiles (128 x 32 float, 128-byte swizzle), the 128 threads load y2's rows
// k .. k+31 for all nr columns, split them and store them K-major in the same
// swizzled layout, one elected thread issues 3 x 4 MMAs (M = 128, N = nr,
// K = 8 each) and commits them to an mbarrier.  Two stages alternate.  Every
// wait is bounded: a wait that runs out sets the error word and the CTA
// still frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace fsim {

namespace {

constexpr int kTcM = 128;                  // rows of a tile (TMEM lanes)
constexpr int kTcK = 32;                   // k per stage (128 bytes of float)
constexpr int kTcThreads = 128;
constexpr int kTcMaxN = 192;               // widest multi-RHS buffer (64 frames)
constexpr uint32_t kTcTileA = kTcM * kTcK * 4;          // 16 KB
constexpr uint32_t kTcTileB = kTcMaxN * kTcK * 4;       // 24 KB
constexpr uint32_t kTcStage = 2 * kTcTileA + 2 * kTcTileB;   // hi/lo of A and B
constexpr uint32_t kTcSmem = 2 * kTcStage + 1024;       // two stages + alignment
constexpr long long kTcSpin = 1ll << 24;   // bound on every mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_head(float a) {
  return __uint_as_float(__float_as_uint(a) & 0xffffe000u);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// true when the phase with the given parity has completed, within the bound
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kTcSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes in groups of 8 (1024 bytes apart); the start address advances by 32
// bytes per 8-wide k step inside the swizzled row
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3fffu);           // start address
  d |= (uint64_t)1 << 16;                           // leading offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride offset: 8 rows
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::tf32, F32 accumulator, A and B K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4)                      // D format F32
         | (2u << 7) | (2u << 10)       // A, B format TF32
         | ((uint32_t)(n >> 3) << 17)   // N / 8
         | ((uint32_t)(m >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

}  // namespace

// u[i][c] += sum_k Sigma^-1[i][k] y2[k][c] over this CTA's rows
// [128 blockIdx.x, +128) and k stages [sps blockIdx.y, +sps); y2 and u are
// row-major with row stride nr (the multi-right-hand-side layout)
__global__ void __launch_bounds__(kTcThreads)
k_sinv_tc(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
          int n2, const float* __restrict__ Y, int nr, float* __restrict__ U, int sps,
          uint32_t tmem_cols, int* __restrict__ err) {
  extern __shared__ uint8_t tc_raw[];
  __shared__ __align__(8) uint64_t bars[4];          // TMA done x2, MMA done x2
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int m0 = blockIdx.x * kTcM;
  const int nstage_all = (n2 + kTcK - 1) / kTcK;
  const int s0 = blockIdx.y * sps, s1 = min(nstage_all, s0 + sps);
  const uint32_t tma_bar[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};
  const uint32_t mma_bar[2] = {smem_u32(&bars[2]), smem_u32(&bars[3])};
  if (tid == 0) {
    mbar_init(tma_bar[0], 1); mbar_init(tma_bar[1], 1);
    mbar_init(mma_bar[0], 1); mbar_init(mma_bar[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)), "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t dtmem = tmem_base;
  const uint32_t idesc = idesc_tf32(kTcM, nr);
  int issued = 0;                                    // stages whose MMAs were issued
  for (int s = s0; s < s1; ++s) {
    const int j = s - s0, slot = j & 1;
    uint8_t* st = smem + slot * kTcStage;
    const uint32_t a_hi = smem_u32(st), a_lo = a_hi + kTcTileA;
    const uint32_t b_hi = a_lo + kTcTileA, b_lo = b_hi + kTcTileB;
    if (j >= 2) {                                    // the slot's previous MMAs are done
      if (!mbar_wait(mma_bar[slot], ((j - 2) >> 1) & 1)) abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag) break;
    const int k0 = s * kTcK;
    if (tid == 0) {
      mbar_expect_tx(tma_bar[slot], 2 * kTcTileA);
      tma_load_2d(a_hi, &tm_hi, k0, m0, tma_bar[slot]);
      tma_load_2d(a_lo, &tm_lo, k0, m0, tma_bar[slot]);
    }
    // y2 rows k0 .. k0+31, all nr columns: head and tail, K-major, swizzled
    const int tot = kTcK * nr;
    for (int e = tid; e < tot; e += kTcThreads) {
      const int kk = e / nr, n = e - kk * nr, k = k0 + kk;
      const float v = k < n2 ? Y[(size_t)k * nr + n] : 0.f;
      const float h = tf32_head(v), l = tf32_head(v - h);
      const uint32_t off = (uint32_t)n * 128u + ((uint32_t)((kk >> 2) ^ (n & 7)) << 4) +
                           (uint32_t)(kk & 3) * 4u;
      *reinterpret_cast<float*>(st + 2 * kTcTileA + off) = h;
      *reinterpret_cast<float*>(st + 2 * kTcTileA + kTcTileB + off) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(tma_bar[slot], (j >> 1) & 1)) {
        abort_flag = 1;
        mbar_wait(tma_bar[slot], (j >> 1) & 1);      // once more for the copies in flight
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int q = 0; q < kTcK / 8; ++q) {
          const uint32_t dk = q * 32;                 // 8 floats = 32 bytes along k
          const uint32_t acc0 = (j > 0 || q > 0) ? 1u : 0u;
          mma_tf32(dtmem, sdesc(a_hi + dk), sdesc(b_hi + dk), idesc, acc0);
          mma_tf32(dtmem, sdesc(a_hi + dk), sdesc(b_lo + dk), idesc, 1u);
          mma_tf32(dtmem, sdesc(a_lo + dk), sdesc(b_hi + dk), idesc, 1u);
        }
        mma_commit(mma_bar[slot]);
      }
    }
    __syncthreads();
    if (abort_flag) break;
    issued = j + 1;
  }
  // the last issued stage's commit covers every MMA of this thread before it
  bool ok = !abort_flag;
  if (issued > 0) {
    const int jl = issued - 1;
    if (!mbar_wait(mma_bar[jl & 1], (jl >> 1) & 1)) ok = false;
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && issued > 0) {
    const int row = m0 + 32 * wid + lane;
    for (int c0 = 0; c0 < nr; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = dtmem + ((uint32_t)(32 * wid) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
          "%28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < n2) {
        float4* dst = reinterpret_cast<float4*>(U + (size_t)row * nr + c0);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          atomicAdd(dst + q, make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                         __uint_as_float(r[4 * q + 2]),
                                         __uint_as_float(r[4 * q + 3])));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtmem),
                 "r"(tmem_cols)
                 : "memory");
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

void tc_split_sinv(const double* sinv, int n2, std::vector<float>& hi, std::vector<float>& lo,
                   int* ld_out) {
  const int ld = (n2 + 31) / 32 * 32;
  hi.assign((size_t)ld * n2, 0.f);
  lo.assign((size_t)ld * n2, 0.f);
  auto head = [](float a) {
    uint32_t u;
    std::memcpy(&u, &a, 4);
    u &= 0xffffe000u;
    std::memcpy(&a, &u, 4);
    return a;
  };
  for (int i = 0; i < n2; ++i)
    for (int k = 0; k < n2; ++k) {
      const float a = (float)sinv[(size_t)i * n2 + k];
      const float h = head(a);
      hi[(size_t)i * ld + k] = h;
      lo[(size_t)i * ld + k] = head(a - h);
    }
  *ld_out = ld;
}

int tc_encode_sinv(const float* d_hi, const float* d_lo, int n2, int ld, void* maps) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return -1;
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n2};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM};
  const cuuint32_t estr[2] = {1, 1};
  CUtensorMap* tm = static_cast<CUtensorMap*>(maps);
  const float* src[2] = {d_hi, d_lo};
  for (int q = 0; q < 2; ++q)
    if (fn(&tm[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)src[q], dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return -1;
  return 0;
}

size_t tc_map_bytes() { return 2 * sizeof(CUtensorMap); }

void tc_set_smem_limits() {
  cudaFuncSetAttribute(k_sinv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
}

bool tc_sinv_supported(const DevMesh& m, int nr) {
  return m.tc_maps != nullptr && nr >= 32 && nr <= kTcMaxN && nr % 32 == 0 && m.n2 > 0;
}

cudaError_t launch_sinv_tc(cudaStream_t s, const DevMesh& m, const float* Y, int nr, float* U,
                           int num_sms, int* err) {
  const int n2 = m.n2;
  cudaError_t e = cudaMemsetAsync(U, 0, sizeof(float) * (size_t)n2 * nr, s);
  if (e != cudaSuccess) return e;
  const int mt = (n2 + kTcM - 1) / kTcM;
  const int nst = (n2 + kTcK - 1) / kTcK;
  int splits = std::max(1, std::min(nst, (num_sms + mt - 1) / mt));
  const int sps = (nst + splits - 1) / splits;
  splits = (nst + sps - 1) / sps;
  uint32_t cols = 32;
  while ((int)cols < nr) cols <<= 1;
  CUtensorMap tm[2];
  std::memcpy(tm, m.tc_maps, sizeof(tm));
  k_sinv_tc<<<dim3(mt, splits), kTcThreads, kTcSmem, s>>>(tm[0], tm[1], n2, Y, nr, U, sps, cols,
                                                          err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fsim
