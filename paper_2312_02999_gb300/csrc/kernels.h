// Device-side mesh state and the host-callable kernel launchers.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace fsim {

// All device pointers of one mesh (owned by the context, see capi.cu).
struct DevMesh {
  int n = 0, T = 0, Ns = 0, Nt = 0, Ne = 0;
  int nf = 0, n1 = 0, n2 = 0;
  // vertices (AoS xyz)
  double* rest = nullptr;
  double* x = nullptr;        // current iterate
  double* xt = nullptr;       // line-search trial
  double* dx = nullptr;       // search direction
  double* g = nullptr;        // gradient g-hat (by vertex)
  uint8_t* pinned = nullptr;
  // tets
  int4* tets = nullptr;
  double* dminv = nullptr;    // 9T SoA: Dm^-1 (row-major entry k at k*T + t)
  double* w = nullptr;        // T
  double* act = nullptr;      // 6T SoA: A00 A01 A02 A11 A12 A22
  float2* act_df = nullptr;   // 6T SoA: the same as float pairs (hi, lo)
  float2* dminv_df = nullptr; // 9T SoA: Dm^-1 as float pairs
  float2* w_df = nullptr;     // T: w as float pairs
  float2* udf = nullptr;      // 3n: displacement x - rest as float pairs (mixed local step)
  double* tetf = nullptr;     // 12T SoA per-tet vertex forces ((a*3+d)*T + t); float64, or
                              // float pairs in the same bytes after a mixed local step
  double* tetf_t = nullptr;   // same at the trial point
  int* vinc_ptr = nullptr;    // vertex -> incident (t*4 + a) slots
  int* vinc_slot = nullptr;
  // proxy
  int64_t* Wptr = nullptr;
  int* Wcol = nullptr;
  double* Wval = nullptr;
  int* tris = nullptr;        // 3 Nt
  int* edges = nullptr;       // 2 Ne (lo, hi), sorted unique
  double* s = nullptr;        // 3 Ns proxy positions at x
  double* st = nullptr;       // 3 Ns proxy positions at the trial point
  double* ds = nullptr;       // 3 Ns proxy step
  float* pbox = nullptr;      // 12 floats per primitive (verts, tris, edges)
  unsigned long long* pkey = nullptr;  // 12 order keys per primitive
  float* sf = nullptr;        // 3 Ns float32 proxy positions
  float* dsf = nullptr;       // 3 Ns float32 proxy step
  unsigned long long* nearl = nullptr;  // pairs within 2 dhat in float32 (cap)
  unsigned long long* vlist = nullptr;  // skin list: pairs within dhat + skin at sb (cap)
  double* cg_r = nullptr;     // CG work vectors (3n each) and 2 device scalars
  double* cg_z = nullptr;
  double* cg_p = nullptr;
  double* cg_q = nullptr;
  double* cg_tmp = nullptr;
  double* cg_red = nullptr;
  double* sb = nullptr;       // 3 Ns proxy positions of the last skin-list build
  double* elen2 = nullptr;    // Ne squared rest lengths of the proxy edges (EE mollifier)
  int ee_moll = 0;            // 1: edge-edge terms carry IPC's mollifier
  double skin = 0.0;          // skin width of the list (length)
  double coord_scale = 1.0;   // 2 x largest |rest coordinate|
  // solver ordering
  int* perm = nullptr;        // nf: position -> vertex
  int* pos = nullptr;         // n: vertex -> position or -1
  int* x2of = nullptr;        // n: vertex -> x2 index or -1
  // factor of K11
  int n_sn = 0, n_levels = 0, max_ns = 0, max_ld = 0;
  int* sn_c0 = nullptr; int* sn_ns = nullptr; int* sn_nr1 = nullptr;
  int64_t* sn_roff = nullptr; int64_t* sn_zoff = nullptr;
  int* sn_rows = nullptr;
  double* Z = nullptr;
  float* Zf = nullptr;
  int* level_sn = nullptr;    // supernodes grouped by level
  int* h_level_ptr = nullptr; // HOST array (n_levels + 1)
  int* h_level_maxns = nullptr;  // HOST: largest ns per level
  int* h_level_maxld = nullptr;  // HOST: largest ns + nr1 per level
  int4* fwd_items = nullptr;  // (J, first row, rows, 0) work items, grouped by level
  int4* bwd_items = nullptr;  // (J, first column, columns, 0)
  int* h_fwd_ptr = nullptr;   // HOST (n_levels + 1)
  int* h_bwd_ptr = nullptr;   // HOST (n_levels + 1)
  int4* bwd_items32 = nullptr;  // (J, first column, columns <= 32, first row) for the batched
                                // solve: rows [first row, + kBwdRowSplit) of Z_J
  int* h_bwd32_ptr = nullptr; // HOST (n_levels + 1)
  double* y1 = nullptr;       // n1*3 forward-solve scratch
  float* y1f = nullptr;
  double* Sinv = nullptr;     // n2 x n2 Schur-complement inverse (Sec. 3.2)
  int* kv_ptr = nullptr;      // K in vertex order (CSR over free vertices), for the CG operator
  int* kv_col = nullptr;
  double* kv_val = nullptr;
  float* Sinvf = nullptr;
  double* Sig = nullptr;      // n2 x n2 Sigma itself (the Schur-only global step)
  double* sh_A = nullptr;     // (3 n2)^2 Sigma-hat, float64 (Schur-only global step)
  float* sh_Af = nullptr;     // (3 n2)^2 Sigma-hat, float32 factor (mixed)
  double* sh_y = nullptr;     // 3 n2 refinement vectors
  double* sh_r = nullptr;
  float* sh_df = nullptr;
  // global-step work (solver positions, AoS 3)
  double* r = nullptr;        // nf*3
  double* u = nullptr;        // n2*3
  float* uf = nullptr;        // n2*3 (mixed)
  float* rf = nullptr;        // nf*3 (mixed)
  // contact work
  int64_t cap = 0;            // capacity of the near-pair and CCD candidate lists
  int64_t cap_act = 0;        // capacity of the constraint set C (pairs, per-pair derivatives)
  unsigned long long* pairs = nullptr;    // keys (type<<62 | i<<31 | j)
  unsigned long long* cand = nullptr;     // CCD candidates
  int* counters = nullptr;    // [0] pairs [1] cand [2] overflow [3] nc [4] nonfinite [5] touching
                              // [6..7] Cholesky info [8] near pairs [9] CCD overflow
                              // [10..14] skin list (k_contact.cu)
  double* scal = nullptr;     // [0] barrier energy [1] alpha [2] elastic energy [3] gnorm2
                              // [4] smallest active pair distance
  double* partials = nullptr; // block partial sums
  int n_partials = 0;
  double* pair_grad = nullptr;   // cap * 12
  double* pair_hess = nullptr;   // cap * 144
  int* x2mark = nullptr;      // n2 (touched flags -> c positions)
  int* clist = nullptr;       // n2 (contact-affected x2 indices)
  // reduced system (capacity n2)
  double* Bc = nullptr;       // (3 n2)^2 dense B-check
  int* bocc = nullptr;        // n2*n2 block occupancy
  double* red = nullptr;      // work for the reduced system
  float* redf = nullptr;
  int64_t red_cap = 0;        // elements of red / redf
  int nc_cap = 0;             // n_c the reduced buffers are sized for
  // Host handles of CUDA graphs replaying fixed launch sequences on this
  // workspace (capi.cu); a fresh workspace copy starts with none.
  struct Graph {
    void* exec = nullptr;       // cudaGraphExec_t
    const void* key = nullptr;  // buffer the sequence was captured on
    int key2 = 0, gen = -1, coop = 0;
    bool alone = true;
    int64_t kernels = 0;        // kernel nodes (counted as launches per replay)
    bool failed = false;        // capture unsupported: launch directly
  };
  static constexpr int kGraphs = 12;
  Graph graphs[kGraphs];
  // side stream and fork / join events of this workspace: the part of the
  // reduced system that does not need the right-hand side runs there while
  // the forward solve runs on the solve's own stream
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  // Phi = K11^-1 K12 Sigma^-1 (n1 x n2, float, stored transposed: row j of
  // Phi_t is column j of Phi): with it the x1 block of Eq. 8 splits into the
  // contact-free solve (which overlaps the reduced system) plus
  // Phi[:, c] v after it (mixed precision)
  float* Phi_t = nullptr;
  float* bx = nullptr;        // nf*3 float solve vector of the contact-free x1 solve
  int red_gen = 0;            // bumped whenever the reduced buffers move
  // lock-step batches (batch.cu): read by the batched kernels from the
  // device copy of a batch table
  int active = 0;             // the frame takes part in the launch
  double kappa_f = 0.0;       // barrier stiffness of the frame
  double ls_scale = 1.0;      // line-search factor of the trial step
  int col = 0;                // frame's column block (3 columns) in multi-RHS buffers
  int one_cta_max = 96;       // mixed reduced system: largest n_c on the one-CTA path
  int bar64 = 0;              // batched barrier: float64 pair eigen-solves for this frame
  int barrier_lanes = 0;      // single-frame barrier: one lane per pair (else a warp)
  // Sigma^-1 split into TF32 head and tail (n2 rows, row stride sinv_ld) and
  // their TMA descriptors (host memory, owned by the mesh) for the tensor-core
  // product of the batched global step
  float* sinv_hi = nullptr;
  float* sinv_lo = nullptr;
  int sinv_ld = 0;
  const void* tc_maps = nullptr;
};

// ---- local step (k_local.cu) ---------------------------------------------
// act_df (optional): the same 6 entries as float pairs for the mixed local step
void launch_actuation(cudaStream_t s, int T, const double* fiber, const double* stretch, double* act,
                      float2* act_df);
// precision 0: float64 SVD; 1: float32 SVD refined to float64 accuracy in
// double-float arithmetic (k_elastic_df; tetf then holds float pairs).
void launch_elastic(cudaStream_t s, const DevMesh& m, const double* x, double* tetf,
                    double* proj, double* partials, int precision);
int elastic_blocks(int T);
// g = per-vertex sums of tetf, written by launch_elastic with the same precision
void launch_gather_forces(cudaStream_t s, const DevMesh& m, const double* tetf, double* g,
                          int precision);
void launch_sum_partials(cudaStream_t s, const double* partials, int n, double* out);

// ---- contact (k_contact.cu) -----------------------------------------------
void launch_proxy(cudaStream_t s, const DevMesh& m, const double* x, double* sp);
// Constraint set at proxy positions sp; appends keys to m.pairs and adds the
// barrier energy to m.scal[0].
void launch_detect(cudaStream_t s, const DevMesh& m, const double* sp, double dhat, double kappa);
// Candidate pairs of the swept boxes sp -> sp + dsp (inflated by dhat) and
// the ACCD time of impact (min into m.scal[1] as ordered bits); the caller
// zeroes counters [1] and [9] and sets scal[1] = 1.
void launch_ccd(cudaStream_t s, const DevMesh& m, const double* sp, const double* dsp,
                double dhat, double ccd_s, int accd_max_iters);
// Per-pair barrier gradient and PSD Hessian blocks (pass A) and x2 marks.
void launch_barrier_pairs(cudaStream_t s, const DevMesh& m, int64_t npairs, const double* sp,
                          double dhat, double kappa, int precision);
void launch_mark_scan(cudaStream_t s, const DevMesh& m);
// Scatter pair gradients into g and Hessian blocks into the dense B-check (3nc)^2.
// B-check and g from the per-pair blocks; n_c is read on the device and
// B-check is written only when n_c <= nc_cap (mode: 1 gradient, 2 B-check, 3 both)
void launch_barrier_scatter(cudaStream_t s, const DevMesh& m, int64_t npairs, int nc_cap, int mode,
                            double* g);
// zero B-check and its block occupancy for the n_c on the device (when n_c <= nc_cap)
void launch_zero_reduced(cudaStream_t s, const DevMesh& m, int nc_cap);
// Reset the CCD outputs: counters[1] = counters[9] = 0 and scal[1] = 1.
void launch_ccd_reset(cudaStream_t s, const DevMesh& m);

// ---- global step (k_solve.cu) ----------------------------------------------
// dx (by vertex) solving (H + B) dx = -g, with B-check already assembled for
// the n_c in counters[3] (read on the device: the launch sequence is fixed
// per workspace and can be captured in a CUDA graph).  num_sms is the CTA
// count of the cooperative reduced-system launch; alone = no other solve
// shares the GPU (selects wider triangular-solve work items).
// nc_host: n_c as read back by the host (selects the reduced-system path
// and skips the launches of the others), or -1 when the host does not know it.
cudaError_t global_step(cudaStream_t s, const DevMesh& m, const double* g, double* dx, int precision,
                        int* info_dev, int num_sms, bool alone, bool dense_schur = false,
                        int nc_host = -1);
// Reduced-system path a global step takes for this n_c and precision (graph key).
int reduced_path(int nc_host, int precision, int one_cta_max);
// Schur-only variant of the x2 block (k_schur.cu): z2 = Sigma-hat^-1 y2 with
// Sigma-hat = Sigma (x) I_3 + B-check assembled densely and factored by
// Cholesky (float64, or float32 + two float64 refinement steps).
cudaError_t sigma_hat_solve(cudaStream_t s, const DevMesh& m, const void* y2, double* z2, int* info,
                            int precision);
void set_schur_smem_limits();
int64_t reduced_workspace_elems(int nc);   // doubles (or floats) needed by the reduced solve
// Global step by CG preconditioned with H (k_pcg.cu): dx for (H + W^T B W) dx = -g
// to a relative residual rel_tol; h_scal2 is 2 pinned host doubles.  Returns 0
// or -1 on a CUDA error; *iters_out receives the CG iterations.
int pcg_global_step(cudaStream_t s, const DevMesh& m, const double* g, double* dx, double rel_tol,
                    int max_iters, int* info_dev, int num_sms, double* h_scal2, int* iters_out);
// z2 = u - Sigma^-1 Q^T v with the push-through reduced system (k_reduced.cu);
// precision 0: float64 factors, 1: float32 factors + float64 refinement.
// y2 (double for precision 0, float for 1) is the Schur right-hand side with
// u = Sigma^-1 y2; it scales the refinement's stopping test.
cudaError_t reduced_solve(cudaStream_t s, const DevMesh& m, const double* u, const void* y2,
                          double* z2, int* info, int num_sms, int precision, int nc_host = -1,
                          bool prepared = false);
// Mixed precision, 0 < nc_host <= 128: forks the workspace's side stream off
// s and launches there the kernels that need only B-check and Sigma^-1 (S,
// L_s, block lists, X, N); reduced_solve(..., prepared = true) joins it.
// Returns false (nothing launched) when that split does not apply.
bool reduced_prepare(cudaStream_t s, const DevMesh& m, const double* u, const void* y2, double* z2,
                     int* info, int num_sms, int nc_host);
// x1 = bx1 + Phi[:, c] v (float64 out, solver order, 3 per position) after a
// prepared reduced solve (k_reduced.cu); reads n_c on the device.
cudaError_t phi_apply(cudaStream_t s, const DevMesh& m, const double* u, const void* y2, double* z2,
                      int* info, const float* bx1, double* x1);
// Phi_t at prefactor time (k_solve.cu), from the float64 factor and Sigma^-1,
// using the mesh workspace's float64 solve vectors as scratch.
cudaError_t compute_phi(cudaStream_t s, const DevMesh& m, float* phi_t);
void set_solver_smem_limits(int max_bytes);
void set_reduced_smem_limits();

// ---- misc ------------------------------------------------------------------
void launch_axpy_positions(cudaStream_t s, int n3, const double* x, const double* dx,
                           const double* alpha_dev, double alpha_scale, double* out);
void launch_gnorm2(cudaStream_t s, const DevMesh& m, const double* g, double* partials, int nblk);
int gnorm_blocks(int n);
void launch_reset_pinned(cudaStream_t s, const DevMesh& m, double* x);
void launch_check_finite(cudaStream_t s, int n, const double* v, int* flag);

// rows of Z_J one batched backward work item covers
constexpr int kBwdRowSplit = 256;

// ---- lock-step batches -------------------------------------------------------
// `tab` is a device array of nb DevMesh copies (frames of one mesh); m0 is a
// host copy of any of them (mesh-wide sizes and constants).  Every launch
// serves the frames whose `active` flag is set; `at` 0 evaluates at x, 1 at xt.
void launch_eval_reset_b(cudaStream_t s, const DevMesh* tab, int nb);
void launch_local_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0, int at);
void launch_proxy_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0, int at);
void launch_detect_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0, int at, double dhat);
void launch_gather_forces_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0);
// x2 marks, per-pair derivatives (largest pair count np_max), n_c list,
// B-check (zeroed and assembled when n_c fits nc_cap) and the gradient
void launch_barrier_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0, int64_t np_max,
                      double dhat);
void launch_gnorm2_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0);
// ds = W dx, candidates and the additive-CCD bound alpha_m into scal[1]
void launch_ccd_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0, double dhat,
                  double ccd_s, int accd_max_iters);
// xt = x + alpha_m ls_scale dx
void launch_axpy_b(cudaStream_t s, const DevMesh* tab, int nb, const DevMesh& m0);

// Global step (Eq. 8-11, mixed precision) of every active frame of a batch:
// one multi-right-hand-side forward pass, one Sigma^-1 product and one
// contact-free backward pass for all frames (k_solve.cu), the reduced
// systems of all frames in batched launches (k_reduced.cu), then
// x1 = bx1 + Phi[:, c] v and dx per frame.
struct BatchStep {
  cudaStream_t s = nullptr, s2 = nullptr;   // main and side stream
  cudaEvent_t ev[4] = {};                   // fork / join events
  const DevMesh* tab = nullptr;             // device table (nb frames)
  const DevMesh* m0 = nullptr;              // host copy of one frame (mesh constants)
  int nb = 0, nr = 0;                       // frames; columns of the multi-RHS buffers
  float* rb = nullptr;                      // nf x nr right-hand sides (solver order)
  float* yb = nullptr;                      // n1 x nr forward result
  float* ub = nullptr;                      // n2 x nr Sigma^-1 y2
  float* bx = nullptr;                      // nf x nr contact-free backward solution
  const void* args_dev = nullptr;           // nb reduced-system argument blocks (device)
  const void* args_host = nullptr;          // the same on the host
  const int* nc_host = nullptr;             // n_c per frame
  const int* cols_dev = nullptr;            // 3 col per frame (device)
  double* const* x1s_dev = nullptr;         // r of each frame (device array of pointers)
  int num_sms = 1;
  bool use_tc = true;                       // Sigma^-1 product on the tensor cores
};
cudaError_t global_step_b(const BatchStep& bs);
// whether the batched solves can serve this mesh with nr columns
bool batch_supported(const DevMesh& m, int nr);
// tensor-core product u = Sigma^-1 y2 over nr multi-RHS columns (k_tc.cu)
void tc_split_sinv(const double* sinv, int n2, std::vector<float>& hi, std::vector<float>& lo,
                   int* ld_out);
int tc_encode_sinv(const float* d_hi, const float* d_lo, int n2, int ld, void* maps);
size_t tc_map_bytes();
void tc_set_smem_limits();
bool tc_sinv_supported(const DevMesh& m, int nr);
// the float32 SIMT form of the same product (k_solve.cu)
cudaError_t launch_sinv_simt(cudaStream_t s, const DevMesh& m, const float* Y, int nr, float* U);
cudaError_t launch_sinv_tc(cudaStream_t s, const DevMesh& m, const float* Y, int nr, float* U,
                           int num_sms, int* err);
size_t reduced_args_bytes();
void reduced_args_fill(void* dst, const DevMesh& m, int active);
cudaError_t reduced_prepare_b(cudaStream_t s2, const void* args_dev, int nb, int num_sms);
cudaError_t reduced_solve_b(cudaStream_t s, const void* args_dev, const void* args_host, int nb,
                            const int* nc_host, int num_sms);
cudaError_t phi_apply_b(cudaStream_t s, const void* args_dev, const int* cols_dev, int nb, int n1,
                        const float* phi_t, const float* bxm, int nr, double* const* x1s_dev);

// number of kernel launches issued through these launchers (per process)
int64_t launch_counter();
void count_launch(int k = 1);

// Optional CUDA-event timing of kernel classes (see fsim_profile in fsim.h).
enum ProfClass {
  PROF_ELASTIC = 0, PROF_DETECT = 1, PROF_TRSV_FWD = 2, PROF_TRSV_BWD = 3, PROF_CHOL = 4,
  PROF_BARRIER = 5, PROF_CCD = 6, PROF_GEMV = 7, PROF_REDUCED = 8, PROF_PCG = 9,
  PROF_SCHUR = 10, PROF_NCLASS = 11
};
struct ProfScope {
  ProfScope(int cls, cudaStream_t s);
  ~ProfScope();
  int slot;
  cudaStream_t stream;
};
// ---------------------------------------------------------------------------
// Bounds-checked builds (-DFSIM_CHECK).  Data-dependent indices (adjacency
// slots, pair primitives, scatter rows, contact lists) are tested before
// use; a failing index is skipped and the first failure of a translation
// unit is kept in its check word: site << 48 | (index & 0xffffffffffff).
// Without FSIM_CHECK the test is a constant true and costs nothing.
// ---------------------------------------------------------------------------
enum CheckSite : int {
  CHECK_GATHER_TET = 1,      // force gather: vertex-tet slot out of the tet range
  CHECK_TRSV_ROW = 2,        // multi-RHS supernodal solves: off-diagonal row position
  CHECK_CLIST = 3            // reduced system / z2 / Phi: contact list entry out of x2
};
#if defined(FSIM_CHECK) && defined(__CUDACC__)
static __device__ unsigned long long g_check_word = 0ull;   // one per translation unit
__device__ __forceinline__ bool check_idx(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_check_word, 0ull,
            ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffull));
  return false;
}
#define FSIM_CHECK_IDX(i, n, site) ::fsim::check_idx((long long)(i), (long long)(n), (site))
// host reader of this translation unit's word (reset to 0 after reading)
#define FSIM_CHECK_READER(name)                                                   \
  uint64_t name() {                                                               \
    unsigned long long v = 0, z = 0;                                              \
    cudaMemcpyFromSymbol(&v, g_check_word, sizeof(v));                            \
    cudaMemcpyToSymbol(g_check_word, &z, sizeof(z));                              \
    return (uint64_t)v;                                                           \
  }
#else
#define FSIM_CHECK_IDX(i, n, site) true
#define FSIM_CHECK_READER(name) \
  uint64_t name() { return 0; }
#endif
uint64_t check_word_local();
uint64_t check_word_solve();
uint64_t check_word_reduced();

// An NVTX range for the lifetime of the object (whole frames, batch iterations)
struct NvtxRange {
  explicit NvtxRange(const char* name);
  ~NvtxRange();
};
void prof_set_mask(unsigned mask);
bool prof_active();
// While a thread captures a CUDA graph its launches are not counted (the
// replays count the graph's kernel nodes instead).
void set_capturing(bool on);
int prof_read(int cls, int64_t* launches, double* total_ms);
void prof_reset();

}  // namespace fsim
