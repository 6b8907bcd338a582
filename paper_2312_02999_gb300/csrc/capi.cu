// C ABI (include/fsim.h): context, mesh upload, prefactor, actuation, the
// Algorithm 1 loop and the step-level entry points.
//
// The host code here only sequences kernels and reads back the few scalars
// that steer the loop (gradient norm, n_c, candidate count, trial energy);
// every arithmetic step of an iteration runs in the CUDA kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "fsim_internal.h"
#include "kernels.h"
#include "runtime.h"

using namespace fsim;

namespace {

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      fprintf(stderr, "fsim: CUDA error %s at %s:%d\n",            \
              cudaGetErrorString(e_), __FILE__, __LINE__);         \
      return FSIM_ECUDA;                                           \
    }                                                              \
  } while (0)

template <typename T>
int dalloc(std::vector<void*>& allocs, T** p, size_t count, size_t* bytes = nullptr) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) { cudaGetLastError(); return FSIM_ENOMEM; }
  allocs.push_back(*p);
  if (bytes) *bytes += sizeof(T) * count;
  return FSIM_OK;
}
template <typename T>
int dalloc(MeshState& ms, T** p, size_t count) { return dalloc(ms.allocs, p, count); }

#define TRY(x)                    \
  do {                            \
    int s_ = (x);                 \
    if (s_ != FSIM_OK) return s_; \
  } while (0)

template <typename T>
int upload(MeshState& ms, cudaStream_t s, T** p, const T* h, size_t count) {
  TRY(dalloc(ms, p, count));
  if (count) {
    cudaError_t e = cudaMemcpyAsync(*p, h, sizeof(T) * count, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return FSIM_ECUDA;
  }
  return FSIM_OK;
}

MeshState* get_mesh(fsim_ctx_t ctx, int id) {
  if (ctx == nullptr || id < 0 || id >= (int)ctx->meshes.size()) return nullptr;
  return ctx->meshes[id].get();
}

void free_list(std::vector<void*>& allocs) {
  for (void* p : allocs) cudaFree(p);
  allocs.clear();
}

void destroy_graphs(DevMesh& m);

void free_mesh(MeshState& ms) {
  destroy_graphs(ms.d);
  free_list(ms.allocs);
  delete[] ms.d.h_level_ptr;
  delete[] ms.d.h_level_maxns;
  delete[] ms.d.h_level_maxld;
  delete[] ms.d.h_fwd_ptr;
  delete[] ms.d.h_bwd_ptr;
  delete[] ms.d.h_bwd32_ptr;
  ms.d.h_bwd32_ptr = nullptr;
  ms.d.h_level_ptr = nullptr;
  ms.d.h_level_maxns = nullptr;
  ms.d.h_level_maxld = nullptr;
  ms.d.h_fwd_ptr = nullptr;
  ms.d.h_bwd_ptr = nullptr;
}

Exec ctx_exec(fsim_ctx_t ctx, MeshState& ms) {
  Exec ex;
  ex.stream = ctx->stream;
  ex.h_counters = ctx->h_counters;
  ex.h_scal = ctx->h_scal;
  ex.coop_ctas = ms.p.coop_ctas > 0 ? std::min(ms.p.coop_ctas, ctx->num_sms) : ctx->num_sms;
  ex.allocs = &ms.allocs;
  return ex;
}

int sync_read(const Exec& ex, const DevMesh& m) {
  CK(cudaMemcpyAsync(ex.h_counters, m.counters, sizeof(int) * kCounters, cudaMemcpyDeviceToHost,
                     ex.stream));
  CK(cudaMemcpyAsync(ex.h_scal, m.scal, sizeof(double) * kScal, cudaMemcpyDeviceToHost, ex.stream));
  CK(cudaStreamSynchronize(ex.stream));
  return FSIM_OK;
}

// Make the reduced-system buffers of workspace m large enough for nc
// contact vertices (grows by 1.5x, at most to n2).
size_t reduced_bytes(int cap) {
  if (cap <= 0) return 0;
  const int64_t n3 = 3 * (int64_t)cap;
  return sizeof(double) * (size_t)(n3 * n3) + sizeof(int) * (size_t)(2 * (int64_t)cap * cap + cap + 32) +
         (sizeof(double) + sizeof(float)) * (size_t)reduced_workspace_elems(cap);
}

int ensure_reduced(const Exec& ex, DevMesh& m, int nc) {
  if (nc <= m.nc_cap && m.Bc != nullptr) return FSIM_OK;
  int cap = std::max(nc, std::max(16, m.nc_cap * 3 / 2));
  cap = std::min(cap, std::max(m.n2, 1));
  const size_t old_bytes = m.Bc != nullptr ? reduced_bytes(m.nc_cap) : 0;
  const size_t new_bytes = reduced_bytes(cap);
  if (ex.grow && new_bytes > old_bytes && ex.grow(ex.grow_user, new_bytes - old_bytes) != 0)
    return FSIM_ENOMEM;
  CK(cudaStreamSynchronize(ex.stream));
  auto release = [&](void* p) {
    if (!p) return;
    cudaFree(p);
    auto& v = *ex.allocs;
    v.erase(std::remove(v.begin(), v.end(), p), v.end());
  };
  release(m.Bc); release(m.bocc); release(m.red); release(m.redf);
  m.Bc = nullptr; m.bocc = nullptr; m.red = nullptr; m.redf = nullptr;
  if (ex.bytes) *ex.bytes -= std::min(*ex.bytes, old_bytes);
  const int64_t n3 = 3 * (int64_t)cap;
  TRY(dalloc(*ex.allocs, &m.Bc, (size_t)(n3 * n3), ex.bytes));
  TRY(dalloc(*ex.allocs, &m.bocc, (size_t)(2 * (int64_t)cap * cap + cap + 32), ex.bytes));
  m.red_cap = reduced_workspace_elems(cap);
  TRY(dalloc(*ex.allocs, &m.red, (size_t)m.red_cap, ex.bytes));
  TRY(dalloc(*ex.allocs, &m.redf, (size_t)m.red_cap, ex.bytes));
  m.nc_cap = cap;
  m.red_gen++;
  return FSIM_OK;
}

// Per-solve buffers of a workspace (everything a frame solve writes).  The
// constant mesh data (factor, Sigma^-1, topology) stays shared.  Used for
// the mesh's own workspace at prefactor and for the server's extra slots.
int alloc_workspace(const MeshState& ms, DevMesh& m, std::vector<void*>& al, size_t* bytes) {
  // a copy must never replay (or destroy) another workspace's graphs, nor
  // use its side stream
  for (auto& g : m.graphs) g = DevMesh::Graph{};
  m.red_gen = 0;
  m.aux_stream = nullptr;
  m.ev_fork = m.ev_join = m.ev_fork2 = m.ev_join2 = nullptr;
  if (cudaStreamCreateWithFlags(&m.aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&m.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&m.ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&m.ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&m.ev_join2, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return FSIM_ECUDA;
  }
  const size_t n = m.n, T = m.T, Ns = m.Ns;
  const size_t np = (size_t)m.Ns + m.Nt + m.Ne;
  TRY(dalloc(al, &m.x, 3 * n, bytes));
  TRY(dalloc(al, &m.xt, 3 * n, bytes));
  TRY(dalloc(al, &m.dx, 3 * n, bytes));
  TRY(dalloc(al, &m.g, 3 * n, bytes));
  TRY(dalloc(al, &m.act, 6 * T, bytes));
  TRY(dalloc(al, &m.act_df, 6 * T, bytes));
  TRY(dalloc(al, &m.udf, 3 * n, bytes));
  TRY(dalloc(al, &m.tetf, 12 * T, bytes));
  TRY(dalloc(al, &m.tetf_t, 12 * T, bytes));
  TRY(dalloc(al, &m.s, 3 * Ns, bytes));
  TRY(dalloc(al, &m.st, 3 * Ns, bytes));
  TRY(dalloc(al, &m.ds, 3 * Ns, bytes));
  TRY(dalloc(al, &m.pbox, 12 * np, bytes));
  TRY(dalloc(al, &m.pkey, 12 * np, bytes));
  TRY(dalloc(al, &m.sf, 3 * Ns, bytes));
  TRY(dalloc(al, &m.dsf, 3 * Ns, bytes));
  TRY(dalloc(al, &m.counters, kCounters, bytes));
  CK(cudaMemset(m.counters, 0, sizeof(int) * kCounters));   // skin list starts invalid
  TRY(dalloc(al, &m.scal, kScal, bytes));
  TRY(dalloc(al, &m.partials, (size_t)m.n_partials, bytes));
  TRY(dalloc(al, &m.y1, 3 * (size_t)std::max(m.n1, 1), bytes));
  TRY(dalloc(al, &m.y1f, 3 * (size_t)std::max(m.n1, 1), bytes));
  TRY(dalloc(al, &m.r, 3 * (size_t)m.nf, bytes));
  TRY(dalloc(al, &m.u, 3 * (size_t)std::max(m.n2, 1), bytes));
  TRY(dalloc(al, &m.rf, 3 * (size_t)m.nf + 8, bytes));
  TRY(dalloc(al, &m.bx, 3 * (size_t)m.nf + 8, bytes));
  TRY(dalloc(al, &m.uf, 3 * (size_t)std::max(m.n2, 1), bytes));
  TRY(dalloc(al, &m.pairs, (size_t)m.cap_act, bytes));
  TRY(dalloc(al, &m.cand, (size_t)m.cap, bytes));
  TRY(dalloc(al, &m.nearl, (size_t)m.cap, bytes));
  TRY(dalloc(al, &m.vlist, (size_t)m.cap, bytes));
  if (ms.p.solver == FSIM_SOLVER_PCG) {
    TRY(dalloc(al, &m.cg_r, 3 * n, bytes));
    TRY(dalloc(al, &m.cg_z, 3 * n, bytes));
    TRY(dalloc(al, &m.cg_p, 3 * n, bytes));
    TRY(dalloc(al, &m.cg_q, 3 * n, bytes));
    TRY(dalloc(al, &m.cg_tmp, 3 * n, bytes));
    TRY(dalloc(al, &m.cg_red, 2, bytes));
  }
  if (ms.p.solver == FSIM_SOLVER_SCHUR && m.n2 > 0) {
    const size_t N = 3 * (size_t)m.n2;
    TRY(dalloc(al, &m.sh_A, N * N, bytes));
    TRY(dalloc(al, &m.sh_Af, N * N, bytes));
    TRY(dalloc(al, &m.sh_y, N, bytes));
    TRY(dalloc(al, &m.sh_r, N, bytes));
    TRY(dalloc(al, &m.sh_df, N, bytes));
  }
  TRY(dalloc(al, &m.sb, 3 * Ns, bytes));
  TRY(dalloc(al, &m.pair_grad, 12 * (size_t)m.cap_act, bytes));
  TRY(dalloc(al, &m.pair_hess, 144 * (size_t)m.cap_act, bytes));
  TRY(dalloc(al, &m.x2mark, (size_t)std::max(m.n2, 1), bytes));
  TRY(dalloc(al, &m.clist, (size_t)std::max(m.n2, 1), bytes));
  m.Bc = nullptr; m.bocc = nullptr; m.red = nullptr; m.redf = nullptr;
  m.red_cap = 0; m.nc_cap = 0;
  (void)ms;
  return FSIM_OK;
}

void destroy_graphs(DevMesh& m) {
  for (auto& g : m.graphs) {
    if (g.exec) cudaGraphExecDestroy((cudaGraphExec_t)g.exec);
    g = DevMesh::Graph{};
  }
  if (m.ev_fork) cudaEventDestroy(m.ev_fork);
  if (m.ev_join) cudaEventDestroy(m.ev_join);
  if (m.ev_fork2) cudaEventDestroy(m.ev_fork2);
  if (m.ev_join2) cudaEventDestroy(m.ev_join2);
  if (m.aux_stream) cudaStreamDestroy(m.aux_stream);
  m.ev_fork = m.ev_join = m.ev_fork2 = m.ev_join2 = nullptr;
  m.aux_stream = nullptr;
}

// Run a fixed launch sequence through a CUDA graph captured on first use
// (one host launch instead of one per kernel).  The graph is recaptured
// when its key buffer, precision, reduced-buffer generation or cooperative
// CTA count changes; with the event profiler on, or where capture is not
// supported, the sequence is launched directly.
template <typename F>
int with_graph(const Exec& ex, DevMesh& m, int slot, const void* key, int key2, int gen, F&& body) {
  DevMesh::Graph& g = m.graphs[slot];
  if (g.failed || prof_active()) return body();
  if (g.exec && (g.key != key || g.key2 != key2 || g.gen != gen || g.coop != ex.coop_ctas ||
                 g.alone != ex.alone)) {
    cudaGraphExecDestroy((cudaGraphExec_t)g.exec);
    g.exec = nullptr;
  }
  if (!g.exec) {
    if (cudaStreamBeginCapture(ex.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      g.failed = true;
      return body();
    }
    set_capturing(true);
    const int rc = body();
    set_capturing(false);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ex.stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc == FSIM_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&exec, graph, 0);
    int64_t kernels = 0;
    if (graph) {
      size_t nn = 0;
      cudaGraphGetNodes(graph, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
      cudaGraphDestroy(graph);
    }
    if (rc != FSIM_OK || e != cudaSuccess || !exec) {
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      g.failed = true;
      return body();      // nothing ran during the capture: launch directly
    }
    g.exec = exec; g.key = key; g.key2 = key2; g.gen = gen; g.coop = ex.coop_ctas; g.alone = ex.alone;
    g.kernels = kernels;
  }
  CK(cudaGraphLaunch((cudaGraphExec_t)g.exec, ex.stream));
  count_launch((int)g.kernels);
  return FSIM_OK;
}

// graph slots: 0-5 global step (by precision and reduced-system path), 6-9
// evaluation (by position buffer and precision), 10-11 CCD (by proxy-position
// buffer)
int graph_slot(const DevMesh& m, int first, int count, const void* key, int key2) {
  for (int k = first; k < first + count; ++k)
    if (m.graphs[k].exec && m.graphs[k].key == key && m.graphs[k].key2 == key2) return k;
  for (int k = first; k < first + count; ++k)
    if (!m.graphs[k].exec && !m.graphs[k].failed) return k;
  for (int k = first; k < first + count; ++k)
    if (!m.graphs[k].failed) return k;
  return first;
}

// ---------------------------------------------------------------------------
// one evaluation at positions xb: local step (energy + per-tet forces into
// tetf), proxy positions sb and the constraint set with barrier energy.
// Leaves E in scal[2], B in scal[0], |C| in counters[0].
// ---------------------------------------------------------------------------
int evaluate(const Exec& ex, const MeshState& ms, const DevMesh& m, const double* xb, double* sb,
             double* tetf, double* proj, int prec, double kappa) {
  cudaStream_t s = ex.stream;
  CK(cudaMemsetAsync(m.counters, 0, sizeof(int) * 3, s));       // |C|, candidates, overflow
  CK(cudaMemsetAsync(m.counters + 5, 0, sizeof(int), s));       // touching pair
  CK(cudaMemsetAsync(m.counters + 8, 0, sizeof(int), s));       // near-pair list
  CK(cudaMemsetAsync(m.scal, 0, sizeof(double) * 1, s));
  launch_elastic(s, m, xb, tetf, proj, m.partials, prec);
  launch_sum_partials(s, m.partials, elastic_blocks(m.T), m.scal + 2);
  launch_proxy(s, m, xb, sb);
  launch_detect(s, m, sb, ms.p.dhat, kappa);
  CK(cudaGetLastError());
  return FSIM_OK;
}

// Gradient g-hat (elastic from tetf + barrier over the pairs in m.pairs at
// sb) into gout, the contact-affected set, B-check and ||g||^2.
// Requires counters[0] (|C|) already on the host in npairs.
// bprec is the precision of the pairs' PSD eigen-solves (prec unless the
// frame switched its contact Hessian to float64).
int gradient_and_hessian(const Exec& ex, const MeshState& ms, DevMesh& m, const double* sb,
                         const double* tetf, double* gout, int64_t npairs, int prec, int* nc_out,
                         double* gn2_out, double kappa, int bprec = -1) {
  cudaStream_t s = ex.stream;
  launch_gather_forces(s, m, tetf, gout, prec);
  CK(cudaMemsetAsync(m.x2mark, 0, sizeof(int) * std::max(m.n2, 1), s));
  launch_barrier_pairs(s, m, npairs, sb, ms.p.dhat, kappa, bprec < 0 ? prec : bprec);
  if (m.n2 > 0) launch_mark_scan(s, m);
  else CK(cudaMemsetAsync(m.counters + 3, 0, sizeof(int), s));
  // n_c stays on the device until the one read-back below: B-check is zeroed
  // and assembled in place when it fits the current reduced buffers
  const int cap_now = m.Bc != nullptr ? m.nc_cap : 0;
  launch_zero_reduced(s, m, cap_now);
  launch_barrier_scatter(s, m, npairs, cap_now, 3, gout);
  const int nb = gnorm_blocks(m.n);
  launch_gnorm2(s, m, gout, m.partials, nb);
  launch_sum_partials(s, m.partials, nb, m.scal + 3);
  TRY(sync_read(ex, m));
  const int nc = ex.h_counters[3];
  TRY(ensure_reduced(ex, m, std::max(nc, 1)));
  if (nc > cap_now) {       // the buffers grew: assemble B-check again
    CK(cudaMemsetAsync(m.Bc, 0, sizeof(double) * 9 * (size_t)nc * nc, s));
    CK(cudaMemsetAsync(m.bocc, 0, sizeof(int) * (size_t)nc * nc, s));
    launch_barrier_scatter(s, m, npairs, m.nc_cap, 2, gout);
  }
  *nc_out = nc;
  *gn2_out = ex.h_scal[3];
  return FSIM_OK;
}

constexpr double kKappaGrowBelow = 0.1;   // adaptive kappa: grow below 0.1 dhat ...
constexpr double kKappaMaxRatio = 100.0;   // ... up to 100 times the start value

int solve_frame_impl(const Exec& ex, const MeshState& ms, DevMesh& m, const double* x_init,
                     bool init_is_dev, int prec, fsim_frame_stats* stats) {
  NvtxRange nv("fsim.frame");
  cudaStream_t s = ex.stream;
  const fsim_params& p = ms.p;
  fsim_frame_stats st{};
  st.alpha_min = 1.0;
  if (x_init != nullptr) {
    CK(cudaMemcpyAsync(m.x, x_init, sizeof(double) * 3 * (size_t)m.n,
                       init_is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  }
  launch_reset_pinned(s, m, m.x);
  CK(cudaMemsetAsync(m.counters + 4, 0, sizeof(int), s));
  launch_check_finite(s, 3 * m.n, m.x, m.counters + 4);
  // barrier stiffness of this frame: starts at the mesh's kappa; with
  // adaptive_kappa it doubles when the smallest active distance falls below
  // kKappaGrowBelow dhat and keeps shrinking (IPC's rule, as the paper uses
  // it), up to kKappaMaxRatio times the start value
  double kappa = ms.kappa;
  int kgen = 0;
  double d_prev = INFINITY;
  auto adapt_kappa = [&](double d_min, double* E_barrier) {
    if (!p.adaptive_kappa) return;
    if (d_min < kKappaGrowBelow * p.dhat && d_min < d_prev && 2.0 * kappa <= kKappaMaxRatio * ms.kappa) {
      kappa *= 2.0;
      *E_barrier *= 2.0;          // B is linear in kappa
      ++kgen;
      st.kappa_doublings++;
    }
    d_prev = d_min;
  };
  auto eval_at = [&](double* xb, double* sb, double* tetf) -> int {
    const int slot = graph_slot(m, 6, 4, xb, prec);
    return with_graph(ex, m, slot, xb, prec, kgen,
                      [&] { return evaluate(ex, ms, m, xb, sb, tetf, nullptr, prec, kappa); });
  };
  TRY(eval_at(m.x, m.s, m.tetf));
  TRY(sync_read(ex, m));
  int rc = FSIM_OK;
  if (ex.h_counters[4]) rc = FSIM_ENONFINITE;
  else if (ex.h_counters[5]) rc = FSIM_EINTERSECTING;
  else if (ex.h_counters[2]) rc = FSIM_ECONTACT_OVERFLOW;
  int64_t npairs = ex.h_counters[0];
  double Eb = ex.h_scal[0];
  adapt_kappa(ex.h_scal[4], &Eb);
  double E = ex.h_scal[2] + Eb;
  double gn = 0.0, tol = 0.0;
  int nc = 0;
  if (rc == FSIM_OK) {
    double gn2;
    TRY(gradient_and_hessian(ex, ms, m, m.s, m.tetf, m.g, npairs, prec, &nc, &gn2, kappa));
    gn = std::sqrt(gn2);
    st.grad_norm0 = gn;
    tol = std::max(p.tol_abs, p.tol_rel * gn);
    if (!std::isfinite(gn)) rc = FSIM_ENONFINITE;
  }
  // precision of the contact Hessian and the global step: the frame's own,
  // until a float32 factor of the reduced (or Schur) system loses positive
  // definiteness; from then on the frame's pair eigen-solves and global steps
  // run in float64 (a frame that got that stiff stays stiff while its pairs
  // stay close, and the float32 eigen-solve's relative floor drops the soft
  // directions of such pairs)
  int gprec = prec;
  while (rc == FSIM_OK) {
    st.n_c = nc;
    st.n_c_max = std::max(st.n_c_max, nc);
    if (gn <= tol) break;
    if (st.iterations >= p.max_iters) { rc = FSIM_ENOT_CONVERGED; break; }
    // global step (Eq. 4 via Eq. 8-11, or the CG comparison configuration)
    if (p.solver == FSIM_SOLVER_PCG) {
      CK(cudaMemsetAsync(m.counters + 6, 0, sizeof(int) * 2, s));
      int cg_it = 0;
      if (pcg_global_step(s, m, m.g, m.dx, p.cg_tol, p.cg_max_iters, m.counters + 6, ex.coop_ctas,
                          ex.h_scal + 6, &cg_it) != 0)
        return FSIM_ECUDA;
      st.cg_iterations += cg_it;
    } else {
      // one graph per precision and reduced-system path (n_c decides the path)
      const bool schur = p.solver == FSIM_SOLVER_SCHUR;
      const int gkey = 8 * gprec + (schur ? 4 : reduced_path(nc, gprec, m.one_cta_max));
      TRY(with_graph(ex, m, graph_slot(m, 0, 6, m.g, gkey), m.g, gkey, m.red_gen, [&]() -> int {
        CK(cudaMemsetAsync(m.counters + 6, 0, sizeof(int) * 2, s));
        CK(global_step(s, m, m.g, m.dx, gprec, m.counters + 6, ex.coop_ctas, ex.alone, schur, nc));
        return FSIM_OK;
      }));
      if (gprec != prec) st.fp64_steps++;
    }
    st.sum_nc3 += (double)nc * nc * nc;
    if (p.solver == FSIM_SOLVER_WOODBURY) st.reduced_steps[reduced_path(nc, gprec, m.one_cta_max)]++;
    // CCD step bound; the ACCD kernel reads the candidate count on the device,
    // and the overflow / factorisation flags are checked at the next read-back
    TRY(with_graph(ex, m, graph_slot(m, 10, 2, m.s, 0), m.s, 0, 0, [&]() -> int {
      launch_proxy(s, m, m.dx, m.ds);
      launch_ccd_reset(s, m);
      launch_ccd(s, m, m.s, m.ds, p.dhat, p.ccd_s, p.accd_max_iters);
      CK(cudaGetLastError());
      return FSIM_OK;
    }));
    // backtracking line search from alpha_m on E-hat = E + B
    bool accepted = false, redone = false;
    double scale = 1.0, Et = 0.0;
    int64_t np_t = 0;
    for (int k = 0; k <= p.max_ls; ++k) {
      launch_axpy_positions(s, 3 * m.n, m.x, m.dx, m.scal + 1, scale, m.xt);
      TRY(eval_at(m.xt, m.st, m.tetf_t));
      TRY(sync_read(ex, m));
      if (k == 0 && ex.h_counters[6] && gprec != FSIM_FP64 && p.solver != FSIM_SOLVER_PCG &&
          !redone) {
        // the float32 factor of the reduced (or Schur) system lost positive
        // definiteness (cond ~ 1 / u32 at very stiff pairs): the contact
        // Hessian at x again with float64 eigen-solves (the trial evaluation
        // replaced the pair list, so x is evaluated again first), this global
        // step in float64, its CCD bound and a fresh line search
        redone = true;
        gprec = FSIM_FP64;
        st.fp64_steps++;
        if (p.solver == FSIM_SOLVER_WOODBURY) {
          st.reduced_steps[reduced_path(nc, prec, m.one_cta_max)]--;
          st.reduced_steps[reduced_path(nc, FSIM_FP64, m.one_cta_max)]++;
        }
        TRY(eval_at(m.x, m.s, m.tetf));
        TRY(sync_read(ex, m));
        {
          double gn2r;
          TRY(gradient_and_hessian(ex, ms, m, m.s, m.tetf, m.g, npairs, prec, &nc, &gn2r, kappa,
                                   gprec));
        }
        CK(cudaMemsetAsync(m.counters + 6, 0, sizeof(int) * 2, s));
        CK(global_step(s, m, m.g, m.dx, FSIM_FP64, m.counters + 6, ex.coop_ctas, ex.alone,
                       p.solver == FSIM_SOLVER_SCHUR, nc));
        launch_proxy(s, m, m.dx, m.ds);
        launch_ccd_reset(s, m);
        launch_ccd(s, m, m.s, m.ds, p.dhat, p.ccd_s, p.accd_max_iters);
        CK(cudaGetLastError());
        scale = 1.0;
        k = -1;
        continue;
      }
      if (k == 0 && ex.h_counters[6]) { rc = FSIM_ENOT_SPD; break; }
      if (k == 0 && ex.h_counters[9]) { rc = FSIM_ECONTACT_OVERFLOW; break; }
      st.ls_trials++;
      Et = ex.h_scal[2] + ex.h_scal[0];
      np_t = ex.h_counters[0];
      if (ex.h_counters[2]) { rc = FSIM_ECONTACT_OVERFLOW; break; }
      if (!ex.h_counters[5] && std::isfinite(Et) && Et <= E + 1e-12 * std::fabs(E)) {
        accepted = true;
        break;
      }
      scale *= 0.5;
    }
    if (rc != FSIM_OK) break;
    if (!accepted) { rc = FSIM_ELS_FAIL; break; }
    st.alpha_min = std::min(st.alpha_min, ex.h_scal[1] * scale);
    std::swap(m.x, m.xt);
    std::swap(m.s, m.st);
    std::swap(m.tetf, m.tetf_t);
    {
      double Ebt = ex.h_scal[0];
      adapt_kappa(ex.h_scal[4], &Ebt);
      E = ex.h_scal[2] + Ebt;
    }
    npairs = np_t;
    st.iterations++;
    double gn2;
    TRY(gradient_and_hessian(ex, ms, m, m.s, m.tetf, m.g, npairs, prec, &nc, &gn2, kappa, gprec));
    gn = std::sqrt(gn2);
    if (!std::isfinite(gn)) rc = FSIM_ENONFINITE;
  }
  st.status = rc;
  st.grad_norm = gn;
  st.energy = E;
  st.contacts = npairs;
  if (stats) *stats = st;
  return rc;
}

}  // namespace

namespace fsim {
int rt_alloc_workspace(const MeshState& ms, DevMesh& m, std::vector<void*>& allocs, size_t* bytes) {
  return alloc_workspace(ms, m, allocs, bytes);
}
int rt_ensure_reduced(const Exec& ex, DevMesh& m, int nc) { return ensure_reduced(ex, m, nc); }
size_t rt_reduced_bytes(int nc_cap) { return reduced_bytes(nc_cap); }
int rt_solve_frame(const Exec& ex, const MeshState& ms, DevMesh& m, const double* x_init,
                   bool init_is_dev, int precision, fsim_frame_stats* stats) {
  return solve_frame_impl(ex, ms, m, x_init, init_is_dev, precision, stats);
}
void rt_free_list(std::vector<void*>& allocs) { free_list(allocs); }
void rt_destroy_graphs(DevMesh& m) { destroy_graphs(m); }
size_t rt_slot_bytes(const MeshState& ms) {
  if (!ms.prefactored) return 0;
  const int cap = std::min(std::max(ms.d.n2, 1), 64);
  return ms.ws_bytes + reduced_bytes(cap);
}
MeshState* rt_mesh(fsim_ctx_t ctx, int mesh_id) { return get_mesh(ctx, mesh_id); }
}  // namespace fsim

// ===========================================================================
extern "C" {

fsim_status fsim_default_params(fsim_params* p) {
  if (!p) return FSIM_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->weight_scale = 1e3;
  p->dhat = 0.0;
  p->kappa = 0.0;
  p->tol_abs = 1e-8;
  p->tol_rel = 0.0;
  p->max_iters = 500;
  p->max_ls = 40;
  p->ccd_s = 0.1;
  p->accd_max_iters = 2000;
  p->contact_capacity = 0;
  p->active_capacity = 0;
  p->skin = 0.0;
  p->solver = FSIM_SOLVER_WOODBURY;
  p->cg_max_iters = 2000;
  p->cg_tol = 1e-8;
  p->adaptive_kappa = 0;
  return FSIM_OK;
}

fsim_status fsim_create(fsim_ctx_t* out, int device) {
  if (!out) return FSIM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return FSIM_EINVAL;
  }
  auto* c = new (std::nothrow) fsim_ctx_s();
  if (!c) return FSIM_ENOMEM;
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete c; return FSIM_ECUDA; }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  // solve streams get the highest priority and the workspaces' side streams
  // the default (lowest): the side stream only fills SMs the critical path
  // leaves free (its work is off the critical path)
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
    delete c;
    return FSIM_ECUDA;
  }
  if (cudaHostAlloc((void**)&c->h_counters, sizeof(int) * kCounters, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&c->h_scal, sizeof(double) * kScal, cudaHostAllocDefault) != cudaSuccess) {
    cudaStreamDestroy(c->stream);
    delete c;
    return FSIM_ENOMEM;
  }
  set_solver_smem_limits(200 * 1024);
  set_reduced_smem_limits();
  set_schur_smem_limits();
  *out = c;
  return FSIM_OK;
}

fsim_status fsim_destroy(fsim_ctx_t ctx) {
  if (!ctx) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& m : ctx->meshes)
    if (m) free_mesh(*m);
  cudaFreeHost(ctx->h_counters);
  cudaFreeHost(ctx->h_scal);
  cudaStreamDestroy(ctx->stream);
  delete ctx;
  return FSIM_OK;
}

fsim_status fsim_launch_count(fsim_ctx_t ctx, int64_t* count) {
  if (!ctx || !count) return FSIM_EINVAL;
  *count = launch_counter();
  return FSIM_OK;
}

fsim_status fsim_mesh_upload(fsim_ctx_t ctx, int* mesh_id, const double* rest_xyz, int64_t n,
                             const int32_t* tets, int64_t T, const uint8_t* pinned,
                             const int32_t* proxy_tris, int64_t Nt, const int64_t* W_rowptr,
                             const int32_t* W_col, const double* W_val, int64_t Ns,
                             const uint8_t* region) {
  if (!ctx || !mesh_id || !rest_xyz || !tets || !pinned || n <= 0 || T <= 0 || n >= (1LL << 30) ||
      T >= (1LL << 30) || Ns < 0 || Nt < 0 || (Ns > 0 && (!W_rowptr || !W_col || !W_val)) ||
      (Nt > 0 && !proxy_tris))
    return FSIM_EINVAL;
  for (int64_t k = 0; k < 4 * T; ++k)
    if (tets[k] < 0 || tets[k] >= n) return FSIM_EINVAL;
  for (int64_t k = 0; k < 3 * Nt; ++k)
    if (proxy_tris[k] < 0 || proxy_tris[k] >= Ns) return FSIM_EINVAL;
  if (Ns > 0) {
    if (W_rowptr[0] != 0) return FSIM_EINVAL;
    for (int64_t r = 0; r < Ns; ++r) {
      if (W_rowptr[r + 1] < W_rowptr[r] || W_rowptr[r + 1] - W_rowptr[r] > 4) return FSIM_EINVAL;
    }
    for (int64_t e = 0; e < W_rowptr[Ns]; ++e)
      if (W_col[e] < 0 || W_col[e] >= n) return FSIM_EINVAL;
  }
  cudaSetDevice(ctx->device);
  auto msp = std::make_unique<MeshState>();
  MeshState& ms = *msp;
  DevMesh& m = ms.d;
  cudaStream_t s = ctx->stream;
  m.n = (int)n; m.T = (int)T; m.Ns = (int)Ns; m.Nt = (int)Nt;
  ms.rest.assign(rest_xyz, rest_xyz + 3 * n);
  ms.tets.assign(tets, tets + 4 * T);
  ms.pinned.assign(pinned, pinned + n);
  // collision-aware set x2: region (if given) plus the free support of W
  ms.x2mask.assign(n, 0);
  if (region)
    for (int64_t v = 0; v < n; ++v) ms.x2mask[v] = region[v] ? 1 : 0;
  if (Ns > 0)
    for (int64_t e = 0; e < W_rowptr[Ns]; ++e) ms.x2mask[W_col[e]] = 1;
  for (int64_t v = 0; v < n; ++v)
    if (pinned[v]) ms.x2mask[v] = 0;
  // proxy edges: sorted unique (lo, hi)
  std::vector<std::pair<int, int>> ed;
  ed.reserve(3 * Nt);
  for (int64_t t = 0; t < Nt; ++t)
    for (int k = 0; k < 3; ++k) {
      int a = proxy_tris[3 * t + k], b = proxy_tris[3 * t + (k + 1) % 3];
      ed.push_back({std::min(a, b), std::max(a, b)});
    }
  std::sort(ed.begin(), ed.end());
  ed.erase(std::unique(ed.begin(), ed.end()), ed.end());
  m.Ne = (int)ed.size();
  std::vector<int> edges(2 * ed.size());
  for (size_t k = 0; k < ed.size(); ++k) { edges[2 * k] = ed[k].first; edges[2 * k + 1] = ed[k].second; }
  // vertex -> incident (t, a) slots
  std::vector<int> vptr(n + 1, 0), vslot(4 * T);
  for (int64_t k = 0; k < 4 * T; ++k) vptr[tets[k] + 1]++;
  for (int64_t v = 0; v < n; ++v) vptr[v + 1] += vptr[v];
  {
    std::vector<int> fill(vptr.begin(), vptr.end() - 1);
    for (int64_t t = 0; t < T; ++t)
      for (int a = 0; a < 4; ++a) vslot[fill[tets[4 * t + a]]++] = (int)(t * 4 + a);
  }
  std::vector<int> tets_i(tets, tets + 4 * T);
  TRY(upload(ms, s, &m.rest, rest_xyz, 3 * n));
  TRY(upload(ms, s, &m.pinned, pinned, n));
  TRY(upload(ms, s, (int**)&m.tets, tets_i.data(), 4 * T));
  TRY(upload(ms, s, &m.vinc_ptr, vptr.data(), n + 1));
  TRY(upload(ms, s, &m.vinc_slot, vslot.data(), 4 * T));
  if (Ns > 0) {
    TRY(upload(ms, s, &m.Wptr, W_rowptr, Ns + 1));
    TRY(upload(ms, s, &m.Wcol, W_col, W_rowptr[Ns]));
    TRY(upload(ms, s, &m.Wval, W_val, W_rowptr[Ns]));
  } else {
    int64_t z = 0;
    TRY(upload(ms, s, &m.Wptr, &z, 1));
    TRY(dalloc(ms, &m.Wcol, 1));
    TRY(dalloc(ms, &m.Wval, 1));
  }
  TRY(upload(ms, s, &m.tris, proxy_tris, 3 * Nt));
  TRY(upload(ms, s, &m.edges, edges.data(), edges.size()));
  {
    double mx = 0.0;
    for (int64_t k = 0; k < 3 * n; ++k) mx = std::max(mx, std::fabs(rest_xyz[k]));
    m.coord_scale = 2.0 * std::max(mx, 1e-30);
    // mean proxy edge length at rest (the default skin of the contact list)
    std::vector<double> sr(3 * (size_t)std::max<int64_t>(Ns, 1), 0.0);
    for (int64_t r = 0; r < Ns; ++r)
      for (int64_t e = W_rowptr[r]; e < W_rowptr[r + 1]; ++e)
        for (int d = 0; d < 3; ++d) sr[3 * r + d] += W_val[e] * rest_xyz[3 * (int64_t)W_col[e] + d];
    double sum = 0.0;
    std::vector<double> el2(std::max<size_t>(ed.size(), 1), 0.0);
    for (size_t k = 0; k < ed.size(); ++k) {
      double l2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double q = sr[3 * ed[k].first + d] - sr[3 * ed[k].second + d];
        l2 += q * q;
      }
      el2[k] = l2;
      sum += std::sqrt(l2);
    }
    ms.mean_edge = ed.empty() ? 0.0 : sum / (double)ed.size();
    TRY(upload(ms, s, &m.elen2, el2.data(), el2.size()));
  }
  m.n_partials = std::max(elastic_blocks(m.T), gnorm_blocks(m.n)) + 16;
  CK(cudaStreamSynchronize(s));
  ctx->meshes.push_back(std::move(msp));
  *mesh_id = (int)ctx->meshes.size() - 1;
  return FSIM_OK;
}

fsim_status fsim_prefactor(fsim_ctx_t ctx, int mesh_id, const fsim_params* p) {
  MeshState* msp = get_mesh(ctx, mesh_id);
  if (!msp || !p || !(p->dhat > 0.0) || !(p->weight_scale > 0.0) || p->max_iters < 0 ||
      p->max_ls < 0 || !(p->ccd_s > 0.0 && p->ccd_s < 1.0) || p->accd_max_iters <= 0 ||
      p->coop_ctas < 0 || (p->solver != FSIM_SOLVER_WOODBURY && p->solver != FSIM_SOLVER_PCG &&
       p->solver != FSIM_SOLVER_SCHUR) ||
      (p->solver == FSIM_SOLVER_PCG && (p->cg_max_iters <= 0 || !(p->cg_tol > 0.0))))
    return FSIM_EINVAL;
  if (msp->prefactored) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  MeshState& ms = *msp;
  DevMesh& m = ms.d;
  cudaStream_t s = ctx->stream;
  ms.p = *p;
  std::vector<double> dminv, w;
  tet_rest_data(ms.rest.data(), ms.tets.data(), m.T, p->weight_scale, dminv, w);
  for (double wt : w)
    if (!(wt > 0.0) || !std::isfinite(wt)) return FSIM_EINVAL;   // degenerate tet
  HostFactor f;
  int rc = build_factor(m.n, ms.rest.data(), ms.tets.data(), m.T, dminv, w, ms.pinned.data(),
                        ms.x2mask, f);
  if (rc != FSIM_OK) return rc;
  ms.kappa = p->kappa > 0.0 ? p->kappa : f.kappa_auto;
  ms.factor_nnz = f.factor_nnz;
  m.nf = f.n_free; m.n1 = f.n1; m.n2 = f.n2;
  TRY(upload(ms, s, &m.dminv, dminv.data(), dminv.size()));
  {   // Dm^-1 as float pairs (hi, lo) for the mixed local step
    std::vector<float2> dd(dminv.size());
    for (size_t k = 0; k < dminv.size(); ++k) {
      const float h = (float)dminv[k];
      dd[k] = make_float2(h, (float)(dminv[k] - (double)h));
    }
    TRY(upload(ms, s, &m.dminv_df, dd.data(), dd.size()));
  }
  TRY(upload(ms, s, &m.w, w.data(), w.size()));
  {   // w as float pairs for the mixed local step
    std::vector<float2> wd(w.size());
    for (size_t k = 0; k < w.size(); ++k) {
      const float h = (float)w[k];
      wd[k] = make_float2(h, (float)(w[k] - (double)h));
    }
    TRY(upload(ms, s, &m.w_df, wd.data(), wd.size()));
  }
  TRY(upload(ms, s, &m.perm, f.perm.data(), f.perm.size()));
  TRY(upload(ms, s, &m.pos, f.pos.data(), f.pos.size()));
  std::vector<int> x2of(m.n, -1);
  for (int q = 0; q < m.n2; ++q) x2of[f.perm[m.n1 + q]] = q;
  TRY(upload(ms, s, &m.x2of, x2of.data(), x2of.size()));
  // supernodes
  const int nsn = (int)f.sn.size();
  m.n_sn = nsn;
  m.n_levels = f.n_levels;
  std::vector<int> c0(nsn), ns(nsn), nr1(nsn);
  std::vector<int64_t> roff(nsn), zoff(nsn);
  m.max_ns = 1; m.max_ld = 1;
  for (int j = 0; j < nsn; ++j) {
    c0[j] = f.sn[j].c0; ns[j] = f.sn[j].ns; nr1[j] = f.sn[j].nr;   // all rows (x1 and x2)
    roff[j] = f.sn[j].rows_off; zoff[j] = f.sn[j].z_off;
    m.max_ns = std::max(m.max_ns, ns[j]);
    m.max_ld = std::max(m.max_ld, ns[j] + nr1[j]);
  }
  if (3 * (size_t)m.max_ld * sizeof(double) > 200 * 1024) return FSIM_EINVAL;
  TRY(upload(ms, s, &m.sn_c0, c0.data(), nsn));
  TRY(upload(ms, s, &m.sn_ns, ns.data(), nsn));
  TRY(upload(ms, s, &m.sn_nr1, nr1.data(), nsn));
  TRY(upload(ms, s, &m.sn_roff, roff.data(), nsn));
  TRY(upload(ms, s, &m.sn_zoff, zoff.data(), nsn));
  TRY(upload(ms, s, &m.sn_rows, f.rows.data(), f.rows.size()));
  TRY(upload(ms, s, &m.Z, f.Z.data(), f.Z.size()));
  {
    std::vector<float> zf(f.Z.begin(), f.Z.end());
    TRY(upload(ms, s, &m.Zf, zf.data(), zf.size()));
    CK(cudaStreamSynchronize(s));
  }
  TRY(upload(ms, s, &m.level_sn, f.level_sn.data(), f.level_sn.size()));
  m.h_level_ptr = new int[f.n_levels + 1];
  m.h_level_maxns = new int[std::max(f.n_levels, 1)];
  m.h_level_maxld = new int[std::max(f.n_levels, 1)];
  m.h_fwd_ptr = new int[f.n_levels + 1];
  m.h_bwd_ptr = new int[f.n_levels + 1];
  m.h_bwd32_ptr = new int[f.n_levels + 1];
  // work items: forward = 32-row chunks of Z_J, backward = 8-column chunks
  // (32-column chunks for the multi-right-hand-side backward solve)
  std::vector<int4> fwd, bwd, bwd32;
  m.h_fwd_ptr[0] = 0;
  m.h_bwd_ptr[0] = 0;
  m.h_bwd32_ptr[0] = 0;
  for (int l = 0; l <= f.n_levels; ++l) m.h_level_ptr[l] = f.level_ptr[l];
  for (int l = 0; l < f.n_levels; ++l) {
    int mx = 1, mxld = 1;
    for (int k = f.level_ptr[l]; k < f.level_ptr[l + 1]; ++k) {
      const int J = f.level_sn[k];
      const int ldj = ns[J] + nr1[J];
      mx = std::max(mx, ns[J]);
      mxld = std::max(mxld, ldj);
      for (int r0 = 0; r0 < ldj; r0 += 32) fwd.push_back(make_int4(J, r0, std::min(32, ldj - r0), 0));
      for (int k0 = 0; k0 < ns[J]; k0 += 8) bwd.push_back(make_int4(J, k0, std::min(8, ns[J] - k0), 0));
      // 32 columns and up to kBwdRowSplit rows each: the long row ranges of
      // the top supernodes spread over many CTAs (partial sums added atomically)
      for (int k0 = 0; k0 < ns[J]; k0 += 32)
        for (int rb = k0; rb < ldj; rb += kBwdRowSplit)
          bwd32.push_back(make_int4(J, k0, std::min(32, ns[J] - k0), rb));
    }
    m.h_level_maxns[l] = mx;
    m.h_level_maxld[l] = mxld;
    m.h_fwd_ptr[l + 1] = (int)fwd.size();
    m.h_bwd_ptr[l + 1] = (int)bwd.size();
    m.h_bwd32_ptr[l + 1] = (int)bwd32.size();
  }
  TRY(upload(ms, s, &m.fwd_items, fwd.data(), fwd.size()));
  TRY(upload(ms, s, &m.bwd_items, bwd.data(), bwd.size()));
  TRY(upload(ms, s, &m.bwd_items32, bwd32.data(), bwd32.size()));
  TRY(upload(ms, s, &m.Sinv, f.sigma_inv.data(), f.sigma_inv.size()));
  if (p->solver == FSIM_SOLVER_SCHUR && !f.sigma.empty())
    TRY(upload(ms, s, &m.Sig, f.sigma.data(), f.sigma.size()));
  {
    std::vector<float> sf(f.sigma_inv.begin(), f.sigma_inv.end());
    TRY(upload(ms, s, &m.Sinvf, sf.data(), sf.size()));
    // TF32 head and tail of Sigma^-1 for the tensor-core product of batches
    if (m.n2 > 0) {
      std::vector<float> hi, lo;
      tc_split_sinv(f.sigma_inv.data(), m.n2, hi, lo, &m.sinv_ld);
      TRY(upload(ms, s, &m.sinv_hi, hi.data(), hi.size()));
      TRY(upload(ms, s, &m.sinv_lo, lo.data(), lo.size()));
      ms.tc_maps.assign((tc_map_bytes() + 7) / 8 + 8, 0);
      // 64-byte aligned view of the storage for the descriptors
      uint64_t* base = ms.tc_maps.data();
      while (((uintptr_t)base & 63) != 0) ++base;
      m.tc_maps = tc_encode_sinv(m.sinv_hi, m.sinv_lo, m.n2, m.sinv_ld, base) == 0 ? base : nullptr;
    }
    CK(cudaStreamSynchronize(s));
  }
  m.cap = p->contact_capacity > 0 ? p->contact_capacity
                                  : std::max<int64_t>(1 << 20, 256 * (int64_t)std::max(m.Nt, 1));
  {   // K in vertex order for the CG operator (rows of pinned vertices empty)
    std::vector<int> kp(m.n + 1, 0), kc;
    std::vector<double> kv;
    std::vector<int> rowlen(m.n, 0);
    for (int q = 0; q < m.nf; ++q) rowlen[f.perm[q]] = f.k_ptr[q + 1] - f.k_ptr[q];
    for (int v = 0; v < m.n; ++v) kp[v + 1] = kp[v] + rowlen[v];
    kc.resize(kp[m.n]);
    kv.resize(kp[m.n]);
    for (int q = 0; q < m.nf; ++q) {
      int o = kp[f.perm[q]];
      for (int e = f.k_ptr[q]; e < f.k_ptr[q + 1]; ++e, ++o) {
        kc[o] = f.perm[f.k_col[e]];
        kv[o] = f.k_val[e];
      }
    }
    TRY(upload(ms, s, &m.kv_ptr, kp.data(), kp.size()));
    TRY(upload(ms, s, &m.kv_col, kc.data(), kc.size()));
    TRY(upload(ms, s, &m.kv_val, kv.data(), kv.size()));
    CK(cudaStreamSynchronize(s));
  }
  m.skin = p->skin > 0.0 ? p->skin : std::max(10.0 * p->dhat, 0.25 * ms.mean_edge);
  m.one_cta_max = p->reduced_one_cta_max > 0 ? std::min(p->reduced_one_cta_max, 96) : 96;
  m.barrier_lanes = p->barrier_lane_per_pair != 0 ? 1 : 0;
  m.ee_moll = p->ee_mollifier ? 1 : 0;
  m.cap_act = p->active_capacity > 0 ? p->active_capacity
                                     : std::max<int64_t>(1 << 16, 16 * (int64_t)std::max(m.Nt, 1));
  m.cap_act = std::min(m.cap_act, m.cap);
  if (m.cap >= (1LL << 31)) return FSIM_EINVAL;
  TRY(dalloc(ms, &ms.gtmp, 3 * (size_t)m.n));
  TRY(dalloc(ms, &ms.dxtmp, 3 * (size_t)m.n));
  ms.ws_bytes = 0;
  TRY(alloc_workspace(ms, m, ms.allocs, &ms.ws_bytes));
  if (m.n1 > 0 && m.n2 > 0) {   // Phi = K11^-1 K12 Sigma^-1 for the mixed global step
    TRY(dalloc(ms, &m.Phi_t, (size_t)m.n1 * m.n2));
    CK(compute_phi(s, m, m.Phi_t));
  }
  CK(cudaMemcpyAsync(m.x, m.rest, sizeof(double) * 3 * (size_t)m.n, cudaMemcpyDeviceToDevice, s));
  {
    Exec ex = ctx_exec(ctx, ms);
    TRY(ensure_reduced(ex, m, std::min(std::max(m.n2, 1), 64)));
  }
  CK(cudaStreamSynchronize(s));
  ms.prefactored = true;
  return FSIM_OK;
}

fsim_status fsim_set_actuation(fsim_ctx_t ctx, int mesh_id, const double* fiber, const double* stretch) {
  MeshState* msp = get_mesh(ctx, mesh_id);
  if (!msp || !fiber || !stretch) return FSIM_EINVAL;
  if (!msp->prefactored) return FSIM_ENOT_READY;
  const int T = msp->d.T;
  for (int t = 0; t < T; ++t) {
    const double a = stretch[t];
    const double f2 = fiber[3 * t] * fiber[3 * t] + fiber[3 * t + 1] * fiber[3 * t + 1] +
                      fiber[3 * t + 2] * fiber[3 * t + 2];
    if (!(a > 0.0) || !std::isfinite(a) || !(f2 > 0.0) || !std::isfinite(f2)) return FSIM_ENONFINITE;
  }
  cudaSetDevice(ctx->device);
  DevMesh& m = msp->d;
  cudaStream_t s = ctx->stream;
  // staging: fiber into tetf (>= 3T doubles), stretch into tetf_t
  CK(cudaMemcpyAsync(m.tetf, fiber, sizeof(double) * 3 * (size_t)T, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m.tetf_t, stretch, sizeof(double) * (size_t)T, cudaMemcpyHostToDevice, s));
  launch_actuation(s, T, m.tetf, m.tetf_t, m.act, m.act_df);
  CK(cudaStreamSynchronize(s));
  msp->actuated = true;
  return FSIM_OK;
}

fsim_status fsim_set_actuation_dev(fsim_ctx_t ctx, int mesh_id, const double* fiber_dev,
                                   const double* stretch_dev) {
  MeshState* msp = get_mesh(ctx, mesh_id);
  if (!msp || !fiber_dev || !stretch_dev) return FSIM_EINVAL;
  if (!msp->prefactored) return FSIM_ENOT_READY;
  cudaSetDevice(ctx->device);
  launch_actuation(ctx->stream, msp->d.T, fiber_dev, stretch_dev, msp->d.act, msp->d.act_df);
  CK(cudaGetLastError());
  msp->actuated = true;
  return FSIM_OK;
}

fsim_status fsim_get_stream(fsim_ctx_t ctx, void** stream) {
  if (!ctx || !stream) return FSIM_EINVAL;
  *stream = (void*)ctx->stream;
  return FSIM_OK;
}

fsim_status fsim_profile(fsim_ctx_t ctx, uint32_t class_mask) {
  if (!ctx) return FSIM_EINVAL;
  prof_set_mask(class_mask);
  return FSIM_OK;
}

fsim_status fsim_profile_read(fsim_ctx_t ctx, int kernel_class, int64_t* launches, double* total_ms) {
  if (!ctx || !launches || !total_ms) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  return prof_read(kernel_class, launches, total_ms) == 0 ? FSIM_OK : FSIM_EINVAL;
}

fsim_status fsim_profile_reset(fsim_ctx_t ctx) {
  if (!ctx) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  prof_reset();
  return FSIM_OK;
}

static int ready(MeshState* ms) {
  if (!ms) return FSIM_EINVAL;
  if (!ms->prefactored || !ms->actuated) return FSIM_ENOT_READY;
  return FSIM_OK;
}

fsim_status fsim_solve_frame(fsim_ctx_t ctx, int mesh_id, const double* x_init, int precision,
                             fsim_frame_stats* stats) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (precision != FSIM_FP64 && precision != FSIM_MIXED) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  const Exec ex = ctx_exec(ctx, *ms);
  const int rc = solve_frame_impl(ex, *ms, ms->d, x_init, false, precision, stats);
  ms->has_x = true;
  return rc;
}

fsim_status fsim_solve_frame_dev(fsim_ctx_t ctx, int mesh_id, const double* x_init_dev,
                                 int precision, fsim_frame_stats* stats) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (precision != FSIM_FP64 && precision != FSIM_MIXED) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  const Exec ex = ctx_exec(ctx, *ms);
  const int rc = solve_frame_impl(ex, *ms, ms->d, x_init_dev, true, precision, stats);
  ms->has_x = true;
  return rc;
}

fsim_status fsim_read_positions(fsim_ctx_t ctx, int mesh_id, double* xyz_out) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  if (!ms || !xyz_out) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  CK(cudaMemcpyAsync(xyz_out, ms->d.x, sizeof(double) * 3 * (size_t)ms->d.n, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FSIM_OK;
}

fsim_status fsim_read_positions_dev(fsim_ctx_t ctx, int mesh_id, double* xyz_out_dev) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  if (!ms || !xyz_out_dev) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  CK(cudaMemcpyAsync(xyz_out_dev, ms->d.x, sizeof(double) * 3 * (size_t)ms->d.n,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FSIM_OK;
}

static int copy_keys(fsim_ctx_t ctx, MeshState& ms, int64_t np, int32_t* keys, int64_t cap,
                     int64_t* count) {
  std::vector<unsigned long long> k(np);
  if (np > 0) {
    CK(cudaMemcpyAsync(k.data(), ms.d.pairs, sizeof(unsigned long long) * np, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  std::sort(k.begin(), k.end());
  *count = np;
  if (np > cap) return FSIM_ECONTACT_OVERFLOW;
  for (int64_t q = 0; q < np; ++q) {
    keys[3 * q] = (int32_t)(k[q] >> 62);
    keys[3 * q + 1] = (int32_t)((k[q] >> 31) & 0x7fffffffULL);
    keys[3 * q + 2] = (int32_t)(k[q] & 0x7fffffffULL);
  }
  return FSIM_OK;
}

fsim_status fsim_read_contacts(fsim_ctx_t ctx, int mesh_id, int32_t* keys, int64_t cap, int64_t* count) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (!count || (cap > 0 && !keys)) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  DevMesh& m = ms->d;
  const Exec ex = ctx_exec(ctx, *ms);
  TRY(evaluate(ex, *ms, m, m.x, m.st, m.tetf_t, nullptr, 0, ms->kappa));
  TRY(sync_read(ex, m));
  if (ctx->h_counters[2]) return FSIM_ECONTACT_OVERFLOW;
  return copy_keys(ctx, *ms, ctx->h_counters[0], keys, cap, count);
}

// ---- step-level entry points ------------------------------------------------
static int stage_x(fsim_ctx_t ctx, MeshState& ms, const double* x) {
  DevMesh& m = ms.d;
  CK(cudaMemcpyAsync(m.xt, x, sizeof(double) * 3 * (size_t)m.n, cudaMemcpyHostToDevice, ctx->stream));
  return FSIM_OK;
}

fsim_status fsim_eval_elastic(fsim_ctx_t ctx, int mesh_id, const double* x, int precision,
                              double* energy_out, double* grad_out, double* proj_out) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (!x || (precision != 0 && precision != 1)) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  DevMesh& m = ms->d;
  cudaStream_t s = ctx->stream;
  TRY(stage_x(ctx, *ms, x));
  if (proj_out && !ms->proj) TRY(dalloc(*ms, &ms->proj, 9 * (size_t)m.T));
  launch_elastic(s, m, m.xt, m.tetf_t, proj_out ? ms->proj : nullptr, m.partials, precision);
  launch_sum_partials(s, m.partials, elastic_blocks(m.T), m.scal + 2);
  launch_gather_forces(s, m, m.tetf_t, ms->gtmp, precision);
  TRY(sync_read(ctx_exec(ctx, *ms), m));
  if (energy_out) *energy_out = ctx->h_scal[2];
  if (grad_out)
    CK(cudaMemcpy(grad_out, ms->gtmp, sizeof(double) * 3 * (size_t)m.n, cudaMemcpyDeviceToHost));
  if (proj_out)
    CK(cudaMemcpy(proj_out, ms->proj, sizeof(double) * 9 * (size_t)m.T, cudaMemcpyDeviceToHost));
  return FSIM_OK;
}

fsim_status fsim_eval_proxy(fsim_ctx_t ctx, int mesh_id, const double* x, double* s_out) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  if (!ms || !x || !s_out) return FSIM_EINVAL;
  if (!ms->prefactored) return FSIM_ENOT_READY;
  cudaSetDevice(ctx->device);
  DevMesh& m = ms->d;
  TRY(stage_x(ctx, *ms, x));
  launch_proxy(ctx->stream, m, m.xt, m.st);
  CK(cudaMemcpyAsync(s_out, m.st, sizeof(double) * 3 * (size_t)m.Ns, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FSIM_OK;
}

fsim_status fsim_eval_contacts(fsim_ctx_t ctx, int mesh_id, const double* x, int32_t* keys,
                               int64_t cap, int64_t* count, double* barrier_energy_out) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (!x || !count || (cap > 0 && !keys)) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  DevMesh& m = ms->d;
  TRY(stage_x(ctx, *ms, x));
  const Exec ex = ctx_exec(ctx, *ms);
  TRY(evaluate(ex, *ms, m, m.xt, m.st, m.tetf_t, nullptr, 0, ms->kappa));
  TRY(sync_read(ex, m));
  if (ctx->h_counters[2]) return FSIM_ECONTACT_OVERFLOW;
  if (barrier_energy_out) *barrier_energy_out = ctx->h_scal[0];
  return copy_keys(ctx, *ms, ctx->h_counters[0], keys, cap, count);
}

fsim_status fsim_eval_barrier(fsim_ctx_t ctx, int mesh_id, const double* x, double* grad_out,
                              int32_t* n_c, int32_t* c_out, double* bcheck_out, int64_t bcheck_cap) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (!x) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  DevMesh& m = ms->d;
  cudaStream_t s = ctx->stream;
  TRY(stage_x(ctx, *ms, x));
  const Exec ex = ctx_exec(ctx, *ms);
  TRY(evaluate(ex, *ms, m, m.xt, m.st, m.tetf_t, nullptr, 0, ms->kappa));
  TRY(sync_read(ex, m));
  if (ctx->h_counters[2]) return FSIM_ECONTACT_OVERFLOW;
  const int64_t np = ctx->h_counters[0];
  // barrier gradient only: zero elastic forces by gathering a zero tetf
  CK(cudaMemsetAsync(m.tetf_t, 0, sizeof(double) * 12 * (size_t)m.T, s));
  int nc = 0;
  double gn2 = 0.0;
  TRY(gradient_and_hessian(ex, *ms, m, m.st, m.tetf_t, ms->gtmp, np, 0, &nc, &gn2, ms->kappa));
  if (n_c) *n_c = nc;
  if (grad_out)
    CK(cudaMemcpy(grad_out, ms->gtmp, sizeof(double) * 3 * (size_t)m.n, cudaMemcpyDeviceToHost));
  if (c_out && nc > 0) CK(cudaMemcpy(c_out, m.clist, sizeof(int) * nc, cudaMemcpyDeviceToHost));
  if (bcheck_out) {
    if ((int64_t)9 * nc * nc > bcheck_cap) return FSIM_EINVAL;
    if (nc > 0)
      CK(cudaMemcpy(bcheck_out, m.Bc, sizeof(double) * 9 * (size_t)nc * nc, cudaMemcpyDeviceToHost));
  }
  return FSIM_OK;
}

fsim_status fsim_check_status(fsim_ctx_t ctx, int32_t* enabled, uint64_t* word) {
  if (!ctx || !enabled || !word) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return FSIM_ECUDA;
#ifdef FSIM_CHECK
  *enabled = 1;
#else
  *enabled = 0;
#endif
  uint64_t w = 0;
  for (uint64_t v : {check_word_local(), check_word_solve(), check_word_reduced()})
    if (w == 0 && v != 0) w = v;
  *word = w;
  return FSIM_OK;
}

fsim_status fsim_eval_sigma_inv_mr(fsim_ctx_t ctx, int mesh_id, const double* y, int32_t ncols,
                                   int32_t tensor_cores, double* u_out) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  if (!ms) return FSIM_EINVAL;
  if (!ms->prefactored) return FSIM_ENOT_READY;
  DevMesh& m = ms->d;
  if (!y || !u_out || ncols < 1 || ncols > 192 || m.n2 <= 0) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  const int n2 = m.n2, nr = (ncols + 31) / 32 * 32;
  if (tensor_cores && !tc_sinv_supported(m, nr)) return FSIM_EINVAL;
  std::vector<float> yf((size_t)n2 * nr, 0.f);
  for (int i = 0; i < n2; ++i)
    for (int c = 0; c < ncols; ++c) yf[(size_t)i * nr + c] = (float)y[(size_t)i * ncols + c];
  float *dy = nullptr, *du = nullptr;
  int* derr = nullptr;
  auto release = [&]() {
    if (dy) cudaFree(dy);
    if (du) cudaFree(du);
    if (derr) cudaFree(derr);
  };
  if (cudaMalloc(&dy, sizeof(float) * yf.size()) != cudaSuccess ||
      cudaMalloc(&du, sizeof(float) * yf.size()) != cudaSuccess ||
      cudaMalloc(&derr, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return FSIM_ENOMEM;
  }
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(dy, yf.data(), sizeof(float) * yf.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = tensor_cores ? launch_sinv_tc(s, m, dy, nr, du, ctx->num_sms, derr)
                     : launch_sinv_simt(s, m, dy, nr, du);
  if (e == cudaSuccess) e = cudaMemcpyAsync(yf.data(), du, sizeof(float) * yf.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess || herr) return FSIM_ECUDA;
  for (int i = 0; i < n2; ++i)
    for (int c = 0; c < ncols; ++c) u_out[(size_t)i * ncols + c] = (double)yf[(size_t)i * nr + c];
  return FSIM_OK;
}

fsim_status fsim_eval_global_step(fsim_ctx_t ctx, int mesh_id, const double* x, int precision,
                                  double* dx_out, int32_t* path_out) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (!x || !dx_out || (precision != 0 && precision != 1)) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  DevMesh& m = ms->d;
  cudaStream_t s = ctx->stream;
  TRY(stage_x(ctx, *ms, x));
  const Exec ex = ctx_exec(ctx, *ms);
  TRY(evaluate(ex, *ms, m, m.xt, m.st, m.tetf_t, nullptr, precision, ms->kappa));
  TRY(sync_read(ex, m));
  if (ctx->h_counters[2]) return FSIM_ECONTACT_OVERFLOW;
  const int64_t np = ctx->h_counters[0];
  int nc = 0;
  double gn2 = 0.0;
  TRY(gradient_and_hessian(ex, *ms, m, m.st, m.tetf_t, ms->gtmp, np, precision, &nc, &gn2, ms->kappa));
  CK(cudaMemsetAsync(m.counters + 6, 0, sizeof(int) * 2, s));
  if (ms->p.solver == FSIM_SOLVER_PCG) {
    int cg_it = 0;
    if (pcg_global_step(s, m, ms->gtmp, ms->dxtmp, ms->p.cg_tol, ms->p.cg_max_iters, m.counters + 6,
                        ex.coop_ctas, ex.h_scal + 6, &cg_it) != 0)
      return FSIM_ECUDA;
  } else {
    CK(global_step(s, m, ms->gtmp, ms->dxtmp, precision, m.counters + 6, ex.coop_ctas, ex.alone,
                   ms->p.solver == FSIM_SOLVER_SCHUR, nc));
  }
  TRY(sync_read(ex, m));
  if (ctx->h_counters[6]) return FSIM_ENOT_SPD;
  CK(cudaMemcpy(dx_out, ms->dxtmp, sizeof(double) * 3 * (size_t)m.n, cudaMemcpyDeviceToHost));
  if (path_out)
    *path_out = ms->p.solver == FSIM_SOLVER_WOODBURY ? reduced_path(nc, precision, m.one_cta_max)
                                                     : FSIM_REDUCED_UNUSED;
  return FSIM_OK;
}

fsim_status fsim_eval_ccd(fsim_ctx_t ctx, int mesh_id, const double* x, const double* dx,
                          double* alpha_out) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (!x || !dx || !alpha_out) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  DevMesh& m = ms->d;
  cudaStream_t s = ctx->stream;
  TRY(stage_x(ctx, *ms, x));
  CK(cudaMemcpyAsync(ms->dxtmp, dx, sizeof(double) * 3 * (size_t)m.n, cudaMemcpyHostToDevice, s));
  launch_proxy(s, m, m.xt, m.st);
  launch_proxy(s, m, ms->dxtmp, m.ds);
  launch_ccd_reset(s, m);
  launch_ccd(s, m, m.st, m.ds, ms->p.dhat, ms->p.ccd_s, ms->p.accd_max_iters);
  TRY(sync_read(ctx_exec(ctx, *ms), m));
  if (ctx->h_counters[9]) return FSIM_ECONTACT_OVERFLOW;
  *alpha_out = ctx->h_scal[1];
  return FSIM_OK;
}

fsim_status fsim_eval_energy(fsim_ctx_t ctx, int mesh_id, const double* x, int precision,
                             double* energy_out, double* grad_norm_out) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  TRY(ready(ms));
  if (!x || (precision != 0 && precision != 1)) return FSIM_EINVAL;
  cudaSetDevice(ctx->device);
  DevMesh& m = ms->d;
  TRY(stage_x(ctx, *ms, x));
  const Exec ex = ctx_exec(ctx, *ms);
  TRY(evaluate(ex, *ms, m, m.xt, m.st, m.tetf_t, nullptr, precision, ms->kappa));
  TRY(sync_read(ex, m));
  if (ctx->h_counters[2]) return FSIM_ECONTACT_OVERFLOW;
  const double E = ctx->h_scal[2] + ctx->h_scal[0];
  const int64_t np = ctx->h_counters[0];
  int nc = 0;
  double gn2 = 0.0;
  TRY(gradient_and_hessian(ex, *ms, m, m.st, m.tetf_t, ms->gtmp, np, 0, &nc, &gn2, ms->kappa));
  if (energy_out) *energy_out = E;
  if (grad_norm_out) *grad_norm_out = std::sqrt(gn2);
  return FSIM_OK;
}

fsim_status fsim_mesh_info_get(fsim_ctx_t ctx, int mesh_id, fsim_mesh_info* info) {
  MeshState* ms = get_mesh(ctx, mesh_id);
  if (!ms || !info) return FSIM_EINVAL;
  const DevMesh& m = ms->d;
  info->n = m.n; info->T = m.T; info->Ns = m.Ns; info->Nt = m.Nt; info->Ne = m.Ne;
  info->n_free = m.nf; info->n1 = m.n1; info->n2 = m.n2;
  info->factor_nnz = ms->factor_nnz;
  info->n_supernodes = m.n_sn;
  info->n_levels = m.n_levels;
  info->workspace_bytes = (int64_t)rt_slot_bytes(*ms);
  info->kappa = ms->kappa;
  return FSIM_OK;
}

}  // extern "C"
