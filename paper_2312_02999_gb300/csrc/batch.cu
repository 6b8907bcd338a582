// Lock-step batches of frame solves: Algorithm 1 for up to `cap` frames of
// one mesh at once, every stage of an iteration one launch for all frames.
//
// A single frame's iteration is a chain of about sixty small launches whose
// duration is set by latency (level-by-level triangular solves, a reduced
// system on one to four SMs, per-pair warps), so one frame leaves most of
// the GPU idle.  Here the frames of a batch advance together: the local
// step, constraint set, barrier derivatives, CCD and line-search trials of
// all frames run as batched launches over a device table of per-frame
// workspaces (blockIdx.y = frame), the triangular solves carry the right-hand
// sides of all frames as one multi-column pass over the factor, and the
// reduced systems of all frames run side by side in one launch per kernel.
// Frames converge at different iterations; a finished frame leaves the batch
// at the end of its iteration and the next pending request takes its slot
// (continuous batching at iteration granularity).  Every frame keeps its own
// iterate, step, line-search factor, stiffness and statistics, so its result
// is that of the same frame solved alone (up to the order of floating-point
// atomics).
//
// Host work per iteration: one read-back of all frames' status words after
// the gradient and one after each line-search trial, as in the single-frame
// loop.  The batch serves the mixed precision of the Woodbury global step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.h"
#include "runtime.h"
#include "batch.h"

using namespace fsim;

namespace {

#define BCK(call)                                                  \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      fprintf(stderr, "fsim: CUDA error %s at %s:%d\n",            \
              cudaGetErrorString(e_), __FILE__, __LINE__);         \
      return FSIM_ECUDA;                                           \
    }                                                              \
  } while (0)
#define BTRY(x)                   \
  do {                            \
    int s_ = (x);                 \
    if (s_ != FSIM_OK) return s_; \
  } while (0)

constexpr int kMaxBatchFrames = 64;        // frames per batch (multi-RHS columns 3 x 64)
constexpr double kKappaGrowBelow = 0.1;    // adaptive kappa, as in the single-frame loop
constexpr double kKappaMaxRatio = 100.0;

enum Phase { FREE = 0, INIT = 1, ITER = 2 };

struct Frame {
  BatchReq br;
  Phase phase = FREE;
  fsim_frame_stats st{};
  double E = 0.0, gn = 0.0, tol = 0.0, kappa = 0.0, d_prev = INFINITY, scale = 1.0;
  int nc = 0;
  int64_t npairs = 0;
  int trial = 0;            // line-search trials since the frame's last global step
  bool redone = false;      // this iteration's step was redone in float64
  bool fp64 = false;        // the frame's global steps use the float64 factors
};

template <typename T>
int dalloc_b(std::vector<void*>& allocs, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    return FSIM_ENOMEM;
  }
  allocs.push_back(*p);
  return FSIM_OK;
}

}  // namespace

namespace fsim {

class Batch {
 public:
  Batch(fsim_ctx_t ctx, MeshState& ms, int cap, cudaStream_t stream)
      : ctx_(ctx), ms_(ms), cap_(cap), s_(stream) {}
  ~Batch() { release(); }

  int init() {
    const DevMesh& m0 = ms_.d;
    nr_ = ((3 * cap_ + 31) / 32) * 32;
    if (!batch_supported(m0, nr_)) return FSIM_EINVAL;
    BCK(cudaStreamCreateWithFlags(&s2_, cudaStreamNonBlocking));
    for (auto& e : ev_) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    frames_.assign(cap_, Frame{});
    tab_.assign(cap_, DevMesh{});
    // per-frame workspaces; counters and scalars of all frames contiguous so
    // that one copy reads every frame's status back
    BTRY(dalloc_b(allocs_, &counters_, (size_t)kCounters * cap_));
    BTRY(dalloc_b(allocs_, &scal_, (size_t)kScal * cap_));
    BCK(cudaMemset(counters_, 0, sizeof(int) * kCounters * cap_));
    for (int f = 0; f < cap_; ++f) {
      DevMesh& m = tab_[f];
      m = m0;
      size_t bytes = 0;
      BTRY(rt_alloc_workspace(ms_, m, allocs_, &bytes));
      bytes_ += bytes + rt_reduced_bytes(std::min(std::max(m.n2, 1), 64));
      m.counters = counters_ + (size_t)kCounters * f;
      m.scal = scal_ + (size_t)kScal * f;
      m.col = f;
      m.active = 0;
      // the reduced systems of a batch run in one launch per kernel, so one
      // path for every 0 < n_c <= 128 (the 4-CTA clusters) keeps the one-CTA
      // and cluster launches from running one after the other; a mesh whose
      // reduced_one_cta_max was set keeps that split
      if (ms_.p.reduced_one_cta_max <= 0) m.one_cta_max = 0;
      Exec ex = exec();
      BTRY(rt_ensure_reduced(ex, m, std::min(std::max(m.n2, 1), 64)));
    }
    const size_t nf = (size_t)m0.nf;
    BTRY(dalloc_b(allocs_, &rb_, nf * nr_));
    BTRY(dalloc_b(allocs_, &yb_, (size_t)std::max(m0.n1, 1) * nr_));
    BTRY(dalloc_b(allocs_, &ub_, (size_t)std::max(m0.n2, 1) * nr_));
    BTRY(dalloc_b(allocs_, &bx_, nf * nr_));
    bytes_ += sizeof(float) * (2 * nf + std::max(m0.n1, 1) + std::max(m0.n2, 1)) * nr_;
    BCK(cudaMemset(rb_, 0, sizeof(float) * nf * nr_));
    BCK(cudaMemset(bx_, 0, sizeof(float) * nf * nr_));
    BTRY(dalloc_b(allocs_, &tab_dev_, (size_t)cap_));
    args_bytes_ = reduced_args_bytes();
    char* ad = nullptr;
    BTRY(dalloc_b(allocs_, &ad, args_bytes_ * cap_));
    args_dev_ = ad;
    args_host_.assign(args_bytes_ * cap_, 0);
    int* cols = nullptr;
    BTRY(dalloc_b(allocs_, &cols, (size_t)cap_));
    cols_dev_ = cols;
    double** x1s = nullptr;
    BTRY(dalloc_b(allocs_, &x1s, (size_t)cap_));
    x1s_dev_ = x1s;
    std::vector<int> hc(cap_);
    for (int f = 0; f < cap_; ++f) hc[f] = 3 * f;
    BCK(cudaMemcpy(cols, hc.data(), sizeof(int) * cap_, cudaMemcpyHostToDevice));
    BCK(cudaHostAlloc((void**)&h_tab_, sizeof(DevMesh) * cap_ * kTabRing, cudaHostAllocDefault));
    for (auto& e : ev_tab_) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    BCK(cudaHostAlloc((void**)&h_counters_, sizeof(int) * kCounters * cap_, cudaHostAllocDefault));
    BCK(cudaHostAlloc((void**)&h_scal_, sizeof(double) * kScal * cap_, cudaHostAllocDefault));
    BCK(cudaHostAlloc((void**)&h_x1s_, sizeof(double*) * cap_, cudaHostAllocDefault));
    BCK(cudaHostAlloc((void**)&h_args_, args_bytes_ * cap_, cudaHostAllocDefault));
    BCK(cudaDeviceSynchronize());
    return FSIM_OK;
  }

  size_t bytes() const { return bytes_; }

  // Solve requests until `pull` has none left and every slot is free.  At
  // every iteration boundary `pull` is asked for a request for each free
  // slot; `done` receives each finished request (after its positions have
  // reached x_host / x_out_dev) with its status and statistics.
  int run(const BatchPull& pull, const BatchDone& done) {
    done_ = &done;
    for (;;) {
      bool any_new = false;
      for (int f = 0; f < cap_; ++f) {
        if (frames_[f].phase != FREE) continue;
        BatchReq br;
        if (!pull(&br)) break;
        frames_[f].br = br;
        const int rc = start_frame(f);
        if (rc == FSIM_ECUDA) return rc;
        if (rc != FSIM_OK) { finish(f, rc, false); continue; }
        any_new = true;
      }
      if (any_new) BTRY(initial_state());
      BTRY(notify());
      bool any_iter = false;
      for (auto& fr : frames_) any_iter |= fr.phase == ITER;
      if (!any_iter) {
        bool any_busy = false;
        for (auto& fr : frames_) any_busy |= fr.phase != FREE;
        if (!any_busy && !any_new) break;
        continue;
      }
      BTRY(iterate());
      BTRY(notify());
    }
    BCK(cudaStreamSynchronize(s_));
    return notify();
  }

 private:
  Exec exec() const {
    Exec ex;
    ex.stream = s_;
    ex.h_counters = ctx_->h_counters;
    ex.h_scal = ctx_->h_scal;
    ex.coop_ctas = ctx_->num_sms;
    ex.alone = false;
    ex.allocs = const_cast<std::vector<void*>*>(&allocs_);
    ex.bytes = nullptr;
    return ex;
  }

  void release() {
    if (s_) cudaStreamSynchronize(s_);
    if (s2_) cudaStreamSynchronize(s2_);
    if (ev_done_) cudaEventDestroy(ev_done_);
    for (auto& e : ev_tab_)
      if (e) cudaEventDestroy(e);
    for (void* p : allocs_) cudaFree(p);
    allocs_.clear();
    for (auto& e : ev_)
      if (e) cudaEventDestroy(e);
    if (s2_) cudaStreamDestroy(s2_);
    if (h_tab_) cudaFreeHost(h_tab_);
    if (h_counters_) cudaFreeHost(h_counters_);
    if (h_scal_) cudaFreeHost(h_scal_);
    if (h_x1s_) cudaFreeHost(h_x1s_);
    if (h_args_) cudaFreeHost(h_args_);
    for (auto& m : tab_) {
      // the per-frame aux streams and events created by rt_alloc_workspace
      if (m.ev_fork) cudaEventDestroy(m.ev_fork);
      if (m.ev_join) cudaEventDestroy(m.ev_join);
      if (m.ev_fork2) cudaEventDestroy(m.ev_fork2);
      if (m.ev_join2) cudaEventDestroy(m.ev_join2);
      if (m.aux_stream) cudaStreamDestroy(m.aux_stream);
      m.ev_fork = m.ev_join = m.ev_fork2 = m.ev_join2 = nullptr;
      m.aux_stream = nullptr;
    }
  }

  // table upload with the active flags of `want` (per frame)
  // (the host copy comes from a ring of pinned tables: an asynchronous copy
  // reads its source when it runs, so a table is not rewritten before the
  // copy that reads it has completed)
  int upload_table(const std::vector<char>& want) {
    const int slot = tab_slot_;
    tab_slot_ = (tab_slot_ + 1) % kTabRing;
    BCK(cudaEventSynchronize(ev_tab_[slot]));
    DevMesh* h = h_tab_ + (size_t)cap_ * slot;
    for (int f = 0; f < cap_; ++f) {
      tab_[f].active = want[f] ? 1 : 0;
      tab_[f].kappa_f = frames_[f].kappa;
      tab_[f].ls_scale = frames_[f].scale;
      h[f] = tab_[f];
    }
    BCK(cudaMemcpyAsync(tab_dev_, h, sizeof(DevMesh) * cap_, cudaMemcpyHostToDevice, s_));
    BCK(cudaEventRecord(ev_tab_[slot], s_));
    return FSIM_OK;
  }

  int read_back() {
    BCK(cudaMemcpyAsync(h_counters_, counters_, sizeof(int) * kCounters * cap_,
                        cudaMemcpyDeviceToHost, s_));
    BCK(cudaMemcpyAsync(h_scal_, scal_, sizeof(double) * kScal * cap_, cudaMemcpyDeviceToHost, s_));
    BCK(cudaStreamSynchronize(s_));
    return FSIM_OK;
  }
  int* cnt(int f) { return h_counters_ + (size_t)kCounters * f; }
  double* scl(int f) { return h_scal_ + (size_t)kScal * f; }

  int start_frame(int f) {
    Frame& fr = frames_[f];
    const BatchReq br = fr.br;
    fr = Frame{};
    fr.br = br;
    const fsim_request& q = br.req;
    fr.st.alpha_min = 1.0;
    tab_[f].bar64 = 0;
    fr.kappa = ms_.kappa;
    DevMesh& m = tab_[f];
    const size_t n = (size_t)m.n, T = (size_t)m.T;
    const bool dev = (q.flags & FSIM_REQ_DEVICE) != 0;
    if (q.mesh_id < 0 || rt_mesh(ctx_, q.mesh_id) != &ms_ || q.precision != FSIM_MIXED)
      return FSIM_EINVAL;
    if (dev) {
      launch_actuation(s_, m.T, q.fiber, q.stretch, m.act, m.act_df);
    } else {
      for (size_t t = 0; t < T; ++t) {
        const double a = q.stretch[t];
        const double f2 = q.fiber[3 * t] * q.fiber[3 * t] + q.fiber[3 * t + 1] * q.fiber[3 * t + 1] +
                          q.fiber[3 * t + 2] * q.fiber[3 * t + 2];
        if (!(a > 0.0) || !std::isfinite(a) || !(f2 > 0.0) || !std::isfinite(f2)) return FSIM_ENONFINITE;
      }
      BCK(cudaMemcpyAsync(m.tetf, q.fiber, sizeof(double) * 3 * T, cudaMemcpyHostToDevice, s_));
      BCK(cudaMemcpyAsync(m.tetf_t, q.stretch, sizeof(double) * T, cudaMemcpyHostToDevice, s_));
      launch_actuation(s_, m.T, m.tetf, m.tetf_t, m.act, m.act_df);
    }
    const double* x0 = q.x_init ? q.x_init : m.rest;
    const cudaMemcpyKind kind =
        (q.x_init && !dev) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    BCK(cudaMemcpyAsync(m.x, x0, sizeof(double) * 3 * n, kind, s_));
    launch_reset_pinned(s_, m, m.x);
    BCK(cudaMemsetAsync(m.counters + 4, 0, sizeof(int), s_));
    launch_check_finite(s_, 3 * m.n, m.x, m.counters + 4);
    fr.phase = INIT;
    return FSIM_OK;
  }

  // The frame's result is queued for copy-out; the request is reported to
  // `done` at the next synchronisation (notify), when the copies are complete.
  void finish(int f, int rc, bool copy = true) {
    Frame& fr = frames_[f];
    fr.st.status = rc;
    if (copy) {
      fr.st.grad_norm = fr.gn;
      fr.st.energy = fr.E;
      fr.st.contacts = fr.npairs;
      DevMesh& m = tab_[f];
      const size_t bytes = sizeof(double) * 3 * (size_t)m.n;
      if (fr.br.req.x_out_dev)
        cudaMemcpyAsync(fr.br.req.x_out_dev, m.x, bytes, cudaMemcpyDeviceToDevice, s_);
      if (fr.br.x_host) cudaMemcpyAsync(fr.br.x_host, m.x, bytes, cudaMemcpyDeviceToHost, s_);
    }
    finished_.push_back({fr.br.user, rc, fr.st});
    fr.phase = FREE;
  }

  int notify() {
    if (finished_.empty()) return FSIM_OK;
    BCK(cudaStreamSynchronize(s_));
    for (const auto& d : finished_) (*done_)(d.user, d.rc, d.st);
    finished_.clear();
    return FSIM_OK;
  }

  void adapt_kappa(Frame& fr, double d_min, double* Eb) {
    if (!ms_.p.adaptive_kappa) return;
    if (d_min < kKappaGrowBelow * ms_.p.dhat && d_min < fr.d_prev &&
        2.0 * fr.kappa <= kKappaMaxRatio * ms_.kappa) {
      fr.kappa *= 2.0;
      *Eb *= 2.0;
      fr.st.kappa_doublings++;
    }
    fr.d_prev = d_min;
  }

  // one evaluation (local step, s, constraint set) of the frames in `want`
  // at x (at = 0) or the trial point (at = 1)
  int evaluate(const std::vector<char>& want, int at) {
    BTRY(upload_table(want));
    const DevMesh& m0 = tab_[0];
    launch_eval_reset_b(s_, tab_dev_, cap_);
    if (at) launch_axpy_b(s_, tab_dev_, cap_, m0);
    launch_local_b(s_, tab_dev_, cap_, m0, at);
    launch_proxy_b(s_, tab_dev_, cap_, m0, at);
    launch_detect_b(s_, tab_dev_, cap_, m0, at, ms_.p.dhat);
    BCK(cudaGetLastError());
    return FSIM_OK;
  }

  // gradient, n_c, B-check and |g|^2 of the frames in `want` (at x)
  int gradient(const std::vector<char>& want) {
    BTRY(upload_table(want));
    const DevMesh& m0 = tab_[0];
    int64_t np_max = 0;
    for (int f = 0; f < cap_; ++f)
      if (want[f]) np_max = std::max(np_max, frames_[f].npairs);
    launch_gather_forces_b(s_, tab_dev_, cap_, m0);
    launch_barrier_b(s_, tab_dev_, cap_, m0, np_max, ms_.p.dhat);
    launch_gnorm2_b(s_, tab_dev_, cap_, m0);
    BCK(cudaGetLastError());
    BTRY(read_back());
    Exec ex = exec();
    for (int f = 0; f < cap_; ++f) {
      if (!want[f]) continue;
      Frame& fr = frames_[f];
      DevMesh& m = tab_[f];
      const int nc = cnt(f)[3];
      const int cap_now = m.Bc != nullptr ? m.nc_cap : 0;
      BTRY(rt_ensure_reduced(ex, m, std::max(nc, 1)));
      if (nc > cap_now) {          // buffers grew: assemble B-check again (one frame)
        BCK(cudaMemsetAsync(m.Bc, 0, sizeof(double) * 9 * (size_t)nc * nc, s_));
        BCK(cudaMemsetAsync(m.bocc, 0, sizeof(int) * (size_t)nc * nc, s_));
        launch_barrier_scatter(s_, m, fr.npairs, m.nc_cap, 2, m.g);
      }
      fr.nc = nc;
      fr.gn = std::sqrt(scl(f)[3]);
    }
    return FSIM_OK;
  }

  // first evaluation and gradient of newly admitted frames
  int initial_state() {
    std::vector<char> want(cap_, 0);
    for (int f = 0; f < cap_; ++f) want[f] = frames_[f].phase == INIT;
    BTRY(evaluate(want, 0));
    BTRY(read_back());
    std::vector<char> grad(cap_, 0);
    for (int f = 0; f < cap_; ++f) {
      if (!want[f]) continue;
      Frame& fr = frames_[f];
      int rc = FSIM_OK;
      if (cnt(f)[4]) rc = FSIM_ENONFINITE;
      else if (cnt(f)[5]) rc = FSIM_EINTERSECTING;
      else if (cnt(f)[2]) rc = FSIM_ECONTACT_OVERFLOW;
      fr.npairs = cnt(f)[0];
      double Eb = scl(f)[0];
      adapt_kappa(fr, scl(f)[4], &Eb);
      fr.E = scl(f)[2] + Eb;
      if (rc != FSIM_OK) { finish(f, rc); continue; }
      grad[f] = 1;
    }
    BTRY(gradient(grad));
    for (int f = 0; f < cap_; ++f) {
      if (!grad[f]) continue;
      Frame& fr = frames_[f];
      fr.st.grad_norm0 = fr.gn;
      fr.tol = std::max(ms_.p.tol_abs, ms_.p.tol_rel * fr.gn);
      fr.phase = ITER;
      if (!std::isfinite(fr.gn)) finish(f, FSIM_ENONFINITE);
    }
    return FSIM_OK;
  }

  // The single-frame float64 global step (Eq. 8-11) and CCD bound of frame f
  // on its own workspace, on the batch's stream.  With `hessian` (the frame's
  // first float64 step) the frame's contact Hessian is first assembled again
  // at x with float64 pair eigen-solves, as it is for the rest of the frame;
  // x is evaluated again because the trial evaluation replaced its pair list.
  int redo_fp64(int f, bool hessian) {
    DevMesh& m = tab_[f];
    const fsim_params& p = ms_.p;
    if (hessian) {
      m.bar64 = 1;
      std::vector<char> one(cap_, 0);
      one[f] = 1;
      BTRY(evaluate(one, 0));
      BTRY(read_back());
      BTRY(gradient(one));
    }
    BCK(cudaMemsetAsync(m.counters + 6, 0, sizeof(int) * 2, s_));
    BCK(global_step(s_, m, m.g, m.dx, FSIM_FP64, m.counters + 6, ctx_->num_sms, false, false,
                    frames_[f].nc));
    launch_proxy(s_, m, m.dx, m.ds);
    launch_ccd_reset(s_, m);
    launch_ccd(s_, m, m.s, m.ds, p.dhat, p.ccd_s, p.accd_max_iters);
    BCK(cudaGetLastError());
    return FSIM_OK;
  }

  int iterate() {
    NvtxRange nv("fsim.batch_iteration");
    const fsim_params& p = ms_.p;
    std::vector<char> act(cap_, 0);
    for (int f = 0; f < cap_; ++f) {
      Frame& fr = frames_[f];
      if (fr.phase != ITER) continue;
      fr.st.n_c = fr.nc;
      fr.st.n_c_max = std::max(fr.st.n_c_max, fr.nc);
      if (fr.gn <= fr.tol) { finish(f, FSIM_OK); continue; }
      if (fr.st.iterations >= p.max_iters) { finish(f, FSIM_ENOT_CONVERGED); continue; }
      act[f] = 1;
    }
    bool any = false;
    for (char a : act) any |= a != 0;
    if (!any) return FSIM_OK;
    // global step of every active frame: the batched mixed-precision step for
    // most, the single-frame float64 step for frames switched to float64
    std::vector<char> gact(cap_, 0);
    bool any_b = false;
    for (int f = 0; f < cap_; ++f) {
      gact[f] = act[f] && !frames_[f].fp64;
      any_b |= gact[f] != 0;
    }
    BTRY(upload_table(gact));
    std::vector<int> nc_host(cap_, 0);
    for (int f = 0; f < cap_; ++f) {
      reduced_args_fill(h_args_ + args_bytes_ * f, tab_[f], gact[f]);
      h_x1s_[f] = tab_[f].r;
      nc_host[f] = gact[f] ? frames_[f].nc : 0;
      if (act[f]) {
        Frame& fr = frames_[f];
        fr.st.sum_nc3 += (double)fr.nc * fr.nc * fr.nc;
        fr.st.reduced_steps[reduced_path(fr.nc, fr.fp64 ? FSIM_FP64 : FSIM_MIXED,
                                         tab_[f].one_cta_max)]++;
      }
    }
    BCK(cudaMemcpyAsync(args_dev_, h_args_, args_bytes_ * cap_, cudaMemcpyHostToDevice, s_));
    BCK(cudaMemcpyAsync(x1s_dev_, h_x1s_, sizeof(double*) * cap_, cudaMemcpyHostToDevice, s_));
    for (int f = 0; f < cap_; ++f)
      if (act[f]) BCK(cudaMemsetAsync(tab_[f].counters + 6, 0, sizeof(int) * 2, s_));
    BatchStep bs;
    bs.s = s_;
    bs.s2 = s2_;
    for (int k = 0; k < 4; ++k) bs.ev[k] = ev_[k];
    bs.tab = tab_dev_;
    bs.m0 = &tab_[0];
    bs.nb = cap_;
    bs.nr = nr_;
    bs.rb = rb_; bs.yb = yb_; bs.ub = ub_; bs.bx = bx_;
    bs.args_dev = args_dev_;
    bs.args_host = h_args_;
    bs.nc_host = nc_host.data();
    bs.cols_dev = cols_dev_;
    bs.x1s_dev = x1s_dev_;
    bs.num_sms = ctx_->num_sms;
    bs.use_tc = ms_.p.sigma_product_simt == 0;
    if (any_b) {
      BCK(global_step_b(bs));
      // CCD step bound of every frame of the batched step
      launch_ccd_b(s_, tab_dev_, cap_, tab_[0], p.dhat, p.ccd_s, p.accd_max_iters);
      BCK(cudaGetLastError());
    }
    for (int f = 0; f < cap_; ++f)
      if (act[f] && frames_[f].fp64) {
        frames_[f].st.fp64_steps++;
        BTRY(redo_fp64(f, false));
      }
    // backtracking line searches, all frames' trials in one evaluation
    std::vector<char> srch = act;
    std::vector<double> Et(cap_, 0.0);
    std::vector<int64_t> npt(cap_, 0);
    std::vector<char> ok(cap_, 0);
    for (int f = 0; f < cap_; ++f) {
      frames_[f].scale = 1.0;
      frames_[f].trial = 0;
      frames_[f].redone = frames_[f].fp64;
    }
    for (int k = 0; k <= p.max_ls + 1; ++k) {
      bool any_s = false;
      for (char c : srch) any_s |= c != 0;
      if (!any_s) break;
      BTRY(evaluate(srch, 1));
      BTRY(read_back());
      if (cnt(0)[15]) return FSIM_ECUDA;       // a tensor-core wait ran out
      for (int f = 0; f < cap_; ++f) {
        if (!srch[f]) continue;
        Frame& fr = frames_[f];
        if (fr.trial == 0 && cnt(f)[6] && !fr.redone) {
          // the float32 factor of the frame's reduced system lost positive
          // definiteness: its step again in float64 (the single-frame global
          // step on its own workspace), then its CCD bound; its line search
          // starts over at the next trial
          fr.redone = true;
          fr.fp64 = true;
          fr.st.fp64_steps++;
          fr.st.reduced_steps[reduced_path(fr.nc, FSIM_MIXED, tab_[f].one_cta_max)]--;
          fr.st.reduced_steps[reduced_path(fr.nc, FSIM_FP64, tab_[f].one_cta_max)]++;
          BTRY(redo_fp64(f, true));
          fr.scale = 1.0;
          continue;
        }
        if (fr.trial > p.max_ls) { srch[f] = 0; continue; }
        if (fr.trial == 0 && cnt(f)[6]) { srch[f] = 0; act[f] = 0; finish(f, FSIM_ENOT_SPD); continue; }
        if (fr.trial == 0 && cnt(f)[9]) { srch[f] = 0; act[f] = 0; finish(f, FSIM_ECONTACT_OVERFLOW); continue; }
        fr.trial++;
        fr.st.ls_trials++;
        const double e = scl(f)[2] + scl(f)[0];
        if (cnt(f)[2]) { srch[f] = 0; act[f] = 0; finish(f, FSIM_ECONTACT_OVERFLOW); continue; }
        if (!cnt(f)[5] && std::isfinite(e) && e <= fr.E + 1e-12 * std::fabs(fr.E)) {
          srch[f] = 0;
          ok[f] = 1;
          Et[f] = e;
          npt[f] = cnt(f)[0];
          fr.st.alpha_min = std::min(fr.st.alpha_min, scl(f)[1] * fr.scale);
          double Ebt = scl(f)[0];
          adapt_kappa(fr, scl(f)[4], &Ebt);
          fr.E = scl(f)[2] + Ebt;
          continue;
        }
        fr.scale *= 0.5;
        if (fr.trial > p.max_ls) srch[f] = 0;     // out of halvings: ELS_FAIL below
      }
    }
    std::vector<char> grad(cap_, 0);
    for (int f = 0; f < cap_; ++f) {
      if (!act[f]) continue;
      Frame& fr = frames_[f];
      if (!ok[f]) { finish(f, FSIM_ELS_FAIL); continue; }
      DevMesh& m = tab_[f];
      std::swap(m.x, m.xt);
      std::swap(m.s, m.st);
      std::swap(m.tetf, m.tetf_t);
      fr.npairs = npt[f];
      fr.st.iterations++;
      grad[f] = 1;
    }
    bool any_g = false;
    for (char c : grad) any_g |= c != 0;
    if (!any_g) return FSIM_OK;
    BTRY(gradient(grad));
    for (int f = 0; f < cap_; ++f)
      if (grad[f] && !std::isfinite(frames_[f].gn)) finish(f, FSIM_ENONFINITE);
    return FSIM_OK;
  }

  fsim_ctx_t ctx_;
  MeshState& ms_;
  int cap_ = 1, nr_ = 32;
  cudaStream_t s_ = nullptr, s2_ = nullptr;
  cudaEvent_t ev_[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<Frame> frames_;
  std::vector<DevMesh> tab_;
  std::vector<void*> allocs_;
  int* counters_ = nullptr;
  double* scal_ = nullptr;
  float *rb_ = nullptr, *yb_ = nullptr, *ub_ = nullptr, *bx_ = nullptr;
  DevMesh* tab_dev_ = nullptr;
  static constexpr int kTabRing = 4;
  DevMesh* h_tab_ = nullptr;       // kTabRing pinned tables of cap_ frames
  cudaEvent_t ev_tab_[kTabRing] = {nullptr, nullptr, nullptr, nullptr};
  int tab_slot_ = 0;
  int* h_counters_ = nullptr;
  double* h_scal_ = nullptr;
  size_t args_bytes_ = 0;
  void* args_dev_ = nullptr;
  std::vector<char> args_host_;
  char* h_args_ = nullptr;
  const int* cols_dev_ = nullptr;
  double** x1s_dev_ = nullptr;
  double** h_x1s_ = nullptr;
  struct Finished {
    void* user;
    int rc;
    fsim_frame_stats st;
  };
  std::vector<Finished> finished_;
  const BatchDone* done_ = nullptr;
  cudaEvent_t ev_done_ = nullptr;
  size_t bytes_ = 0;
};

Batch* batch_create(fsim_ctx_t ctx, MeshState& ms, int cap, cudaStream_t stream, int* status) {
  auto* b = new (std::nothrow) Batch(ctx, ms, cap, stream);
  if (!b) { *status = FSIM_ENOMEM; return nullptr; }
  *status = b->init();
  if (*status != FSIM_OK) { delete b; return nullptr; }
  return b;
}
void batch_destroy(Batch* b) { delete b; }
size_t batch_bytes(const Batch* b) { return b ? b->bytes() : 0; }
int batch_run(Batch* b, const BatchPull& pull, const BatchDone& done) { return b->run(pull, done); }
bool batch_servable(const MeshState& ms, const fsim_request& q) {
  return ms.prefactored && q.precision == FSIM_MIXED && ms.p.solver == FSIM_SOLVER_WOODBURY &&
         batch_supported(ms.d, 32);
}

}  // namespace fsim

extern "C" fsim_status fsim_solve_batch(fsim_ctx_t ctx, int32_t n_req, const fsim_request* reqs,
                                        int32_t max_frames, double* const* x_out,
                                        fsim_frame_stats* stats) {
  if (!ctx || n_req < 0 || (n_req > 0 && !reqs) || max_frames < 1 || max_frames > kMaxBatchFrames)
    return FSIM_EINVAL;
  if (n_req == 0) return FSIM_OK;
  const int mesh_id = reqs[0].mesh_id;
  MeshState* ms = rt_mesh(ctx, mesh_id);
  if (!ms) return FSIM_EINVAL;
  if (!ms->prefactored) return FSIM_ENOT_READY;
  for (int i = 0; i < n_req; ++i) {
    const fsim_request& q = reqs[i];
    if (q.mesh_id != mesh_id || q.precision != FSIM_MIXED || !q.fiber || !q.stretch ||
        (q.flags & ~FSIM_REQ_DEVICE))
      return FSIM_EINVAL;
  }
  if (ms->p.solver != FSIM_SOLVER_WOODBURY) return FSIM_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FSIM_ECUDA;
  int rc = FSIM_OK;
  Batch* b = batch_create(ctx, *ms, std::min<int>(max_frames, n_req), ctx->stream, &rc);
  if (!b) return rc;
  int next = 0, first_err = FSIM_OK;
  const BatchPull pull = [&](BatchReq* out) {
    if (next >= n_req) return false;
    out->req = reqs[next];
    out->user = reinterpret_cast<void*>((intptr_t)next);
    out->x_host = x_out ? x_out[next] : nullptr;
    ++next;
    return true;
  };
  const BatchDone done = [&](void* user, int st_rc, const fsim_frame_stats& st) {
    const int i = (int)reinterpret_cast<intptr_t>(user);
    if (stats) stats[i] = st;
    if (st_rc != FSIM_OK && first_err == FSIM_OK) first_err = st_rc;
  };
  rc = batch_run(b, pull, done);
  batch_destroy(b);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return FSIM_ECUDA;
  return rc != FSIM_OK ? rc : first_err;
}
