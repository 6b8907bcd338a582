#!/usr/bin/env python3
"""Benchmark: converged frames/s of the actuated face solve (PD + IPC).

Workload: the synthetic 30k-vertex face mesh (ellipsoidal soft-tissue shell,
3 cm thick, skull pinned, mouth slit with two lip lobes; 16 seeded Gaussian
actuation bumps, stretch in [0.6, 1], random fibres), frames of 100-frame
sequences whose bump coefficients are interpolated between 5 seeded
keyframes; every sequence (one per client stream) animates its own keyframes.
One step = one frame of every stream, each solved to convergence by
Algorithm 1 (every iteration on the GPU) and warm-started from the stream's
previous frame.

value : frames/s of the request server in lock-step batch mode (mixed
        precision): the clients submit each stream's next frame as soon as its
        previous one is back; the batch workers take queued frames into the
        slots of finished frames at every iteration boundary.  Inputs are
        resident in HBM; CUDA events bracket the timed region.
e2e   : the same through the public C API with host buffers: each request's
        actuation and warm start are copied from host memory at submit and
        its converged positions are read back.
Beside it: the per-request server at 8 streams (the low-latency operating
point), the float64 form at the headline's load, single-sequence latency,
per-frame error against the stored oracle frames, per-class rooflines and
the CPU oracle baseline.  Under torchrun (N > 1) every rank serves its own
streams (replicas, no collective on the data path); value = all frames /
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged frames/s, 30k-vert face mesh; p50/p99 frame latency, mixed vs FP64"
GOLD = os.path.join(ROOT, "tests", "golden", "face_seq3_f20_f21.npz")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-target", type=int, default=30000)
    # 96 sequences in three concurrent 32-frame batches: 149 frames/s at p50 / p99
    # 0.58 / 0.62 s on one GB300 (64 in two batches: 135 at 0.41 / 0.46 s; 128 in
    # four: 155 at 0.76 / 0.82 s)
    ap.add_argument("--streams", type=int, default=96,
                    help="concurrent frame sequences of the headline (batch-mode) leg")
    ap.add_argument("--batch-frames", type=int, default=32, help="frames per lock-step batch")
    ap.add_argument("--batch-workers", type=int, default=3, help="concurrent batches")
    ap.add_argument("--lowlat-streams", type=int, default=8,
                    help="sequences (and per-request workers) of the low-latency leg")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed frames per stream of the float64 served leg")
    ap.add_argument("--quick", action="store_true",
                    help="skip the float64 served leg, the host-buffer leg and the low-latency leg")
    ap.add_argument("--legs", choices=["all", "single", "served", "compare", "cpu-frame", "configs"],
                    default="all",
                    help="single: only the single-sequence legs (profiling runs); served: only "
                         "the headline served leg (profiling runs); compare: "
                         "global step by Schur + Woodbury vs PD-preconditioned CG, at kappa and "
                         "10 kappa (the paper's solver comparison), float64; cpu-frame: one whole "
                         "oracle face frame on the host; configs: the batched (4 meshes) and "
                         "served (8 meshes, Poisson arrivals) workloads")
    ap.add_argument("--first-frame", type=int, default=20,
                    help="first frame of each sequence (solved from rest, untimed)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# replicas over ranks (host logic only; tests/test_replicas_gloo.py runs it
# on two gloo ranks on the CPU)
# ---------------------------------------------------------------------------
def stream_seeds(rank, streams):
    """Keyframe seed of each of this rank's request streams: every (rank,
    stream) animates its own sequence, so ranks share no frame and need no
    data-path collective."""
    return [3 + rank * streams + s for s in range(streams)]


def max_over_ranks(value, world, device=None):
    """Largest of the ranks' values (the timed region's duration): the whole
    job is as slow as its slowest replica.  float64 all-reduce(MAX)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_fps(world, streams, steps, max_ms):
    """Frames of all ranks (world x streams x steps) over the slowest rank's
    timed region."""
    return world * streams * steps / (max_ms / 1e3)


def percentile(v, q):
    s = sorted(v)
    if not s:
        return None
    k = min(len(s) - 1, max(0, int(round(q / 100.0 * (len(s) - 1)))))
    return s[k]


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                       "-i", str(self.gpu), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle leg (also the reference arm)
# ---------------------------------------------------------------------------
# A sample of oracle iterations in the contact regime: on the 30k face, frame
# 21 of sequence 3 started from the oracle's own frame-20 result (the stored
# oracle frames: the lips touch there), extrapolated by the oracle's own
# iteration count for that frame (also stored); on other meshes, frame
# `first` from rest and the sampled frame's own count is unknown, so the
# extrapolation uses the stored face count.
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from paper_2312_02999_gb300 import inputs as I
from oracle import solver as S
gold = {gold!r}
mesh = I.face_shell(n_target={n})
field = I.bump_field(mesh, seed=2)
coeffs = I.keyframe_coeffs(seed=3)
t0 = time.perf_counter()
pr = S.Problem(mesh.rest, mesh.tets, mesh.pinned, mesh.proxy_tris, mesh.W_rowptr, mesh.W_col,
               mesh.W_val, S.Params(dhat=mesh.dhat, tol_abs=mesh.tol_abs, tol_rel=mesh.tol_rel))
setup = time.perf_counter() - t0
x0, frame, per_frame, whole = mesh.rest, {first}, None, {whole}
if os.path.exists(gold):
    g = np.load(gold)
    per_frame = int(g["iterations1"])
    if int(g["n"]) == mesh.n and not whole:
        x0, frame = g["x0"], int(g["frames"][1])
out = []
for k in range({steps}):
    a = I.bump_actuation(field, coeffs[frame])
    pr.set_actuation(a.fiber, a.stretch)
    t = time.perf_counter()
    x, st = pr.solve_frame(x0, max_iters={iters}, record=False)
    out.append((time.perf_counter() - t, st.iterations, st.status))
print(json.dumps({{"setup_s": setup, "samples": out, "frame": frame, "per_frame": per_frame,
                  "from_oracle_state": frame != {first}}}))
"""


def run_oracle_sample(n_target, steps, iters, first, whole=False, timeout=1800):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, gold=GOLD, n=n_target, steps=steps, iters=iters,
                                 first=first, whole=bool(whole))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_fps(res, samples):
    """frames/s from timed oracle iterations: 1 / (s per iteration x iterations
    per frame), the per-frame count being the oracle's own for the sampled
    frame (stored with the oracle frames) or, failing that, 90."""
    per_iter = [t / max(it, 1) for t, it, _ in samples]
    iters = res["per_frame"] or 90
    return 1.0 / (statistics.mean(per_iter) * iters), iters


def cpu_baseline(n_target, first):
    res = run_oracle_sample(n_target, steps=1, iters=3, first=first)
    fps, iters = oracle_fps(res, res["samples"])
    t, it, _ = res["samples"][0]
    where = (f"face frame {res['frame']} from the oracle's frame-{res['frame'] - 1} result (in "
             "contact)" if res["from_oracle_state"] else f"face frame {res['frame']} from rest")
    return {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": (f"{it} oracle iterations of {where}: full sparse LU of the contact system "
                       f"each iteration, {t:.1f} s; frames/s = 1 / (s per iteration x {iters} "
                       "iterations, the oracle's own count for that frame); single thread")}


def bench_config(args, world):
    S, K = args.streams, args.steps
    return {"workload": f"face_shell_{round(args.n_target / 1000)}k", "n_target": args.n_target,
            "form": "served, lock-step batches",
            "streams": S, "batch_frames": args.batch_frames, "batch_workers": args.batch_workers,
            "frames_per_stream": K,
            "step": f"{S} frames, one per stream (each warm-started from its own previous frame)",
            "frames": f"sequence frames {args.first_frame}.. (first solved from rest, then "
                      f"{args.warmup - 1} warm-up frames, then the timed frames)",
            "l2": ("served legs: each frame is ~90 solver iterations over >129 MB of distinct "
                   "data (shared factor and Sigma^-1, per-frame workspaces of 0.16 GB); "
                   "single-stream legs flush L2 (256 MB write) before every frame"),
            "timing": "CUDA events bracketing the whole timed region (all streams)",
            "parallelism": f"replicas x{world}"}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = args.warmup + args.steps
    res = run_oracle_sample(args.n_target, steps=n, iters=1, first=args.first_frame)
    timed = res["samples"][args.warmup:]
    value, iters = oracle_fps(res, timed)
    s_frame = 1.0 / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": s_frame * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "precision": "float64", "data": "synthetic",
            "config": bench_config(args, world),
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"1 oracle iteration of face frame {res['frame']} per step "
                                       f"({'from the oracle frame-%d result, in contact' % (res['frame'] - 1) if res['from_oracle_state'] else 'from rest'}), "
                                       f"{n} steps, x {iters} iterations per frame (the oracle's "
                                       "own count); single thread"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cpu_frame(args):
    """One whole oracle face frame on the host (all iterations), timed."""
    if dist_env()[0] != 0:
        return
    res = run_oracle_sample(args.n_target, steps=1, iters=500, first=args.first_frame, whole=False,
                            timeout=7200)
    t, it, st = res["samples"][0]
    print(json.dumps({"cpu_frame": {"frame": res["frame"], "from_oracle_state": res["from_oracle_state"],
                                    "seconds": t, "iterations": it, "status": st,
                                    "frames_per_s": 1.0 / t, "cores": 1}}), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def stream_actuations(I, field, first, n_frames, seed):
    # entry 0 is unused (index 1 = the sequence's frame `first`)
    coeffs = I.keyframe_coeffs(seed=seed)
    return [I.bump_actuation(field, coeffs[min(first + f - 1, len(coeffs) - 1)])
            for f in range(n_frames + 1)]


def run_compare(args):
    """Per-iteration global-step time of the paper's method (Schur + Woodbury,
    Eq. 8-11) against its comparison configuration (CG preconditioned with H),
    at the automatic kappa and at 10 kappa, on the same face frames (float64)."""
    import numpy as np
    import torch
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim
    from paper_2312_02999_gb300 import inputs as I
    F0, K = args.first_frame, max(1, min(args.steps, 2))
    mesh = I.face_shell(n_target=args.n_target)
    field = I.bump_field(mesh, seed=2)
    acts = stream_actuations(I, field, F0, K + 1, seed=3)
    cls = fsim.PROF_CLASSES
    gstep = ["trsv_fwd", "trsv_bwd", "sigma_gemv", "reduced"]
    out = {}
    with fsim.Context(0) as ctx:
        kappa0 = None
        for solver, name in ((fsim.SOLVER_WOODBURY, "woodbury"), (fsim.SOLVER_PCG, "pcg"),
                             (fsim.SOLVER_SCHUR, "schur")):
            for kmul in (1.0, 10.0):
                m = ctx.upload(mesh)
                p = fsim.params_for(mesh, solver=solver)
                if kappa0 is not None:
                    p.kappa = kmul * kappa0
                m.prefactor(p)
                if kappa0 is None:
                    kappa0 = m.info()["kappa"]
                    if kmul != 1.0:
                        raise RuntimeError("first run must use the automatic kappa")
                m.set_actuation(acts[1].fiber, acts[1].stretch)
                m.solve_frame(mesh.rest, precision=fsim.FP64, check=True)
                ctx.profile((1 << len(cls)) - 1)
                ctx.profile_reset()
                it, cg, t_ms = 0, 0, 0.0
                for f in range(2, K + 2):
                    m.set_actuation(acts[f].fiber, acts[f].stretch)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    stream = torch.cuda.ExternalStream(ctx.stream_ptr())
                    e0.record(stream)
                    rc, st = m.solve_frame(None, precision=fsim.FP64, check=False)
                    e1.record(stream)
                    e1.synchronize()
                    if rc != 0:
                        raise RuntimeError(f"{name} frame {f}: {fsim.STATUS_NAMES.get(rc, rc)}")
                    it += st["iterations"]
                    cg += st["cg_iterations"]
                    t_ms += e0.elapsed_time(e1)
                prof = {c: ctx.profile_read(i)[1] for i, c in enumerate(cls)}
                ctx.profile(0)
                if solver == fsim.SOLVER_PCG:
                    g_ms = prof["pcg"]
                elif solver == fsim.SOLVER_SCHUR:
                    g_ms = prof["trsv_fwd"] + prof["trsv_bwd"] + prof["schur"]
                else:
                    g_ms = sum(prof[c] for c in gstep)
                out[f"{name}_kappa_x{int(kmul)}"] = {
                    "global_step_ms_per_iter": g_ms / max(it, 1), "frame_ms": t_ms / K,
                    "iterations": it, "cg_iterations": cg}
    w1, c1, s1 = out["woodbury_kappa_x1"], out["pcg_kappa_x1"], out["schur_kappa_x1"]
    w10, c10, s10 = out["woodbury_kappa_x10"], out["pcg_kappa_x10"], out["schur_kappa_x10"]
    line = {"comparison": "global step, Schur + Woodbury (Eq. 8-11) vs Schur only (dense Sigma-hat, "
                          "Sec. 3.1) vs PD-preconditioned CG",
            "workload": f"face_shell_{round(args.n_target / 1000)}k", "frames": f"{F0 + 1}..{F0 + K}", "precision": "float64",
            "results": out,
            "pcg_over_woodbury_gstep": c1["global_step_ms_per_iter"] / w1["global_step_ms_per_iter"],
            "schur_over_woodbury_gstep": s1["global_step_ms_per_iter"] / w1["global_step_ms_per_iter"],
            "kappa_x10_cost_ratio": {
                "woodbury": w10["global_step_ms_per_iter"] / w1["global_step_ms_per_iter"],
                "schur": s10["global_step_ms_per_iter"] / s1["global_step_ms_per_iter"],
                "pcg": c10["global_step_ms_per_iter"] / c1["global_step_ms_per_iter"]}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import threading

    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim
    from paper_2312_02999_gb300 import inputs as I

    W, K, S = args.warmup, args.steps, args.streams
    mesh = I.face_shell(n_target=args.n_target)
    field = I.bump_field(mesh, seed=2)
    F0 = args.first_frame
    ctx = fsim.Context(local)
    m = ctx.upload(mesh)
    t0 = time.perf_counter()
    m.prefactor(fsim.params_for(mesh))
    prefactor_s = time.perf_counter() - t0
    info = m.info()
    dev = torch.device("cuda", local)
    # every stream animates its own keyframe sequence on the shared fibre field
    fiber = torch.tensor(field.fiber, dtype=torch.float64, device=dev).contiguous()
    stretch = []
    for sd in stream_seeds(rank, S):
        a = stream_actuations(I, field, F0, W + K, seed=sd)
        stretch.append(torch.tensor(np.stack([f.stretch for f in a]), dtype=torch.float64,
                                    device=dev).contiguous())
    xbuf = [[torch.empty((mesh.n, 3), dtype=torch.float64, device=dev) for _ in range(2)]
            for _ in range(S)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.ExternalStream(ctx.stream_ptr(), device=dev)
    T, n = mesh.T, mesh.n
    diag = float(np.linalg.norm(mesh.rest.max(0) - mesh.rest.min(0)))

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- single-stream legs: one sequence, frames back to back ----------
    def single(prec, profile):
        m.set_actuation_dev(fiber.data_ptr(), stretch[0][1].data_ptr())
        m.solve_frame(mesh.rest, precision=fsim.FP64, check=True)    # frame 1 from rest
        for f in range(2, W + 1):
            m.set_actuation_dev(fiber.data_ptr(), stretch[0][f].data_ptr())
            m.solve_frame(None, precision=prec, check=False)
        x_warm = m.positions()
        barrier()

        def frames(record):
            times, stats = [], []
            for k, f in enumerate(range(W + 1, W + K + 1)):
                with torch.cuda.stream(stream):
                    flush.fill_(float(f))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.set_actuation_dev(fiber.data_ptr(), stretch[0][f].data_ptr())
                rc, st = m.solve_frame(x_warm if (k == 0 and not record) else None, precision=prec,
                                       check=False)
                e1.record(stream)
                e1.synchronize()
                if rc != 0:
                    raise RuntimeError(f"frame {f} failed: {fsim.STATUS_NAMES.get(rc, rc)}")
                times.append(e0.elapsed_time(e1))
                stats.append(st)
            return times, stats

        times, stats = frames(True)
        out = {"times": times, "stats": stats, "classes": None, "prof_stats": None}
        if profile:
            # replay the same frames from the same state with per-class events
            ctx.profile((1 << len(fsim.PROF_CLASSES)) - 1)
            ctx.profile_reset()
            _, pst = frames(False)
            out["classes"] = {c: ctx.profile_read(i) for i, c in enumerate(fsim.PROF_CLASSES)}
            out["prof_stats"] = pst
            ctx.profile(0)
        return out

    # ---- per-frame error against the stored oracle frames (face only) -----
    def oracle_error():
        if not os.path.exists(GOLD):
            return None
        g = np.load(GOLD)
        if int(g["n"]) != mesh.n:
            return None
        coeffs = I.keyframe_coeffs(seed=int(g["seq_seed"]))
        out = {}
        for name, prec in (("mixed", fsim.MIXED), ("fp64", fsim.FP64)):
            errs = []
            for k, f in enumerate(g["frames"].tolist()):
                a = I.bump_actuation(field, coeffs[f])
                m.set_actuation(a.fiber, a.stretch)
                rc, st = m.solve_frame(mesh.rest if k == 0 else None, precision=prec, check=False)
                errs.append(float(np.abs(m.positions() - g[f"x{k}"]).max()) / diag)
            out[name] = errs
        return {"frames": g["frames"].tolist(), "max_abs_error_over_diag": out,
                "bars": {"mixed": 1e-6, "fp64": 1e-9},
                "note": "frame 20 from rest, frame 21 warm-started from the GPU's frame 20"}

    # ---- one batched step with per-class events (the headline's kernels) --
    def batch_profile():
        nb = min(S, args.batch_frames)
        xs = [xbuf[s][0].data_ptr() for s in range(nb)]
        ctx.profile((1 << len(fsim.PROF_CLASSES)) - 1)
        ctx.profile_reset()
        rc, sts = fsim.solve_batch_dev(ctx, m, [fiber.data_ptr()] * nb,
                                       [stretch[s][1].data_ptr() for s in range(nb)],
                                       [0] * nb, xs, max_frames=nb)
        classes = {c: ctx.profile_read(i) for i, c in enumerate(fsim.PROF_CLASSES)}
        ctx.profile(0)
        if rc != 0:
            raise RuntimeError(f"batched profile step: {fsim.STATUS_NAMES.get(rc, rc)}")
        return {"frames": nb, "classes": classes, "stats": sts}

    # ---- served legs: S sequences through the request server ---------------
    def served(prec, device_inputs, nstreams, workers, batch_frames, frames_timed,
               timed_clock=False, warm=None):
        srv = fsim.Server(ctx, workers=workers, batch_frames=batch_frames)
        lat, stats = [], []
        lock = threading.Lock()
        host_fib = host_str = None
        if not device_inputs:
            host_fib = torch.tensor(field.fiber).pin_memory().numpy()
            host_str = [stretch[s].cpu().pin_memory().numpy() for s in range(nstreams)]
        cur = [None] * nstreams
        nwarm = W if warm is None else warm

        def client(s, frames, record):
            for f in frames:
                if device_inputs:
                    out = xbuf[s][f % 2]
                    t = srv.submit_dev(m, fiber.data_ptr(), stretch[s][f].data_ptr(),
                                       cur[s].data_ptr() if cur[s] is not None else 0,
                                       out.data_ptr(), prec)
                    rc, _, st, l, q = srv.wait(t)
                    cur[s] = out
                else:
                    t = srv.submit(m, host_fib, host_str[s][f], cur[s], prec)
                    rc, x, st, l, q = srv.wait(t)
                    cur[s] = x
                if rc != 0:
                    raise RuntimeError(f"stream {s} frame {f}: {fsim.STATUS_NAMES.get(rc, rc)}")
                if record:
                    with lock:
                        lat.append(l)
                        stats.append(st)

        def run(frames, record):
            errs = []

            def wrap(s):
                try:
                    client(s, frames, record)
                except Exception as e:      # reported below, never swallowed
                    errs.append(e)
            th = [threading.Thread(target=wrap, args=(s,)) for s in range(nstreams)]
            for t_ in th:
                t_.start()
            for t_ in th:
                t_.join()
            if errs:
                raise errs[0]

        run(range(1, nwarm + 1), False)
        barrier()
        clk = Clocks(local) if (timed_clock and rank == 0) else None
        if clk:
            clk.start()
        launches0 = ctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(range(nwarm + 1, nwarm + frames_timed + 1), True)
        e1.record(stream)        # every request has completed (wait synchronised its stream)
        e1.synchronize()
        total_ms = e0.elapsed_time(e1)
        launches = ctx.launch_count() - launches0
        barrier()
        clocks = clk.stop() if clk else None
        sinfo = srv.info()
        srv.close()
        return {"total_ms": max_over_ranks(total_ms, world, dev), "lat": lat, "stats": stats,
                "launches": launches, "clocks": clocks, "server": sinfo,
                "streams": nstreams, "frames": frames_timed}

    results = {}
    if args.legs == "served":
        r = served(fsim.MIXED, True, S, args.batch_workers, args.batch_frames, K)
        if rank == 0:
            print(json.dumps({"partial": "headline served leg only",
                              "value": whole_job_fps(world, S, K, r["total_ms"]),
                              "latency_ms": {"p50": percentile(r["lat"], 50),
                                             "p99": percentile(r["lat"], 99)},
                              "gpu_launches": int(r["launches"])}), flush=True)
        ctx.close()
        return
    results["single_mixed"] = single(fsim.MIXED, profile=True)
    results["single_fp64"] = single(fsim.FP64, profile=False)
    if args.legs == "single":
        if rank == 0:
            sm = results["single_mixed"]
            print(json.dumps({"partial": "single-sequence legs only",
                              "mixed_ms_per_frame": statistics.mean(sm["times"]),
                              "fp64_ms_per_frame": statistics.mean(results["single_fp64"]["times"]),
                              "iterations": [st["iterations"] for st in sm["stats"]]}), flush=True)
        ctx.close()
        return
    BF, BW = args.batch_frames, args.batch_workers
    results["served_mixed"] = served(fsim.MIXED, True, S, BW, BF, K, timed_clock=True)
    if not args.quick:
        L = min(args.lowlat_streams, S)
        results["lowlat_mixed"] = served(fsim.MIXED, True, L, L, 0, K)
        results["served_fp64"] = served(fsim.FP64, True, S, args.lowlat_streams, 0,
                                        args.fp64_steps, warm=1)
        results["e2e_mixed"] = served(fsim.MIXED, False, S, BW, BF, K)
    bprof = batch_profile() if rank == 0 else None
    oerr = oracle_error() if rank == 0 else None
    if rank != 0:
        ctx.close()
        return

    def fps(r):
        return whole_job_fps(world, r["streams"], r["frames"], r["total_ms"])

    def lat(r):
        return {"p50": percentile(r["lat"], 50), "p99": percentile(r["lat"], 99)}

    sm, s64 = results["single_mixed"], results["single_fp64"]
    srv_m = results["served_mixed"]
    value = fps(srv_m)
    iters = [st["iterations"] for st in srv_m["stats"]]
    rooflines = batch_rooflines(bprof, info)
    dominant = dominant_roofline(rooflines)
    single_leg = lambda r: {
        "value": world * K / (sum(r["times"]) / 1e3) if world == 1 else None,
        "ms_per_frame": statistics.mean(r["times"]),
        "latency_ms": {"p50": percentile(r["times"], 50), "p99": percentile(r["times"], 99)},
        "ms_per_iter": sum(r["times"]) / max(1, sum(st["iterations"] for st in r["stats"])),
        "iterations_mean": statistics.mean(st["iterations"] for st in r["stats"])}
    iters_prof = max(1, sum(st["iterations"] for st in sm["prof_stats"]))
    disjoint = {c: v for c, v in sm["classes"].items() if c != "chol"}
    classes = {c: {"launches": v[0], "ms_per_iter": round(v[1] / iters_prof, 4)}
               for c, v in disjoint.items()}
    paths = [0, 0, 0, 0]
    for st in srv_m["stats"]:
        paths = [a + b for a, b in zip(paths, st["reduced_steps"])]
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": srv_m["total_ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (mixed)", "precision": "mixed",
        "data": "synthetic",
        "config": dict(bench_config(args, world), n=int(info["n"]), tets=int(info["T"]),
                       n1=int(info["n1"]), n2=int(info["n2"]),
                       workspace_bytes=int(info["workspace_bytes"]),
                       prefactor_s=round(prefactor_s, 2)),
        "latency_ms": lat(srv_m),
        "iterations_mean": statistics.mean(iters),
        "n_c_max": max(st["n_c_max"] for st in srv_m["stats"]),
        "contacts_max": max(st["contacts"] for st in srv_m["stats"]),
        "reduced_steps": {"cooperative": paths[0], "none": paths[1], "one_cta": paths[2],
                          "cluster": paths[3]},
        "single_stream": {"mixed": single_leg(sm), "fp64": single_leg(s64)},
        "gpu_launches": int(srv_m["launches"]),
        "clocks": srv_m["clocks"],
        "roofline": dominant,
        "rooflines": rooflines,
        "kernel_classes_single_mixed": classes,
        "oracle_error": oerr,
    }
    if "served_fp64" in results:
        r = results["served_fp64"]
        line["fp64"] = {"value": fps(r), "unit": "frames/s", "latency_ms": lat(r),
                        "streams": r["streams"], "workers": args.lowlat_streams,
                        "form": "per-request server (float64 is not batched)",
                        "iterations_mean": statistics.mean(st["iterations"] for st in r["stats"])}
        r = results["lowlat_mixed"]
        line["low_latency"] = {"value": fps(r), "unit": "frames/s", "latency_ms": lat(r),
                               "streams": r["streams"], "form": "per-request server, one worker "
                                                                "per stream"}
        e = results["e2e_mixed"]
        line["e2e"] = {"value": fps(e), "unit": "frames/s",
                       "h2d_bytes_per_step": int(S * (32 * T + 24 * n)),
                       "d2h_bytes_per_step": int(S * 24 * n),
                       "latency_ms": lat(e)}
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(args.n_target, args.first_frame)
        except Exception as ex:  # reported, never silently replaced
            line["cpu_baseline"] = {"error": str(ex)[-300:]}
    print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------
# rooflines of the batched kernel classes (one batched step, CUDA events)
# ---------------------------------------------------------------------------
FP32_TFLOPS_PEAK = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock


def _measured_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured bf16 burst (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback bf16 burst"


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# The unit of work of the mixed local step per tet: the double-float and
# float32 operations of its first double-float formulation, with separate
# products and additions (FMA = 2 flop): Du 180, F 501, M 468, float32 Jacobi
# polar rotation ~1200, re-orthonormalisation 372, S = R1^T M 558, rotation
# correction 305, p = R A 468, D and |D|^2 369, forces 738.  It is kept fixed
# so that a faster form of the same arithmetic (fused dot products and sums)
# shows as a higher rate.
LOCAL_FLOP_PER_TET = 5160.0
# DRAM bytes per tet of k_elastic_df_b (ncu dram__bytes_read.sum + write.sum
# of one 16-frame launch on face_shell_30k, 152.8 + 182.0 MB over 16 x 148,056
# tets; profiles/k_elastic_df_b_face30k_batch16.md), scaled to a launch by its
# tets; traffic grows with the tets a launch processes
LOCAL_DRAM_BYTES_PER_TET = 141.3
TF32_PER_BF16 = 1.1 / 2.25     # nominal dense TF32 / BF16 tensor rates


def dominant_roofline(rooflines):
    """The roofline of the dominant kernel: the one with the largest share of
    this workload's launch list (ncu, serialised), k_elastic_df_b, the local
    step, at about a quarter (profiles/launches_face30k_served_96streams.md).
    The "reduced" class brackets several kernels that overlap the backward
    solve on the side stream, so its event time also holds the SMs it waits
    for."""
    return next((r for r in rooflines if r["kernel_class"] == "local_step"), None)


def batch_rooflines(bprof, info):
    if not bprof:
        return []
    nb = bprof["frames"]
    it = max(1, max(st["iterations"] for st in bprof["stats"]))
    T, n, n2 = int(info["T"]), int(info["n"]), int(info["n2"])
    nnz = int(info["factor_nnz"])
    hbm, hbm_src = _measured_hbm()
    out = []
    for cls, (launches, ms) in bprof["classes"].items():
        if launches == 0:
            continue
        avg = ms / launches
        e = {"kernel_class": cls, "launches": launches, "avg_ms": avg, "ms": ms, "frames": nb,
             "traffic": None}
        if cls == "local_step":
            flop = LOCAL_FLOP_PER_TET * T * nb
            ach = flop / (avg * 1e-3) / 1e12
            e.update({"bound": "alu", "kernel": "k_elastic_df_b (+ k_disp_df_b, partial sums)",
                      "achieved": ach, "peak": FP32_TFLOPS_PEAK, "unit": "TFLOP/s",
                      "frac": ach / FP32_TFLOPS_PEAK,
                      "work": f"{LOCAL_FLOP_PER_TET:.0f} float32 flop per tet x T x frames",
                      "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (derived)",
                      "bytes_per_launch": (96.0 + 144.0 * nb) * T + 48.0 * n * nb,
                      "traffic": LOCAL_DRAM_BYTES_PER_TET * T * nb,
                      "traffic_source": "ncu DRAM bytes of a 16-frame launch, per tet, x tets "
                                        "of this launch"})
        elif cls in ("trsv_fwd", "trsv_bwd"):
            lv = max(int(info["n_levels"]), 1)
            byts = (4.0 * nnz + 2 * 4.0 * 3 * nb * int(info["n_free"])) / lv
            ach = byts / (avg * 1e-3) / 1e9
            e.update({"bound": "hbm", "kernel": f"k_{cls[5:]}_mr (all frames' right-hand sides)",
                      "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                      "peak_source": hbm_src,
                      "work": "float32 factor entries (read once for all frames) + right-hand "
                              "sides in and out, per level launch (total / levels)"})
        elif cls == "sigma_gemv":
            nr = (3 * nb + 31) // 32 * 32
            flop = 3 * 2.0 * n2 * n2 * nr
            ach = flop / (avg * 1e-3) / 1e12
            pk, pk_src = _measured_bf16()
            pk *= TF32_PER_BF16
            e.update({"bound": "tensor", "kernel": "k_sinv_tc (tcgen05 kind::tf32) + k_unpack_mr",
                      "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                      "peak_source": pk_src + " x nominal TF32/BF16 ratio 1.1/2.25",
                      "work": "3 TF32 products (head/tail split) x 2 n2^2 nr flop"})
        elif cls in ("reduced", "chol"):
            flop = 18.0 * sum(st["sum_nc3"] for st in bprof["stats"]) / it
            ach = flop / (avg * 1e-3) / 1e12
            e.update({"bound": "alu", "kernel": "batched reduced systems (k_small_*_b, k_clus_v_b)",
                      "achieved": ach, "peak": FP32_TFLOPS_PEAK, "unit": "TFLOP/s",
                      "frac": ach / FP32_TFLOPS_PEAK,
                      "work": "(2/3)(3 n_c)^3 = 18 n_c^3 flop per frame per global step "
                              "(mean over the batch's iterations)",
                      "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (derived)"})
        else:
            e.update({"bound": "latency", "kernel": cls, "achieved": None, "peak": None,
                      "unit": None, "frac": None})
        out.append(e)
    return out


# ---------------------------------------------------------------------------
# the batched (4 meshes) and served (8 meshes, Poisson arrivals) workloads
# ---------------------------------------------------------------------------
def run_configs(args):
    import threading

    import numpy as np
    from paper_2312_02999_gb300 import build
    build.build()
    from paper_2312_02999_gb300 import fsim
    from paper_2312_02999_gb300 import inputs as I
    if dist_env()[0] != 0:
        return
    ctx = fsim.Context(0)
    out = {}
    # batched form: 4 face meshes, 16 frames each (frames 20..35 of one
    # keyframe sequence per mesh), one lock-step batch per mesh
    cfg4 = []
    total_frames, total_ms = 0, 0.0
    for nt in (5000, 15000, 30000, 60000):
        mesh = I.face_shell(n_target=nt)
        field = I.bump_field(mesh, seed=2)
        coeffs = I.keyframe_coeffs(seed=7)
        m = ctx.upload(mesh)
        t0 = time.perf_counter()
        m.prefactor(fsim.params_for(mesh))
        pf = time.perf_counter() - t0
        reqs = [(m, field.fiber, I.bump_actuation(field, coeffs[20 + k]).stretch, None)
                for k in range(16)]
        fsim.solve_batch(ctx, reqs[:2], max_frames=2, want_positions=False)      # warm-up
        t0 = time.perf_counter()
        rc, _, sts = fsim.solve_batch(ctx, reqs, max_frames=16, want_positions=False)
        ms = (time.perf_counter() - t0) * 1e3
        if rc != 0:
            raise RuntimeError(f"config 4, mesh {nt}: {fsim.STATUS_NAMES.get(rc, rc)}")
        total_frames += len(reqs)
        total_ms += ms
        cfg4.append({"mesh": f"face_shell_{round(nt / 1000)}k", "n": mesh.n, "T": mesh.T,
                     "n2": int(m.info()["n2"]), "prefactor_s": round(pf, 2),
                     "frames": len(reqs), "ms": ms, "frames_per_s": len(reqs) / (ms / 1e3),
                     "iterations_mean": statistics.mean(st["iterations"] for st in sts),
                     "n_c_max": max(st["n_c_max"] for st in sts),
                     "n_c_range": [min(st["n_c_max"] for st in sts), max(st["n_c_max"] for st in sts)]})
    out["batched_4_meshes"] = {"meshes": cfg4, "frames": total_frames,
                               "frames_per_s": total_frames / (total_ms / 1e3),
                               "form": "fsim_solve_batch, 16 frames of one mesh per batch, mixed",
                               "frames_from": "rest pose"}
    # served form: 8 meshes, 64 bumps each, 64-dim request coefficient
    # vectors, Poisson arrivals, 150 GB memory budget
    sizes = (2000, 5000, 10000, 20000, 30000, 50000, 75000, 100000)
    meshes = []
    for k, nt in enumerate(sizes):
        mesh = I.face_shell(n_target=nt)
        field = I.bump_field(mesh, n_bumps=64, seed=11 + k)
        m = ctx.upload(mesh)
        t0 = time.perf_counter()
        m.prefactor(fsim.params_for(mesh))
        meshes.append((mesh, field, m, time.perf_counter() - t0))
    N = 48
    coeffs = I.request_coeffs(N * 8, n_bumps=64, seed=5)
    rng = np.random.default_rng(9)
    legs = []
    for prec_name, prec, workers, bframes in (("mixed", fsim.MIXED, 4, 8),
                                              ("mixed_per_request", fsim.MIXED, 8, 0),
                                              ("fp64", fsim.FP64, 8, 0)):
        for rate in (50, 100, 200, 500, 1000, 2000):
            picks = rng.integers(0, len(meshes), size=N)
            gaps = rng.exponential(1.0 / rate, size=N)
            reqs = []
            for i in range(N):
                mesh, field, m, _ = meshes[picks[i]]
                a = I.bump_actuation(field, coeffs[(legs.__len__() * N + i) % len(coeffs)], depth=0.4)
                reqs.append((m, a.fiber, a.stretch))
            srv = fsim.Server(ctx, workers=workers, batch_frames=bframes,
                              mem_budget_bytes=150 * 1024 ** 3)
            tickets, t_start = [], time.perf_counter()
            t_next = t_start
            for i, (mm, fb, st_) in enumerate(reqs):
                t_next += gaps[i]
                delay = t_next - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets.append(srv.submit(mm, fb, st_, None, prec))
            res = [srv.wait(t) for t in tickets]
            span = time.perf_counter() - t_start
            srv.close()
            bad = [r[0] for r in res if r[0] != 0]
            lats = [r[3] for r in res]
            legs.append({"precision": prec_name, "rate_req_per_s": rate, "requests": N,
                         "workers": workers, "batch_frames": bframes,
                         "frames_per_s": N / span, "latency_ms": {"p50": percentile(lats, 50),
                                                                  "p99": percentile(lats, 99)},
                         "failed": len(bad),
                         "status": {fsim.STATUS_NAMES.get(c, str(c)): int(n) for c, n in
                                    zip(*np.unique([r[0] for r in res], return_counts=True))},
                         "fp64_global_steps": int(sum(r[2]["fp64_steps"] for r in res))})
    out["served_8_meshes"] = {"meshes": [{"mesh": f"face_shell_{round(nt / 1000)}k", "n": me[0].n,
                                          "n2": int(me[2].info()["n2"]),
                                          "prefactor_s": round(me[3], 2)}
                                         for nt, me in zip(sizes, meshes)],
                              "legs": legs, "budget_bytes": 150 * 1024 ** 3,
                              "requests": "64-dim seeded coefficient vectors over 64 Gaussian "
                                          "bumps per mesh, from the rest pose, mesh uniform"}
    print(json.dumps({"configs": out}), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.legs == "compare":
        if dist_env()[0] == 0:
            run_compare(args)
        return
    if args.legs == "cpu-frame":
        run_cpu_frame(args)
        return
    if args.legs == "configs":
        run_configs(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
