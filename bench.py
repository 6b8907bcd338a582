#!/usr/bin/env python3
"""Benchmark: converged frames/s of the actuated face solve (PD + IPC).

Workload: the synthetic 30k-vertex face mesh (ellipsoidal soft-tissue shell,
3 cm thick, skull pinned, mouth slit with two lip lobes; 16 seeded Gaussian
actuation bumps, stretch in [0.6, 1], random fibres), frames of the 100-frame
sequence whose bump coefficients are interpolated between 5 seeded keyframes.
One step = one frame solved to convergence by Algorithm 1 (every iteration on
the GPU), warm-started from the previous frame.

value : frames/s with the frame's actuation already resident in HBM (mixed
        precision; the float64 form is reported beside it), events on the
        solver's stream, L2 flushed between frames (256 MB write).
e2e   : the same frames through the public C API with host buffers: each
        step copies the actuation and the warm start from pinned host memory
        and reads the converged positions back.
Under torchrun (N > 1) every rank solves its own independent sequence
(replicas, no collective on the data path); value = all frames / max time.
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
FP64_TFLOPS_PEAK = 1.25      # GB300 nominal dense FP64 (profiling recipe table)
ORACLE_ITERS_PER_FRAME = 90  # mean accepted iterations per face frame (GPU and oracle agree)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-target", type=int, default=30000)
    ap.add_argument("--only", choices=["both", "mixed", "fp64"], default="both",
                    help="precisions to time (profiling runs use one)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n_target, n_frames, seed_offset=0):
    from paper_2312_02999_gb300 import inputs as I
    mesh = I.face_shell(n_target=n_target)
    field = I.bump_field(mesh, seed=2)
    coeffs = I.keyframe_coeffs(seed=3 + seed_offset)
    acts = [I.bump_actuation(field, coeffs[f]) for f in range(n_frames + 1)]
    return mesh, acts


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
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from paper_2312_02999_gb300 import inputs as I
from oracle import solver as S
mesh = I.face_shell(n_target={n})
field = I.bump_field(mesh, seed=2)
coeffs = I.keyframe_coeffs(seed=3)
out = []
t0 = time.perf_counter()
pr = S.Problem(mesh.rest, mesh.tets, mesh.pinned, mesh.proxy_tris, mesh.W_rowptr, mesh.W_col,
               mesh.W_val, S.Params(dhat=mesh.dhat, tol_abs=mesh.tol_abs, tol_rel=mesh.tol_rel))
setup = time.perf_counter() - t0
for k in range({steps}):
    a = I.bump_actuation(field, coeffs[1 + k])
    pr.set_actuation(a.fiber, a.stretch)
    t = time.perf_counter()
    x, st = pr.solve_frame(mesh.rest, max_iters={iters}, record=False)
    out.append((time.perf_counter() - t, st.iterations))
print(json.dumps({{"setup_s": setup, "samples": out}}))
"""


def run_oracle_sample(n_target, steps, iters):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, n=n_target, steps=steps, iters=iters)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    per_iter = [t / max(it, 1) for t, it in res["samples"]]
    s_per_frame = statistics.mean(per_iter) * ORACLE_ITERS_PER_FRAME
    return 1.0 / s_per_frame, res


def cpu_baseline(n_target):
    fps, res = run_oracle_sample(n_target, steps=1, iters=2)
    return {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": (f"2 iterations of face frame 1 (full sparse LU of the contact system each "
                       f"iteration), {res['samples'][0][0]:.1f} s; frames/s = 1 / (s per iteration x "
                       f"{ORACLE_ITERS_PER_FRAME} iterations per frame); single thread")}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = args.warmup + args.steps
    fps, res = run_oracle_sample(args.n_target, steps=n, iters=1)
    timed = res["samples"][args.warmup:]
    per_iter = [t / max(it, 1) for t, it in timed]
    s_frame = statistics.mean(per_iter) * ORACLE_ITERS_PER_FRAME
    value = 1.0 / s_frame
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": s_frame * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "face_shell_30k", "n_target": args.n_target, "frames": args.steps},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"1 iteration of each of {n} face frames, extrapolated by "
                                       f"{ORACLE_ITERS_PER_FRAME} iterations per frame"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def percentile(v, q):
    s = sorted(v)
    if not s:
        return None
    k = min(len(s) - 1, max(0, int(round(q / 100.0 * (len(s) - 1)))))
    return s[k]


def run_ours(args):
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

    W, K = args.warmup, args.steps
    mesh, acts = workload(args.n_target, W + K, seed_offset=rank)
    ctx = fsim.Context(local)
    m = ctx.upload(mesh)
    m.prefactor(fsim.params_for(mesh))
    info = m.info()
    dev = torch.device("cuda", local)
    fiber = torch.tensor(acts[0].fiber, dtype=torch.float64, device=dev).contiguous()
    stretch = torch.tensor(np.stack([a.stretch for a in acts]), dtype=torch.float64,
                           device=dev).contiguous()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.ExternalStream(ctx.stream_ptr(), device=dev)
    T = mesh.T
    # host (pinned) inputs for the e2e leg
    fiber_h = torch.tensor(acts[0].fiber, dtype=torch.float64).pin_memory().numpy()
    stretch_h = torch.tensor(np.stack([a.stretch for a in acts]), dtype=torch.float64).pin_memory().numpy()
    xbuf_h = torch.empty((mesh.n, 3), dtype=torch.float64).pin_memory().numpy()

    def set_frame(f):
        m.set_actuation_dev(fiber.data_ptr(), stretch[f].data_ptr())

    def solve_sequence(prec, record_ms, frames):
        times, stats = [], []
        for f in frames:
            with torch.cuda.stream(stream):
                flush.fill_(float(f))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            set_frame(f)
            rc, st = m.solve_frame(None, precision=prec, check=False)
            e1.record(stream)
            e1.synchronize()
            if rc != 0:
                raise RuntimeError(f"frame {f} failed: {fsim.STATUS_NAMES.get(rc, rc)} {st}")
            if record_ms:
                times.append(e0.elapsed_time(e1))
            stats.append(st)
        return times, stats

    def reset():
        set_frame(0)
        m.solve_frame(mesh.rest, precision=fsim.FP64, check=True)

    results = {}
    dominant = None
    legs = [("fp64", fsim.FP64), ("mixed", fsim.MIXED)]
    if args.only != "both":
        legs = [l for l in legs if l[0] == args.only]
    for prec_name, prec in legs:
        reset()
        # warm-up frames; the first pass also finds the dominant kernel class
        if prec_name == "mixed":
            ctx.profile((1 << len(fsim.PROF_CLASSES)) - 1)
            ctx.profile_reset()
        solve_sequence(prec, False, range(1, W + 1))
        if prec_name == "mixed":
            tot = [ctx.profile_read(c)[1] for c in range(len(fsim.PROF_CLASSES))]
            dominant = int(np.argmax(tot))
            ctx.profile(1 << dominant)
            ctx.profile_reset()
        x_after_warm = m.positions()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = Clocks(local) if rank == 0 else None
        if clk:
            clk.start()
        launches0 = ctx.launch_count()
        times, stats = solve_sequence(prec, True, range(W + 1, W + K + 1))
        launches = ctx.launch_count() - launches0
        torch.cuda.synchronize()
        clocks = clk.stop() if clk else None
        prof = ctx.profile_read(dominant) if prec_name == "mixed" else None
        ctx.profile(0)
        total_ms = sum(times)
        if world > 1:
            t = torch.tensor([total_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total_ms = float(t.item())
        results[prec_name] = {"times": times, "stats": stats, "total_ms": total_ms,
                              "launches": launches, "clocks": clocks, "prof": prof,
                              "x_after_warm": x_after_warm}

    if args.only != "both" or args.no_e2e:
        if rank == 0:
            r = results[args.only if args.only != "both" else "mixed"]
            print(json.dumps({"partial": True, "leg": list(results), "frames_per_s":
                              {k: world * K / (v["total_ms"] / 1e3) for k, v in results.items()},
                              "iterations": [s["iterations"] for s in r["stats"]]}), flush=True)
        ctx.close()
        return
    # e2e (mixed): host buffers through the public API, same timed frames
    m.solve_frame(results["mixed"]["x_after_warm"], precision=fsim.FP64, check=False)
    xbuf_h[:] = results["mixed"]["x_after_warm"]
    if world > 1:
        torch.distributed.barrier()
    e2e_times = []
    for f in range(W + 1, W + K + 1):
        with torch.cuda.stream(stream):
            flush.fill_(float(f))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.set_actuation(fiber_h, stretch_h[f])
        rc, st = m.solve_frame(xbuf_h, precision=fsim.MIXED, check=False)
        out = m.positions()
        xbuf_h[:] = out
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_total = sum(e2e_times)
    if world > 1:
        t = torch.tensor([e2e_total], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_total = float(t.item())

    if rank != 0:
        ctx.close()
        return
    mix, f64 = results["mixed"], results["fp64"]
    value = world * K / (mix["total_ms"] / 1e3)
    fp64_value = world * K / (f64["total_ms"] / 1e3)
    iters = [s["iterations"] for s in mix["stats"]]
    # roofline of the dominant kernel class (events around each of its launches)
    cls_name = fsim.PROF_CLASSES[dominant]
    n_launch, ms = mix["prof"]
    avg_ms = ms / max(n_launch, 1)
    roof = roofline_entry(cls_name, info, mesh, avg_ms, n_launch, mix)
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": mix["total_ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (mixed)", "data": "synthetic",
        "config": {"workload": "face_shell_30k", "n": int(info["n"]), "tets": int(info["T"]),
                   "n1": int(info["n1"]), "n2": int(info["n2"]), "frames": K,
                   "precision": "mixed", "l2": "flushed between frames (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": percentile(mix["times"], 50), "p99": percentile(mix["times"], 99)},
        "fp64": {"value": fp64_value, "unit": "frames/s", "ms_per_step": f64["total_ms"] / K,
                 "latency_ms": {"p50": percentile(f64["times"], 50),
                                "p99": percentile(f64["times"], 99)},
                 "iterations_mean": statistics.mean(s["iterations"] for s in f64["stats"])},
        "iterations_mean": statistics.mean(iters),
        "n_c_max": max(s["n_c_max"] for s in mix["stats"]),
        "contacts_max": max(s["contacts"] for s in mix["stats"]),
        "e2e": {"value": world * K / (e2e_total / 1e3), "unit": "frames/s",
                "h2d_bytes_per_step": int(32 * T + 24 * mesh.n), "d2h_bytes_per_step": int(24 * mesh.n)},
        "gpu_launches": int(mix["launches"]),
        "clocks": mix["clocks"],
        "roofline": roof,
    }
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(args.n_target)
        except Exception as e:  # reported, never silently replaced
            line["cpu_baseline"] = {"error": str(e)[-300:]}
    print(json.dumps(line), flush=True)
    ctx.close()


def roofline_entry(cls_name, info, mesh, avg_ms, n_launch, res):
    """Algorithmic work per launch of the dominant class / measured duration."""
    T = int(info["T"])
    nnz = int(info["factor_nnz"])
    lv = max(int(info["n_levels"]), 1)
    if cls_name == "local_step":
        flops = 510.0 * T          # float64 flops per tet of the mixed local step
        ach = flops / (avg_ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP64_TFLOPS_PEAK, "unit": "TFLOP/s",
                "frac": ach / FP64_TFLOPS_PEAK, "traffic": None, "kernel": "k_elastic<1>",
                "launches": n_launch, "avg_ms": avg_ms, "work": "510 fp64 flop/tet x T"}
    if cls_name in ("trsv_fwd", "trsv_bwd"):
        byts = 4.0 * nnz / lv      # float32 factor entries per level launch (average)
        ach = byts / (avg_ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": 6777.0, "unit": "GB/s",
                "frac": ach / 6777.0, "traffic": None, "kernel": f"k_{cls_name}_chunk<float>",
                "launches": n_launch, "avg_ms": avg_ms, "work": "4 B x factor entries / levels"}
    return {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None, "kernel": cls_name, "launches": n_launch, "avg_ms": avg_ms}


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
