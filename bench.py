"""FSIB time-step benchmark on GB300.

Workload (default): 3D Navier-Stokes, FP64, periodic unit cube, N = 64^3 modes,
lat-long elastic membrane of M = 10082 points (radius 0.25, seeded ellipsoid),
cot-weight springs sigma = 1, rho = 1, mu = 0.01, dt = 1e-4, NUFFT tol 1e-12.
A step is one full FSIB time step (Algorithm 1): force, type-1 NUFFT, two
dealiased V-hat solves with BE/CN updates, two type-2 NUFFTs, position updates.

python bench.py --gpus N --steps K --warmup W [--impl reference]

Prints one JSON line (rank 0). Under torchrun every rank advances its own
independent replica of the workload (the problem does not shard: replicas only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2302_08694_gb300 import workloads as wl  # noqa: E402

METRIC = "FSIB steps/s and NUFFT pts/s, FP32-mixed & batched vs FP64 at stated error"
L2_FLUSH_BYTES = 512 * 1024 * 1024  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--native-fp64", action="store_true", help="FP64 arithmetic instead of double-float")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for k, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(k)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_problem(fsib, prob, precision):
    pb = fsib.Problem(prob.N, prob.d, prob.M, prob.mu, prob.rho, prob.dt, prob.tol, precision=precision)
    if prob.force == "mesh":
        pb.set_force_mesh(prob.tri, prob.Xref, prob.stiffness)
    else:
        pb.set_force_curve(prob.stiffness)
    return pb


def time_oracle_steps(prob, nsteps):
    from oracle import spectral as sp
    from oracle import stepper as st
    force = st.mesh_model(prob.Xref, prob.tri, prob.stiffness)
    N = prob.N
    X = prob.X0.copy()
    u = np.zeros((3, N, N, N), dtype=complex)
    U = np.zeros_like(X)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        X, u, U = st.ns_step(X, u, U, force, N, prob.mu, prob.rho, prob.dt)
    return time.perf_counter() - t0


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    prob = wl.config_ns3d_fp64()
    k = max(1, min(args.steps, 10))
    w = min(args.warmup, 1)
    if w:
        time_oracle_steps(prob, w)
    t = time_oracle_steps(prob, k)
    v = k / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": k, "warmup": w, "ms_per_step": 1e3 * t / k, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": prob.name, "d": 3, "N": prob.N, "M": prob.M, "nsteps_config": prob.nsteps},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{k} full oracle steps (direct non-uniform sums, numpy BLAS/FFT) of the "
                                       f"workload, {w} warm-up; K capped at 10 to bound the run"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2302_08694_gb300 import fsib

    rank, local, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = wl.config_ns3d_fp64()
    pb = make_problem(fsib, prob, "fp64")
    if args.native_fp64:
        pb.set_option("native_fp64", 1)  # re-plans; the mesh model survives
    stream = torch.cuda.current_stream()

    X = torch.from_numpy(prob.X0.copy()).to(dev)
    u = pb.new_spec(device=dev)
    U = pb.interp(u, X)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        pb.step(X, u, U, nsteps=1)
    barrier()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if \
        os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    sampler = ClockSampler(gpu_index)
    time.sleep(0.25)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for s in range(args.steps):
        flush.zero_()  # L2 flush between timed iterations (outside the events)
        ev[s][0].record(stream)
        pb.step(X, u, U, nsteps=1)
        ev[s][1].record(stream)
    barrier()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    t_rank = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_rank, op=dist.ReduceOp.MAX)
    ms_max = float(t_rank.item())
    value = world * args.steps / (ms_max * 1e-3)
    launches = int(pb.info("launches_per_step"))

    # NUFFT throughput, type-1 and type-2 separately (same workload, FP64)
    c = pb.force(X)
    fh = pb.new_spec(device=dev)
    reps = 20
    t1 = t2 = 0.0
    for r in range(reps + 2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pb.spread(X, c, None, out=fh)
        b.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            t1 += a.elapsed_time(b)
        flush.zero_()
        a.record(stream)
        pb.interp(u, X, out=U)
        b.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            t2 += a.elapsed_time(b)
    pts1 = prob.M / (t1 / reps * 1e-3)
    pts2 = prob.M / (t2 / reps * 1e-3)

    # per-launch-site timing (CUDA events around each launch site, direct launches)
    pb.profile(True)
    pb.profile_reset()
    nprof = max(3, min(args.steps, 20))
    Xp, up, Up = X.clone(), u.clone(), U.clone()
    for _ in range(nprof):
        flush.zero_()
        pb.step(Xp, up, Up, nsteps=1)
    sites = pb.profile_entries()
    pb.profile(False)
    tot = sum(s["total_ms"] for s in sites)
    top = max(sites, key=lambda s: s["total_ms"])
    pk, pk_src = peaks()
    fp64_peak = fsib.measure_peak(0)  # GFLOP/s
    fp32_peak = fsib.measure_peak(1)
    avg_ms = top["total_ms"] / top["launches"]
    gbs = top["bytes"] / (avg_ms * 1e-3) / 1e9
    gfl = top["flops"] / (avg_ms * 1e-3) / 1e9
    t_mem = top["bytes"] / (pk["hbm_gbs"] * 1e9)
    t_alu = top["flops"] / (fp64_peak * 1e9)
    if t_alu > t_mem:
        roof = {"bound": "alu", "achieved": gfl / 1e3, "peak": fp64_peak / 1e3, "unit": "TFLOP/s",
                "frac": gfl / fp64_peak}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"]}
    roof.update({"traffic": None, "kernel": top["name"], "share": top["total_ms"] / tot,
                 "bytes_per_launch": top["bytes"], "flops_per_launch": top["flops"],
                 "avg_launch_ms": avg_ms, "peak_source": (pk_src if roof["bound"] == "hbm" else
                                                          "measured FP64 FMA microbenchmark (fsib_measure_peak)"),
                 "hbm_frac": gbs / pk["hbm_gbs"], "fp64_fma_peak_tflops": fp64_peak / 1e3,
                 "fp32_fma_peak_tflops": fp32_peak / 1e3})
    breakdown = sorted(({"site": s["name"], "ms_per_step": s["total_ms"] / nprof,
                         "share": s["total_ms"] / tot,
                         "gbs": s["bytes"] * s["launches"] / (s["total_ms"] * 1e-3) / 1e9,
                         "gflops": s["flops"] * s["launches"] / (s["total_ms"] * 1e-3) / 1e9}
                        for s in sites), key=lambda z: -z["ms_per_step"])

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(prob.X0.copy()).pin_memory()
        uh = torch.zeros(pb.spec_shape, dtype=pb.spec_dtype).pin_memory()
        Uh = torch.zeros_like(Xh).pin_memory()
        ke = max(3, min(args.steps, 30))
        pb.step(Xh, uh, Uh, nsteps=1)
        t0 = time.perf_counter()
        for _ in range(ke):
            pb.step(Xh, uh, Uh, nsteps=1)  # H2D of (X, u-hat, U), step, D2H, synchronous
        te = time.perf_counter() - t0
        nb = Xh.numel() * 8 + uh.numel() * uh.element_size() + Uh.numel() * 8
        e2e = {"value": world * ke / te, "unit": "steps/s", "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        k = 2
        t = time_oracle_steps(prob, k)
        cpu = {"value": k / t, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{k} full oracle steps of the same workload (direct non-uniform sums, numpy BLAS/FFT)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": prob.name, "d": 3, "N": prob.N, "M": prob.M, "nf": int(pb.info("nf")),
                           "Nt": int(pb.info("Nt")), "width": int(pb.info("width")), "tol": prob.tol,
                           "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas{world}"},
                "nufft_pts_per_s": {"type1": world * pts1, "type2": world * pts2},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches * args.steps, "launches_per_step": launches,
                "breakdown": breakdown[:12]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
