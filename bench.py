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
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32-mixed workload block")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload block")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the differentiable workload block")
    ap.add_argument("--no-sweep", action="store_true", help="skip the NUFFT point-count sweep")
    ap.add_argument("--no-validation", action="store_true",
                    help="skip the validation blocks (2D sine circle, Poiseuille channel and Stokes circle, "
                         "3D spheres)")
    ap.add_argument("--workload", choices=["ns3d_fp64", "ns3d_mixed", "ns2d_circle", "poiseuille",
                                           "sphere_elastic", "sphere_tension", "stokes2d"],
                    default="ns3d_fp64",
                    help="workload of the main line (profiling runs use ns3d_mixed for the FP32 kernels)")
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
    """nvidia-smi clocks and throttle reasons sampled every 20 ms; stop(t0, t1) keeps the
    samples taken inside the timed region [t0, t1] (host wall clock), or all of them when
    none falls inside (a region shorter than the sampling interval)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "20"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    @staticmethod
    def _when(stamp):
        import datetime
        try:
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except Exception:
            return None

    def stop(self, t0=None, t1=None):
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
        inside = [r for r in rows if t0 is not None and t1 is not None
                  and (lambda w: w is not None and t0 <= w <= t1)(self._when(r[0]))]
        use = inside or rows
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in use:
            try:
                sm.append(float(r[2]))
                smax = max(smax, float(r[3]))
                for k, v in zip(names, r[6:10]):
                    if v.strip().lower() == "active":
                        reasons.add(k)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "timed region" if inside else "whole sampling run"}


NATIVE_FP64 = False


def make_problem(fsib, prob, precision):
    pb = fsib.Problem(prob.N, prob.d, prob.M, prob.mu, prob.rho, prob.dt,
                      1e-12 if precision == "fp64" else 1e-6, precision=precision)
    if precision == "fp64" and NATIVE_FP64:
        pb.set_option("native_fp64", 1)
    if prob.force == "mesh":
        pb.set_force_mesh(prob.tri, prob.Xref, prob.stiffness)
    elif prob.force == "target":
        pb.set_force_target(prob.extra["Xtarget"], prob.stiffness, prob.extra["omega"])
    elif prob.force == "tension":
        pb.set_force_tension(prob.tri, prob.stiffness)
    else:
        pb.set_force_curve(prob.stiffness)
    if "fbody" in prob.extra:
        pb.set_body_force(prob.extra["fbody"])
    return pb


def time_oracle_steps(prob, nsteps):
    from oracle import spectral as sp
    from oracle import stepper as st
    if prob.force == "mesh":
        force = st.mesh_model(prob.Xref, prob.tri, prob.stiffness)
    elif prob.force == "target":
        force = st.target_model(prob.extra["Xtarget"], prob.stiffness, prob.extra["omega"])
    elif prob.force == "tension":
        force = st.tension_model(prob.tri, prob.stiffness)
    else:
        force = st.curve_model(prob.stiffness)
    N, d = prob.N, prob.d
    X = prob.X0.copy()
    u = np.zeros((d,) + (N,) * d, dtype=complex)
    U = np.zeros_like(X)
    fbody = prob.extra.get("fbody")
    t0 = time.perf_counter()
    for _ in range(nsteps):
        if prob.rho > 0:
            X, u, U = st.ns_step(X, u, U, force, N, prob.mu, prob.rho, prob.dt, fbody=fbody)
        else:
            X = st.stokes_step(X, force, N, prob.mu, prob.dt)
    return time.perf_counter() - t0


def workload_of(name):
    """(problem, precision) of a named benchmark workload."""
    if name == "ns3d_mixed":
        return wl.config_ns3d_mixed(), "mixed"
    if name == "ns2d_circle":
        return wl.config_ns2d_circle(), "fp64"
    if name == "poiseuille":
        return wl.config_poiseuille(N=64), "fp64"
    if name in ("sphere_elastic", "sphere_tension"):
        return wl.config_ns3d_sphere(name.split("_")[1]), "fp64"
    if name == "stokes2d":
        return wl.config_stokes2d(), "fp64"
    return wl.config_ns3d_fp64(), "fp64"


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    prob, _ = workload_of(args.workload if args.workload != "ns3d_mixed" else "ns3d_fp64")
    k = max(1, min(args.steps, 10))
    w = min(args.warmup, 1)
    if w:
        time_oracle_steps(prob, w)
    t = time_oracle_steps(prob, k)
    v = k / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": k, "warmup": w, "ms_per_step": 1e3 * t / k, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": prob.name, "d": prob.d, "N": prob.N, "M": prob.M, "nsteps_config": prob.nsteps},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{k} full oracle steps (direct non-uniform sums, numpy BLAS/FFT) of the "
                                       f"workload, {w} warm-up; K capped at 10 to bound the run"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a site, from one
# ncu capture of the current kernels per workload: the spread site (k_box_slices, k_scan2,
# k_slice_boxes, k_spread_box3[_dd]; profiles/spread_site_traffic.txt has the command and the
# per-kernel figures) and the mixed product pass (k_wrows_product<float, 192>;
# profiles/kernels_ns3d_N128_M40322_mixed.txt). Set an entry to None when those kernels change.
SITE_TRAFFIC = {("ns3d_N64_M10082_fp64", "spread"): 3843840.0,
                ("ns3d_N128_M40322_mixed", "spread"): 9039872.0,
                ("ns3d_N128_M40322_mixed", "nl.rows_product"): 112303360.0}
# The bound that limits a site when it is not HBM, from the same capture: the mixed product
# pass runs its L1/shared-memory pipe at 89 % of peak (l1tex__throughput).
SITE_OTHER_BOUND = {("ns3d_N128_M40322_mixed", "nl.rows_product"):
                    {"bound": "shared memory", "frac": 0.891, "metric": "l1tex__throughput (ncu)"}}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def max_over_ranks(ms_local, world, device="cpu"):
    """Slowest rank's time (ms): the whole job finishes when its last replica does."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(steps, ms_max, world):
    """Whole-job throughput of independent replicas: every rank advanced `steps` steps."""
    return world * steps / (ms_max * 1e-3)


def step_bytes(prob, prec, nf, Nt):
    """Algorithmic bytes of one whole step (every fine and dealiasing grid written once and read
    once, spectra read and written once per use, points read once): type-1 and type-2
    2 d G s + d K c + M d (8 + s) each; the nonlinear term 2 d K c + 2 d D s + d(d+1) D s + d K c;
    an update 3 d K c; Navier-Stokes = t1 + 2 t2 + 2 V + 2 updates, Stokes = 2 t1 + 2 t2 + 2
    Stokeslets (2 d K c each). G = nf^d, K = N^d, D = Nt^d; s, c = bytes per real, complex."""
    d, N, M = prob.d, prob.N, prob.M
    s = 4.0 if prec == "mixed" else 8.0
    c = 2.0 * s
    G, K, D = float(nf) ** d, float(N) ** d, float(Nt) ** d
    t = 2 * d * G * s + d * K * c + M * d * (8 + s)
    if prob.rho > 0:
        V = 2 * d * K * c + 2 * d * D * s + d * (d + 1) * D * s + d * K * c
        return t + 2 * t + 2 * V + 2 * 3 * d * K * c
    return 2 * t + 2 * t + 2 * 2 * d * K * c


def step_roofline(prob, prec, nf, Nt, ms_per_step, pk):
    """Whole-step HBM fraction from the algorithmic bytes (the step skips rows no window
    reaches, so it moves fewer bytes than this model counts); pk: the measured peaks."""
    b = step_bytes(prob, prec, nf, Nt)
    gbs = b / (ms_per_step * 1e-3) / 1e9
    hbm = float(pk["hbm_gbs"])
    return {"algorithmic_bytes_per_step": b, "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm}


def roofline_of(site, prec, pk, pk_src, fp64_peak, fp32_peak):
    """Binding roofline of one launch site: HBM (algorithmic bytes) or ALU (algorithmic flops).

    FP64 mode is compared with the measured native FP64 FMA rate (its flops are FP64-accurate
    operations, carried out in double-float on the FP32 pipes); mixed mode with the FP32 FMA rate.
    """
    avg_ms = site["total_ms"] / site["launches"]
    gbs = site["bytes"] / (avg_ms * 1e-3) / 1e9
    gfl = site["flops"] / (avg_ms * 1e-3) / 1e9
    alu_peak = fp64_peak if prec == "fp64" else fp32_peak
    t_mem = site["bytes"] / (pk["hbm_gbs"] * 1e9)
    t_alu = site["flops"] / (alu_peak * 1e9)
    if t_alu > t_mem:
        r = {"bound": "alu", "achieved": gfl / 1e3, "peak": alu_peak / 1e3, "unit": "TFLOP/s", "frac": gfl / alu_peak,
             "peak_source": ("measured FP64 FMA rate (fsib_measure_peak kind 0)" if prec == "fp64" else
                             "measured FP32 FMA rate (fsib_measure_peak kind 1)")}
    else:
        r = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
             "peak_source": f"MEASURED_PEAKS hbm_gbs ({pk_src})"}
    r.update({"kernel": site["name"], "bytes_per_launch": site["bytes"], "flops_per_launch": site["flops"],
              "avg_launch_ms": avg_ms, "hbm_frac": gbs / pk["hbm_gbs"],
              "alu_frac": gfl / alu_peak if alu_peak else None})
    return r


def measure(fsib, torch, prob, prec, steps, warmup, dev, flush, world=1, barrier=None, sampler_idx=None,
            nufft_reps=20, nprof=20):
    """Time one workload: steps/s (CUDA events around each step, L2 flushed between steps),
    NUFFT pts/s for type-1 and type-2, and the per-launch-site breakdown."""
    stream = torch.cuda.current_stream()
    pb = make_problem(fsib, prob, prec)
    X = torch.from_numpy(prob.X0.copy()).to(dev)
    u = pb.new_spec(device=dev)
    U = pb.interp(u, X)
    t_tune = time.perf_counter()
    shapes = pb.autotune(X, u, U) if prob.rho > 0 else pb.autotune(X)  # on copies; X, u, U unchanged
    t_tune = time.perf_counter() - t_tune
    for _ in range(warmup):
        pb.step(X, u, U, nsteps=1)
    if barrier:
        barrier()
    sampler = ClockSampler(sampler_idx) if sampler_idx is not None else None
    if sampler:
        time.sleep(0.25)
    ev = [_events(torch) for _ in range(steps)]
    if barrier:
        barrier()
    torch.cuda.synchronize()
    t_begin = time.time()
    for s in range(steps):
        flush.zero_()  # L2 flush between timed iterations (outside the events)
        ev[s][0].record(stream)
        pb.step(X, u, U, nsteps=1)
        ev[s][1].record(stream)
    if barrier:
        barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop(t_begin, time.time()) if sampler else None
    ms = sum(a.elapsed_time(b) for a, b in ev)
    launches = int(pb.info("launches_per_step"))
    # NUFFT throughput, type-1 and type-2 separately
    c = pb.force(X)
    fh = pb.new_spec(device=dev)
    t1 = t2 = 0.0
    for r in range(nufft_reps + 2):
        for kind in (1, 2):
            flush.zero_()
            a, b = _events(torch)
            a.record(stream)
            if kind == 1:
                pb.spread(X, c, None, out=fh)
            else:
                pb.interp(u, X, out=U)
            b.record(stream)
            torch.cuda.synchronize()
            if r >= 2:
                if kind == 1:
                    t1 += a.elapsed_time(b)
                else:
                    t2 += a.elapsed_time(b)
    # per-launch-site timing (CUDA events around each launch site, direct launches)
    pb.profile(True)
    pb.profile_reset()
    Xp, up, Up = X.clone(), u.clone(), U.clone()
    for _ in range(nprof):
        flush.zero_()
        pb.step(Xp, up, Up, nsteps=1)
    sites = pb.profile_entries()
    pb.profile(False)
    info = {k: pb.info(k) for k in ("nf", "Nt", "width")}
    return {"pb": pb, "X": X, "u": u, "U": U, "ms": ms, "launches": launches, "clocks": clocks,
            "launch_shapes": dict(shapes, autotune_seconds=round(t_tune, 2)),
            "pts1": prob.M / (t1 / nufft_reps * 1e-3), "pts2": prob.M / (t2 / nufft_reps * 1e-3),
            "sites": sites, "nprof": nprof, "info": info}


def breakdown_of(sites, nprof, top=12):
    tot = sum(s["total_ms"] for s in sites)
    rows = sorted(({"site": s["name"], "ms_per_step": s["total_ms"] / nprof, "share": s["total_ms"] / tot,
                    "gbs": s["bytes"] * s["launches"] / (s["total_ms"] * 1e-3) / 1e9,
                    "gflops": s["flops"] * s["launches"] / (s["total_ms"] * 1e-3) / 1e9}
                   for s in sites), key=lambda z: -z["ms_per_step"])
    return rows[:top]


def rel_err(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def mixed_block(fsib, torch, dev, flush, pk, pk_src, fp64_peak, fp32_peak, steps, warmup):
    """FP32-mixed workload (N = 128^3, M = 40322) with its error against an FP64 run of the same seed."""
    prob = wl.config_ns3d_mixed()
    m = measure(fsib, torch, prob, "mixed", steps, warmup, dev, flush, nufft_reps=10, nprof=10)
    top = max(m["sites"], key=lambda s: s["total_ms"])
    # error report: one transform each, and a few steps from the same initial state
    pm = m["pb"]
    p64 = make_problem(fsib, prob, "fp64")
    X0 = torch.from_numpy(prob.X0.copy()).to(dev)
    c = p64.force(X0)
    f64 = p64.spread(X0, c).cpu().numpy()
    f32 = pm.spread(X0, c).cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(33)
    H = (rng.standard_normal(p64.spec_shape) + 1j * rng.standard_normal(p64.spec_shape)) * 1e-3
    u64 = torch.from_numpy(H).to(dev)
    U64 = p64.interp(u64, X0).cpu().numpy()
    U32 = pm.interp(u64.to(torch.complex64), X0).cpu().numpy()
    nerr = 5
    Xa, ua = X0.clone(), p64.new_spec(device=dev)
    Ua = p64.interp(ua, Xa)
    Xb, ub = X0.clone(), pm.new_spec(device=dev)
    Ub = pm.interp(ub, Xb)
    p64.step(Xa, ua, Ua, nsteps=nerr)
    pm.step(Xb, ub, Ub, nsteps=nerr)
    torch.cuda.synchronize()
    x0 = prob.X0
    errs = {"type1_rel_l2": rel_err(f32, f64), "type2_rel_l2": rel_err(U32, U64),
            f"steps{nerr}_displacement_rel_l2": rel_err(Xb.cpu().numpy() - x0, Xa.cpu().numpy() - x0),
            f"steps{nerr}_uhat_rel_l2": rel_err(ub.cpu().numpy().astype(np.complex128), ua.cpu().numpy())}
    p64.close()
    return {"workload": prob.name, "value": steps / (m["ms"] * 1e-3), "unit": "steps/s",
            "ms_per_step": m["ms"] / steps, "steps": steps, "dtype": "f32 transforms, f64 positions/forces",
            "nufft_pts_per_s": {"type1": m["pts1"], "type2": m["pts2"]},
            "config": {"N": prob.N, "M": prob.M, "tol": prob.tol, **{k: int(v) for k, v in m["info"].items()}},
            "error_vs_fp64_run": errs, "launch_shapes": m["launch_shapes"],
            "roofline": dict(roofline_of(top, "mixed", pk, pk_src, fp64_peak, fp32_peak),
                             traffic=SITE_TRAFFIC.get((prob.name, top["name"])),
                             limiter=SITE_OTHER_BOUND.get((prob.name, top["name"]))),
            "step_roofline": step_roofline(prob, "mixed", m["info"]["nf"], m["info"]["Nt"], m["ms"] / steps, pk),
            "breakdown": breakdown_of(m["sites"], m["nprof"], 8)}


def batched_block(fsib, torch, dev, flush, steps, warmup):
    """64 independent problems (2D/3D, N in {32..128}, M in [128, 20000]), FP32-mixed, autotuned,
    advanced by one CUDA graph launch per step."""
    probs = wl.config_batched()
    n = len(probs)
    B = fsib.Batch([p.N for p in probs], [p.d for p in probs], [p.M for p in probs], [p.mu for p in probs],
                   [p.rho for p in probs], [p.dt for p in probs], [p.tol for p in probs], precision="mixed")
    X, u, U = [], [], []
    for p, m in zip(probs, B.members):
        if p.force == "mesh":
            m.set_force_mesh(p.tri, p.Xref, p.stiffness)
        else:
            m.set_force_curve(p.stiffness)
        Xi = torch.from_numpy(p.X0.copy()).to(dev)
        X.append(Xi)
        u.append(m.new_spec(device=dev))
        U.append(torch.zeros_like(Xi))
    t0 = time.perf_counter()
    B.autotune(X, u, U)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        B.step(X, u, U, nsteps=1)
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = _events(torch)
        a.record(stream)
        B.step(X, u, U, nsteps=1)
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
    ok = all(bool(torch.isfinite(x).all()) for x in X)
    tuned = {}
    for p, m in zip(probs, B.members):
        k = f"{p.d}d_N{p.N}"
        tuned.setdefault(k, {kk: int(m.info(kk)) for kk in ("fft_tile", "fft_rows", "spread_slice")})
    mtot = sum(p.M for p in probs)
    bytes_step = sum(step_bytes(p, "mixed", int(m.info("nf")), int(m.info("Nt"))) for p, m in zip(probs, B.members))
    hbm = float(peaks()[0]["hbm_gbs"])
    gbs = bytes_step / (ms / steps * 1e-3) / 1e9
    out = {"workload": f"batched{n}_mixed", "problems": n, "value": n * steps / (ms * 1e-3),
           "unit": "problem-steps/s", "batch_steps_per_s": steps / (ms * 1e-3), "ms_per_batch_step": ms / steps,
           "boundary_points_per_s": mtot * steps / (ms * 1e-3), "total_points": mtot,
           "launches_per_batch_step": int(B.info("launches_per_step")), "autotune_seconds": tune_s,
           "finite": ok, "n_2d": sum(p.d == 2 for p in probs), "n_3d": sum(p.d == 3 for p in probs),
           "tuned_shapes": tuned,
           "step_roofline": {"algorithmic_bytes_per_batch_step": bytes_step, "achieved_gbs": gbs, "peak_gbs": hbm,
                             "frac": gbs / hbm}}
    B.close()
    return out


def nufft_sweep(fsib, torch, dev, flush, sizes=(10**4, 10**5, 10**6, 10**7, 10**8), reps=3):
    """NUFFT pts/s against M: uniform random points in the unit cube, N = 128^3, FP32-mixed,
    tol 1e-6 (the point-dominated regime). Each transform: sort + spread + FFT passes +
    deconvolution (type 1), or deconvolution + FFT passes + sort + interp (type 2)."""
    stream = torch.cuda.current_stream()
    out = []
    gen = torch.Generator(device=dev)
    for M in sizes:
        gen.manual_seed(8000 + len(out))
        try:
            pb = fsib.Problem(128, 3, M, 1.0, 0.0, 1e-4, 1e-6, precision="mixed")
            X = torch.rand((3, M), generator=gen, device=dev, dtype=torch.float64)
            c = torch.randn((3, M), generator=gen, device=dev, dtype=torch.float64)
            fh = pb.new_spec(device=dev)
            uh = (torch.randn(pb.spec_shape, generator=gen, device=dev, dtype=torch.float32)
                  + 1j * torch.randn(pb.spec_shape, generator=gen, device=dev, dtype=torch.float32)) * 1e-2
            U = torch.empty_like(X)
        except Exception as e:  # noqa: BLE001 - report and go on with the other sizes
            out.append({"M": M, "skipped": str(e)[:200]})
            continue
        t = {1: 0.0, 2: 0.0}
        for r in range(reps + 2):
            for kind in (1, 2):
                flush.zero_()
                a, b = _events(torch)
                a.record(stream)
                if kind == 1:
                    pb.spread(X, c, None, out=fh)
                else:
                    pb.interp(uh, X, out=U)
                b.record(stream)
                torch.cuda.synchronize()
                if r >= 2:
                    t[kind] += a.elapsed_time(b)
        out.append({"M": M, "type1_pts_per_s": M / (t[1] / reps * 1e-3), "type2_pts_per_s": M / (t[2] / reps * 1e-3),
                    "type1_ms": t[1] / reps, "type2_ms": t[2] / reps})
        pb.close()
        del X, c, fh, uh, U
        torch.cuda.empty_cache()
    return {"workload": "uniform random points, N = 128^3, mixed, tol 1e-6", "points": out}


def adjoint_block(fsib, torch, dev, reps=2):
    """Differentiable 3D Stokes (N = 96^3, M = 20002, K = 50, checkpoints every 10): gradient of
    sum_j (|X_j^K - c| - R)^2 w.r.t. X^0 and sigma by the FP32-mixed adjoint, checked against
    central finite differences of the FP64 forward on random directions."""
    prob = wl.config_stokes3d_adjoint()
    K, ck = prob.nsteps, prob.extra["ckpt_every"]
    R = prob.extra["target_radius"]
    center = torch.from_numpy(prob.X0.mean(axis=1)).to(dev)[:, None]
    pm = make_problem(fsib, prob, "mixed")
    p64 = make_problem(fsib, prob, "fp64")
    X0 = torch.from_numpy(prob.X0.copy()).to(dev)
    sigma0 = prob.stiffness

    def loss_grad(pb, x0, sig):
        pb.set_force_mesh(prob.tri, prob.Xref, sig)
        X = x0.clone()
        pb.step(X, nsteps=K)
        r = torch.sqrt(((X - center) ** 2).sum(0))
        e = r - R
        return float((e * e).sum()), (2 * e / r)[None, :] * (X - center)

    L, dLdXK = loss_grad(pm, X0, sigma0)  # warm-up: first-call set-up (graph capture, buffers)
    g0, gs = pm.step_adjoint(X0, K, ck, dLdXK)
    torch.cuda.synchronize()
    t_fwd = t_adj = 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        X = X0.clone()
        pm.step(X, nsteps=K)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        g0, gs = pm.step_adjoint(X0, K, ck, dLdXK)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        t_fwd += (t1 - t0) / reps
        t_adj += (t2 - t1) / reps
    t_mixed = t_fwd + t_adj
    _, dL64 = loss_grad(p64, X0, sigma0)
    g64, gs64 = p64.step_adjoint(X0, K, ck, dL64)
    rng = np.random.default_rng(55)
    checks = []
    eps = 1e-6
    for _ in range(2):
        v = torch.from_numpy(rng.standard_normal(prob.X0.shape)).to(dev)
        lp, _ = loss_grad(p64, X0 + eps * v, sigma0)
        lm, _ = loss_grad(p64, X0 - eps * v, sigma0)
        fd = (lp - lm) / (2 * eps)
        checks.append({"fd": fd, "adjoint_mixed": float((g0 * v).sum()), "adjoint_fp64": float((g64 * v).sum())})
    lp, _ = loss_grad(p64, X0, sigma0 + eps)
    lm, _ = loss_grad(p64, X0, sigma0 - eps)
    fds = (lp - lm) / (2 * eps)
    rel = lambda a, b: abs(a - b) / max(abs(b), 1e-300)
    out = {"workload": prob.name, "K": K, "ckpt_every": ck, "loss": L,
           "seconds_forward_plus_adjoint_mixed": t_mixed, "seconds_forward": t_fwd,
           "seconds_adjoint": t_adj,
           "steps_per_s_forward_plus_adjoint": K / t_mixed,
           "grad_check_fd_fp64": {
               "x0_rel_err_mixed": max(rel(c["adjoint_mixed"], c["fd"]) for c in checks),
               "x0_rel_err_fp64": max(rel(c["adjoint_fp64"], c["fd"]) for c in checks),
               "sigma_rel_err_mixed": rel(float(gs.cpu()), fds), "sigma_rel_err_fp64": rel(float(gs64.cpu()), fds),
               "directions": len(checks)}}
    pm.close()
    p64.close()
    return out


def _chunked_steps(torch, pb, X, u, U, total, chunk, flush, stream, probe=None):
    """Advance `total` steps in graph-replayed chunks; device time of the chunks (L2
    flushed between chunks, outside the events); probe(step) runs after each chunk."""
    ms, done = 0.0, 0
    while done < total:
        n = min(chunk, total - done)
        flush.zero_()
        a, b = _events(torch)
        a.record(stream)
        pb.step(X, u, U, nsteps=n)
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        done += n
        if probe:
            probe(done)
    return ms


def validation_block(fsib, torch, dev, flush, cpu_sample=True):
    """The paper's 2D checks, run on the library (FP64 transforms): sine-velocity circle
    (Sec. 5.2.1: area over T = 10, temporal order at t = 0.1), the Poiseuille channel on
    target-point walls (Sec. 5.2.2: flux against Eq. poiseuille_flux, effective boundary width
    against N), and the Stokes circle with normal and tangent forces (Sec. 6.1: pressure jump,
    convergence studies up to N = 1024, jump widths)."""
    from paper_2302_08694_gb300 import validation as va
    stream = torch.cuda.current_stream()
    out = {}
    # -- circle in the sine flow: N = 64, N_b = 202, dt = 1e-3, T = 10
    prob = wl.config_ns2d_circle()
    pb = make_problem(fsib, prob, "fp64")
    X = torch.from_numpy(prob.X0.copy()).to(dev)
    u = torch.from_numpy(prob.extra["u0"]).to(dev)
    U = pb.interp(u, X)
    A0 = pb.invariants(X)["volume"]
    area = []

    def probe(step):
        area.append(pb.invariants(X)["volume"] / A0)
    ms = _chunked_steps(torch, pb, X, u, U, prob.nsteps, 100, flush, stream, probe)
    Xn = X.cpu().numpy()
    r = np.hypot(Xn[0] - Xn[0].mean(), Xn[1] - Xn[1].mean())
    circle = {"workload": prob.name, "steps": prob.nsteps, "steps_per_s": prob.nsteps / (ms * 1e-3),
              "ms_per_step": ms / prob.nsteps, "timing": "graph replays of 100 steps, L2 flushed between",
              "area_ratio_min": min(area), "area_ratio_max": max(area), "area_ratio_final": area[-1],
              "radius_rel_spread_final": float(r.std() / r.mean())}
    if cpu_sample:
        from oracle import spectral as osp
        from oracle import stepper as ost
        force = ost.curve_model(prob.stiffness)
        Xo = prob.X0.copy()
        uo = osp.half_to_full(prob.extra["u0"], prob.N, 2)
        Uo = osp.interp_direct(uo, Xo, prob.N)
        k = 20
        t0 = time.perf_counter()
        for _ in range(k):
            Xo, uo, Uo = ost.ns_step(Xo, uo, Uo, force, prob.N, prob.mu, prob.rho, prob.dt)
        circle["cpu_baseline"] = {"value": k / (time.perf_counter() - t0), "unit": "steps/s",
                                  "cores": cpu_threads(), "kind": "oracle",
                                  "sample": f"{k} oracle steps of the same workload"}
    # temporal order: dt = 0.002 / 2^j against dt = 0.002 / 64 at t = 0.1 (same N, N_b)
    sols = {}
    for j in (0, 1, 2, 3, 4, 6):
        dt = 0.002 / 2 ** j
        pj = wl.config_ns2d_circle(dt=dt, T=0.1)
        pbj = make_problem(fsib, pj, "fp64")
        Xj = torch.from_numpy(pj.X0.copy()).to(dev)
        uj = torch.from_numpy(pj.extra["u0"]).to(dev)
        Uj = pbj.interp(uj, Xj)
        pbj.step(Xj, uj, Uj, nsteps=pj.nsteps)
        sols[dt] = uj.cpu().numpy()
        pbj.close()
    ref = sols[0.002 / 64]
    errs = {f"{dt:g}": rel_err(v, ref) for dt, v in sols.items() if dt != 0.002 / 64}
    ev = list(errs.values())
    circle["temporal_error_at_t0.1"] = errs
    circle["temporal_order"] = [float(np.log2(a / b)) for a, b in zip(ev[:-1], ev[1:])]
    # space and time together (Fig. spatial_conv): N = 8 * 2^r, N_b = 26 * 2^r, dt = 0.001 / 2^r, T = 0.1
    spectra = []
    for rr in range(6):
        pj = wl.config_ns2d_circle(N=8 * 2 ** rr, Nb=26 * 2 ** rr, dt=0.001 / 2 ** rr, T=0.1)
        pbj = make_problem(fsib, pj, "fp64")
        Xj = torch.from_numpy(pj.X0.copy()).to(dev)
        uj = torch.from_numpy(pj.extra["u0"]).to(dev)
        Uj = pbj.interp(uj, Xj)
        pbj.step(Xj, uj, Uj, nsteps=pj.nsteps)
        spectra.append(uj.cpu().numpy())
        pbj.close()
    se = va.successive_errors(spectra)
    circle["space_time_convergence"] = {"N": [8 * 2 ** rr for rr in range(6)], "successive_rel_l2": se,
                                        "orders": [float(np.log2(a / b)) for a, b in zip(se[:-1], se[1:])]}
    out["sine_circle"] = circle
    pb.close()
    # -- Poiseuille channel: flux history and effective wall width against N
    chan = []
    for N in (8, 16, 32, 64, 128):
        pp = wl.config_poiseuille(N=N)
        ex = pp.extra
        pbp = make_problem(fsib, pp, "fp64")
        Xp = torch.from_numpy(pp.X0.copy()).to(dev)
        up = pbp.new_spec(device=dev)
        Up = pbp.interp(up, Xp)
        D, f0 = ex["D"], ex["f0"]
        steady = va.poiseuille_steady_flux(f0, pp.mu, D)
        marks = {int(round(t / pp.dt)): t for t in (0.05, 0.1, 0.2, 0.5, 1.0, 2.0, 3.0)}
        hist = []

        def probe_c(step, pbp=pbp, up=up, marks=marks, hist=hist, steady=steady):
            if step in marks:
                hist.append((marks[step], pbp.band_flux(up, 0, 1, *ex["band"]) / steady - 1.0))
        chunk = max(1, min(int(round(0.05 / pp.dt)), 1000))
        msp = _chunked_steps(torch, pbp, Xp, up, Up, pp.nsteps, chunk, flush, stream, probe_c)
        flux = pbp.band_flux(up, 0, 1, *ex["band"])
        h = 1.0 / N
        ana = va.poiseuille_flux([t for t, _ in hist], f0, pp.mu, pp.rho, D) / steady - 1.0
        chan.append({"N": N, "Nb": 2 * N, "dt": pp.dt, "steps": pp.nsteps,
                     "steps_per_s": pp.nsteps / (msp * 1e-3),
                     "flux_rel_history": [[t, v, float(a)] for (t, v), a in zip(hist, ana)],
                     "effective_width_over_h": (D - va.effective_width(flux, f0, pp.mu)) / h})
        pbp.close()
    out["poiseuille"] = {"K": wl.config_poiseuille().stiffness, "by_N": chan,
                         "flux_rel_history_columns": ["t", "(Phi - Phi_eq)/Phi_eq FSIB", "same, Eq. poiseuille_flux"]}
    # -- normal-force circle (Sec. 6.1): u = 0 and a pressure jump F/r across the circle
    r, Nb = 0.25, 1024
    th = 2 * np.pi * np.arange(Nb) / Nb
    Xc = torch.from_numpy(np.stack([0.5 + r * np.cos(th), 0.5 + r * np.sin(th)])).to(dev)
    Fc = torch.from_numpy(np.stack([np.cos(th), np.sin(th)])).to(dev)
    wc = torch.full((Nb,), 2 * np.pi / Nb, dtype=torch.float64, device=dev)
    p_in, p_out = -(1 - np.pi * r * r) / r, np.pi * r
    Y = torch.tensor([[0.5, 0.0], [0.5, 0.0]], dtype=torch.float64, device=dev)
    rows = []
    for N in (32, 64, 128, 256):
        pbc = fsib.Problem(N, 2, Nb, 1.0, 0.0, 1e-3, 1e-12)
        fh = pbc.spread(Xc, Fc, wc)
        uc = pbc.new_spec(device=dev)
        pbc.fluid_step(fh, uc)
        P = pbc.pressure_at(pbc.pressure(fh), Y).cpu().numpy()
        rows.append({"N": N, "p_centre": float(P[0]), "p_corner": float(P[1]),
                     "rel_err_centre": float(abs(P[0] - p_in) / abs(p_in)),
                     "rel_err_corner": float(abs(P[1] - p_out) / p_out),
                     "max_abs_u_hat": float(uc.abs().max())})
        pbc.close()
    # width of the pressure jump (Fig. reso_stokes), N and N_b refined together (h_b close to L/N):
    # jump height over the steepest slope, of the band-limited pressure and of its samples on
    # the Eulerian grid of the centreline (central differences over 2h)
    widths = []
    for N in (32, 64, 128, 256):
        Nbw = int(np.ceil(2 * np.pi * r * N))
        thw = 2 * np.pi * np.arange(Nbw) / Nbw
        Xw = torch.from_numpy(np.stack([0.5 + r * np.cos(thw), 0.5 + r * np.sin(thw)])).to(dev)
        Fw = torch.from_numpy(np.stack([np.cos(thw), np.sin(thw)])).to(dev)
        ww = torch.full((Nbw,), 2 * np.pi / Nbw, dtype=torch.float64, device=dev)
        pbw = fsib.Problem(N, 2, Nbw, 1.0, 0.0, 1e-3, 1e-12)
        ph = pbw.pressure(pbw.spread(Xw, Fw, ww))
        h = 1.0 / N
        yf = np.linspace(0.5 + r - 4 * h, 0.5 + r + 4 * h, 801)
        yg = np.arange(N) * h
        Pf = pbw.pressure_at(ph, torch.from_numpy(np.stack([np.full_like(yf, 0.5), yf])).to(dev)).cpu().numpy()
        Pg = pbw.pressure_at(ph, torch.from_numpy(np.stack([np.full_like(yg, 0.5), yg])).to(dev)).cpu().numpy()
        jump = 1.0 / r
        widths.append({"N": N, "Nb": Nbw,
                       "width_over_h_max_slope": float(jump / np.max(np.abs(np.gradient(Pf, yf))) / h),
                       "width_over_h_grid": float(jump / (np.max(np.abs(Pg[2:] - Pg[:-2])) / (2 * h)) / h)})
        pbw.close()
    out["normal_circle_pressure"] = {"r": r, "Nb": Nb, "F": 1.0, "p_inside_exact": p_in, "p_outside_exact": p_out,
                                     "by_N": rows, "jump_width": widths}
    out["stokes_circle"] = stokes_circle_block(fsib, torch, dev)
    out["steady_poiseuille"] = steady_channel_block(fsib, torch, dev)
    return out


def stokes_circle_block(fsib, torch, dev):
    """The paper's 2D Stokes circle studies (Sec. 6.1) on the library (FP64 transforms, Stokes,
    mu = 1): a circle of radius r = L/4 at the centre carries N_b points with a unit force per
    unit theta (weights 2 pi / N_b), either along the outward normal ('normal': u = 0, pressure
    jump F/r) or along the clockwise tangent ('tangent': p constant, a circulating flow).
    Reported: the coupling study at fixed N_b = 64 with N = 4 .. 1024, the first-order study with
    N and N_b refined together (N = 8 .. 1024), the exponential convergence in N_b at N = 128,
    and the width of the jump of du_x/dy across the circle on the vertical centreline."""
    r = 0.25

    def circle(Nb, kind):
        th = 2 * np.pi * np.arange(Nb) / Nb
        X = np.stack([0.5 + r * np.cos(th), 0.5 + r * np.sin(th)])
        F = np.stack([np.cos(th), np.sin(th)]) if kind == "normal" else np.stack([np.sin(th), -np.cos(th)])
        w = np.full(Nb, 2 * np.pi / Nb)
        return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (X, F, w)]

    def solve(N, Nb, kind):
        """(problem, f-hat, u-hat, U at the points) of one Stokes solve."""
        X, F, w = circle(Nb, kind)
        pb = fsib.Problem(N, 2, Nb, 1.0, 0.0, 1e-3, 1e-12)
        fh = pb.spread(X, F, w)
        uh = pb.new_spec(device=dev)
        pb.fluid_step(fh, uh)
        return pb, fh, uh, pb.interp(uh, X)

    def at(N, spec, Y):
        """Both components of a half spectrum at the points Y ([2][n])."""
        probe = fsib.Problem(N, 2, Y.shape[1], 1.0, 0.0, 1e-3, 1e-12)
        V = probe.interp(spec, torch.from_numpy(np.ascontiguousarray(Y)).to(dev)).cpu().numpy()
        probe.close()
        return V

    def grid_points(N):
        g = np.arange(N) / N
        gy, gx = np.meshgrid(g, g, indexing="ij")
        return np.stack([gx.ravel(), gy.ravel()])

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    p_in, p_out = -(1 - np.pi * r * r) / r, np.pi * r
    out = {"r": r, "mu": 1.0, "F": 1.0}
    # -- coupling of L/N and h_b: N_b = 64, N = 4 .. 1024 (Fig. circle:error_Nh)
    Nb, Ns = 64, [2 ** k for k in range(2, 11)]
    Nfine = Ns[-1]
    _, _, ut_fine, Ut_fine = solve(Nfine, Nb, "tangent")
    Ut_fine = Ut_fine.cpu().numpy()
    rows = []
    for N in Ns:
        Yg = grid_points(N)
        inside = np.hypot(Yg[0] - 0.5, Yg[1] - 0.5) < r
        pbn, fhn, uhn, _ = solve(N, Nb, "normal")
        P = at(N, torch.stack([pbn.pressure(fhn), torch.zeros_like(uhn[1])]), Yg)[0]
        pex = np.where(inside, p_in, p_out)
        pbt, fht, uht, Ut = solve(N, Nb, "tangent")
        row = {"N": N, "h_b_over_h": 2 * np.pi * r / Nb * N,
               "normal_p_grid_rel_err": rel(P, pex),
               "normal_u_hat_max": float(uhn.abs().max()),
               "tangent_p_hat_max": float(pbt.pressure(fht).abs().max())}
        if N < Nfine:
            row["tangent_U_points_rel_diff_vs_N1024"] = rel(Ut.cpu().numpy(), Ut_fine)
            row["tangent_u_grid_rel_diff_vs_N1024"] = rel(at(N, uht, Yg), at(Nfine, ut_fine, Yg))
        rows.append(row)
        pbn.close()
        pbt.close()
    out["coupling_Nb64"] = rows
    # -- N and N_b refined together, tangent case (Fig. u_Nh_h_comp): successive differences of U
    # at the coarse points (theta_j of N_b is theta_2j of 2 N_b)
    Us, diffs = [], []
    for k in range(8):
        N, Nbk = 8 * 2 ** k, 4 * 2 ** k
        pbk, _, _, Uk = solve(N, Nbk, "tangent")
        Us.append(Uk.cpu().numpy())
        pbk.close()
    for k in range(7):
        diffs.append(rel(Us[k], Us[k + 1][:, ::2]))
    out["tangent_refined_together"] = {
        "N": [8 * 2 ** k for k in range(8)], "Nb": [4 * 2 ** k for k in range(8)],
        "successive_rel_diff": diffs,
        "orders": [float(np.log2(diffs[k] / diffs[k + 1])) for k in range(6)]}
    # -- exponential convergence in N_b at N = 128 (Fig. err_2_N): centreline x = L/2, grid y
    N = 128
    Yc = np.stack([np.full(N, 0.5), np.arange(N) / N])
    pexc = np.where(np.abs(Yc[1] - 0.5) < r, p_in, p_out)
    perr, udiff, uprev, un, pt = [], [], None, [], []
    for Nbk in (4, 8, 16, 32, 64):
        pbn, fhn, uhn, _ = solve(N, Nbk, "normal")
        perr.append(rel(at(N, torch.stack([pbn.pressure(fhn), torch.zeros_like(uhn[1])]), Yc)[0], pexc))
        un.append(float(np.max(np.abs(at(N, uhn, Yc)))))
        pbt, fht, uht, _ = solve(N, Nbk, "tangent")
        ux = at(N, uht, Yc)[0]
        pt.append(float(np.max(np.abs(at(N, torch.stack([pbt.pressure(fht), torch.zeros_like(uht[1])]), Yc)[0]))))
        if uprev is not None:
            udiff.append(rel(uprev, ux))
        uprev = ux
        pbn.close()
        pbt.close()
    out["Nb_convergence_N128"] = {"Nb": [4, 8, 16, 32, 64], "normal_p_centreline_rel_err": perr,
                                  "normal_u_centreline_max": un, "tangent_p_centreline_max": pt,
                                  "tangent_ux_centreline_successive_rel_diff": udiff}
    # -- width of the jump of du_x/dy (Fig. reso_stokes, tangent case): the jump (F/(mu r)) over
    # the steepest slope of du_x/dy on a fine probe line across the top of the circle
    widths = []
    for N in (32, 64, 128, 256):
        Nbw = int(np.ceil(2 * np.pi * r * N))
        pbw, _, uhw, _ = solve(N, Nbw, "tangent")
        h = 1.0 / N
        yf = np.linspace(0.5 + r - 4 * h, 0.5 + r + 4 * h, 801)
        ux = at(N, uhw, np.stack([np.full_like(yf, 0.5), yf]))[0]
        d1 = np.gradient(ux, yf)
        yg = np.arange(N) * h
        ug = at(N, uhw, np.stack([np.full_like(yg, 0.5), yg]))[0]
        dg = (ug[2:] - ug[:-2]) / (2 * h)            # du_x/dy on the grid, central differences
        widths.append({"N": N, "Nb": Nbw,
                       "width_over_h_max_slope": float((1.0 / r) / np.max(np.abs(np.gradient(d1, yf))) / h),
                       "width_over_h_grid": float((1.0 / r) / (np.max(np.abs(dg[2:] - dg[:-2])) / (2 * h)) / h),
                       "dux_dy_change_over_8h": float(d1[-1] - d1[0])})
        pbw.close()
    out["tangent_dux_dy_jump_width"] = widths
    return out


def steady_channel_block(fsib, torch, dev):
    """The paper's steady Poiseuille convergence study (Sec. 5.2.2): a channel of width D = L
    bounded by one wall at y = 0 (periodic in y), mu = 0.1, f0 = 100, N = N_b = 8 .. 512, on the
    library's Stokes path (FP64 transforms). At equilibrium the wall carries the force that
    balances the body force, the same on every marker (the markers X_i = (i h, 0) are
    equispaced), so it is spread with omega = h; the Stokeslet drops the k = 0 mode, so the
    uniform body force acts only through the mean flow, which the no-slip condition fixes:
    u = u_S - U_S(X_wall). Errors: relative 2-norm on the Eulerian grid of the line x = L/2
    against Eq. steady_poiseuille_velo, with D and with the effective width D_e of the computed
    flux (walls moved by (D - D_e)/2 into the fluid)."""
    mu, f0, L = 0.1, 100.0, 1.0
    rows = []
    for k in range(7):
        N = 8 * 2 ** k
        h = L / N
        X = np.stack([np.arange(N) * h, np.zeros(N)])
        F = np.stack([np.full(N, -f0 * L * L / (N * h)), np.zeros(N)])   # sum_i omega F_i = -f0 L^2
        Xt, Ft, wt = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (X, F, np.full(N, h))]
        pb = fsib.Problem(N, 2, N, mu, 0.0, 1e-3, 1e-12)
        uh = pb.new_spec(device=dev)
        pb.fluid_step(pb.spread(Xt, Ft, wt), uh)
        ubar = -float(pb.interp(uh, Xt)[0].mean())
        pb.close()
        yg = np.arange(N) * h
        probe = fsib.Problem(N, 2, N, mu, 0.0, 1e-3, 1e-12)
        ug = probe.interp(uh, torch.from_numpy(np.stack([np.full(N, 0.5), yg])).to(dev))[0].cpu().numpy() + ubar
        probe.close()
        flux = ubar * L   # the non-zero y modes integrate to zero over a period
        De = (12.0 * mu * flux / f0) ** (1.0 / 3.0)
        dlt = 0.5 * (L - De)
        u_ex = f0 / (2 * mu) * yg * (L - yg)
        u_e = np.where((yg > dlt) & (yg < L - dlt), f0 / (2 * mu) * (yg - dlt) * (L - dlt - yg), 0.0)
        rows.append({"N": N, "Nb": N, "rel_err": float(np.linalg.norm(ug - u_ex) / np.linalg.norm(u_ex)),
                     "rel_err_effective_width": float(np.linalg.norm(ug - u_e) / np.linalg.norm(u_e)),
                     "effective_width_over_h": (L - De) / h})
    e = [r["rel_err"] for r in rows]
    ee = [r["rel_err_effective_width"] for r in rows]
    return {"mu": mu, "f0": f0, "D": L, "by_N": rows,
            "orders": [float(np.log2(e[i] / e[i + 1])) for i in range(len(e) - 1)],
            "orders_effective_width": [float(np.log2(ee[i] / ee[i + 1])) for i in range(len(ee) - 1)]}


def validation_3d_block(fsib, torch, dev, flush, max_refine=5):
    """The paper's 3D sphere checks on the library (FP64 transforms): a sphere of radius L/3 in
    the sine flow, elastic (Sec. 6.2.3) and surface tension (Sec. 6.2.4). Paper configuration
    (N = 32, four refinements, dt = 1e-3, T = 1): volume over the run; convergence study
    (N = 4 * 2^r, r + 1 refinements, dt = 0.004 / 2^r, T = 0.2): successive relative L2
    differences of the velocity field and their orders."""
    from paper_2302_08694_gb300 import validation as va
    stream = torch.cuda.current_stream()
    out = {}
    for model in ("elastic", "tension"):
        prob = wl.config_ns3d_sphere(model)
        pb = make_problem(fsib, prob, "fp64")
        X = torch.from_numpy(prob.X0.copy()).to(dev)
        u = torch.from_numpy(prob.extra["u0"]).to(dev)
        U = pb.interp(u, X)
        V0 = pb.invariants(X)["volume"]
        vol = []

        def probe(step):
            vol.append(pb.invariants(X)["volume"] / V0)
        ms = _chunked_steps(torch, pb, X, u, U, prob.nsteps, 100, flush, stream, probe)
        Xn = X.cpu().numpy()
        r = np.linalg.norm(Xn - Xn.mean(axis=1, keepdims=True), axis=0)
        res = {"workload": prob.name, "M": prob.M, "steps": prob.nsteps, "steps_per_s": prob.nsteps / (ms * 1e-3),
               "ms_per_step": ms / prob.nsteps, "volume_ratio_min": min(vol), "volume_ratio_max": max(vol),
               "volume_ratio_final": vol[-1], "radius_rel_spread_final": float(r.std() / r.mean())}
        pb.close()
        spectra, rows = [], []
        for rr in range(max_refine + 1):
            N, level, dt = 4 * 2 ** rr, 1 + rr, 0.004 / 2 ** rr
            pr = wl.config_ns3d_sphere(model, level=level, N=N, dt=dt, T=0.2)
            pbr = make_problem(fsib, pr, "fp64")
            Xr = torch.from_numpy(pr.X0.copy()).to(dev)
            ur = torch.from_numpy(pr.extra["u0"]).to(dev)
            Ur = pbr.interp(ur, Xr)
            V0r = pbr.invariants(Xr)["volume"]
            a, b = _events(torch)
            a.record(stream)
            pbr.step(Xr, ur, Ur, nsteps=pr.nsteps)
            b.record(stream)
            torch.cuda.synchronize()
            rows.append({"N": N, "M": pr.M, "dt": dt, "steps": pr.nsteps,
                         "ms_per_step": a.elapsed_time(b) / pr.nsteps,
                         "volume_ratio_final": pbr.invariants(Xr)["volume"] / V0r})
            spectra.append(ur.cpu().numpy())
            pbr.close()
        errs = va.successive_errors(spectra)
        res["convergence"] = {"runs": rows, "successive_rel_l2": errs,
                              "orders": [float(np.log2(x / y)) for x, y in zip(errs[:-1], errs[1:])]}
        out[model] = res
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2302_08694_gb300 import fsib

    rank, local, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if \
        os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    prob, prec = workload_of(args.workload)
    m = measure(fsib, torch, prob, prec, args.steps, args.warmup, dev, flush, world, barrier, gpu_index)
    pb = m["pb"]
    ms_max = max_over_ranks(m["ms"], world, dev)
    value = replica_value(args.steps, ms_max, world)

    pk, pk_src = peaks()
    fp64_peak = fsib.measure_peak(0)  # GFLOP/s
    fp32_peak = fsib.measure_peak(1)
    top = max(m["sites"], key=lambda s: s["total_ms"])
    roof = roofline_of(top, prec, pk, pk_src, fp64_peak, fp32_peak)
    roof.update({"traffic": SITE_TRAFFIC.get((prob.name, top["name"])),
                 "limiter": SITE_OTHER_BOUND.get((prob.name, top["name"])),
                 "share": top["total_ms"] / sum(s["total_ms"] for s in m["sites"]),
                 "fp64_fma_peak_tflops": fp64_peak / 1e3, "fp32_fma_peak_tflops": fp32_peak / 1e3})

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

    mixed = None
    if not args.no_mixed:
        mixed = mixed_block(fsib, torch, dev, flush, pk, pk_src, fp64_peak, fp32_peak,
                            steps=max(3, min(args.steps, 50)), warmup=max(3, args.warmup))
        mixed["value"] *= world
        mixed["nufft_pts_per_s"] = {k: v * world for k, v in mixed["nufft_pts_per_s"].items()}

    batched = None
    if not args.no_batched:
        batched = batched_block(fsib, torch, dev, flush, steps=max(3, min(args.steps, 20)), warmup=max(3, args.warmup))
        for k in ("value", "batch_steps_per_s", "boundary_points_per_s"):
            batched[k] *= world

    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_block(fsib, torch, dev)

    sweep = None
    if not args.no_sweep:
        sweep = nufft_sweep(fsib, torch, dev, flush)

    validation = validation_3d = None
    if not args.no_validation and rank == 0 and world == 1:
        validation = validation_block(fsib, torch, dev, flush, cpu_sample=not args.no_cpu_baseline)
        validation_3d = validation_3d_block(fsib, torch, dev, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and prec == "fp64":
        k = 2 if prob.d == 3 else 20
        t = time_oracle_steps(prob, k)
        cpu = {"value": k / t, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{k} full oracle steps of the same workload (direct non-uniform sums, numpy BLAS/FFT)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": prob.name, "d": prob.d, "N": prob.N, "M": prob.M,
                           **{k: int(v) for k, v in m["info"].items()}, "tol": prob.tol,
                           "arithmetic": ("double-float transforms (FP64-accurate), FP64 positions/forces"
                                          if prec == "fp64" else "FP32 transforms, FP64 positions/forces"),
                           "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas{world}"},
                "nufft_pts_per_s": {"type1": world * m["pts1"], "type2": world * m["pts2"]},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": m["clocks"],
                "step_roofline": step_roofline(prob, prec, m["info"]["nf"], m["info"]["Nt"], ms_max / args.steps, pk),
                "gpu_launches": m["launches"] * args.steps, "launches_per_step": m["launches"],
                "launch_shapes": m["launch_shapes"],
                "breakdown": breakdown_of(m["sites"], m["nprof"]), "mixed": mixed, "batched": batched, "nufft_sweep": sweep,
                "adjoint": adjoint, "validation_2d": validation,
                "validation_3d": validation_3d}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    global NATIVE_FP64
    args = parse()
    NATIVE_FP64 = args.native_fp64
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
