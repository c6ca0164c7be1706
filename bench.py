"""FSIB time-step benchmark on GB300.

Headline workload: 3D Navier-Stokes in the FP64 form, periodic unit cube, N = 64^3
modes, lat-long elastic membrane of M = 10082 points (radius 0.25, seeded ellipsoid),
cot-weight springs sigma = 1, rho = 1, mu = 0.01, dt = 1e-4, NUFFT tol 1e-12. A step
is one full FSIB time step (Algorithm 1): force, type-1 NUFFT, two dealiased V-hat
solves with BE/CN updates, two type-2 NUFFTs, position updates.

The FP64 form computes its transforms in double-float arithmetic (pairs of floats,
"df64"); the native-FP64 arithmetic of the same form, the FP32-mixed form (N = 128^3,
M = 40322) and the batched form (64 uneven problems) are measured beside it.

python bench.py --gpus N --steps K --warmup W [--impl reference] [--detail PATH]

Prints one compact JSON line (rank 0), last on stdout. --detail PATH writes the long
report (per-site breakdowns, launch shapes, optional adjoint and NUFFT-sweep blocks)
to PATH instead. Under torchrun every rank advances its own independent replica of
the workload (the problem does not shard: replicas only).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2302_08694_gb300 import workloads as wl  # noqa: E402

METRIC = "FSIB steps/s and NUFFT pts/s, FP32-mixed & batched vs FP64 at stated error"
L2_FLUSH_BYTES = 512 * 1024 * 1024  # > 129 MB L2

# GB300 unit counts and clock (sm_103a): 152 SMs, 128 FP32 lanes per SM, 2070 MHz maximum SM
# clock. A double-float multiply-add into an accumulator (TwoProd, two cross-term FMAs, TwoSum of
# the high parts, two adds of the low parts) issues 12 FP32-pipe instructions, so the df64 peak is
# the FP32 instruction rate / 12 multiply-adds, 2 flops each.
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
DF64_FP32_INSTR_PER_FMA = 12
DF64_PEAK_GFLOPS = SM_COUNT * FP32_LANES * SM_MAX_GHZ * 2.0 / DF64_FP32_INSTR_PER_FMA


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--native-fp64", action="store_true",
                    help="headline FP64 form in native FP64 arithmetic instead of double-float")
    ap.add_argument("--no-native", action="store_true", help="skip the native-FP64 sub-object")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32-mixed sub-object")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched sub-object")
    ap.add_argument("--adjoint", action="store_true", help="time the differentiable workload (detail file)")
    ap.add_argument("--sweep", action="store_true", help="NUFFT point-count sweep (detail file)")
    ap.add_argument("--detail", default=None, help="write the long report (JSON) to this path")
    ap.add_argument("--batch-size", type=int, default=64,
                    help="problems of the batched workload taken (the first K of its 64; profiling runs)")
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


def make_problem(fsib, prob, precision, native=False):
    pb = fsib.Problem(prob.N, prob.d, prob.M, prob.mu, prob.rho, prob.dt,
                      1e-12 if precision == "fp64" else 1e-6, precision=precision)
    if precision == "fp64" and native:
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


def initial_spectrum(prob):
    """u-hat at t = 0 as a half spectrum (zero unless the workload starts from a flow)."""
    if "u0" in prob.extra:
        return prob.extra["u0"].copy()
    return np.zeros((prob.d,) + (prob.N,) * (prob.d - 1) + (prob.N // 2,), dtype=complex)


def oracle_steps(prob, nsteps):
    """The FP64 oracle (direct non-uniform sums, numpy BLAS/FFT) advanced nsteps from the
    workload's initial state: (seconds, X, full-spectrum u-hat or None)."""
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
    u = sp.half_to_full(initial_spectrum(prob), N, d)
    U = sp.interp_direct(u, X, N) if "u0" in prob.extra else np.zeros_like(X)
    fbody = prob.extra.get("fbody")
    t0 = time.perf_counter()
    for _ in range(nsteps):
        if prob.rho > 0:
            X, u, U = st.ns_step(X, u, U, force, N, prob.mu, prob.rho, prob.dt, fbody=fbody)
        else:
            X = st.stokes_step(X, force, N, prob.mu, prob.dt)
    return time.perf_counter() - t0, X, (u if prob.rho > 0 else None)


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
    """The reference arm: the FP64 oracle timed on the host cores, on the same workload."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    prob, _ = workload_of(args.workload if args.workload != "ns3d_mixed" else "ns3d_fp64")
    k = max(1, min(args.steps, 10))
    w = min(args.warmup, 1)
    if w:
        oracle_steps(prob, w)
    t, _, _ = oracle_steps(prob, k)
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


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the site's dominant
# kernel, from one ncu --set full capture of the current kernels per workload
# (profiles/kernel_spread_df64_ns3d_N64_M10082.txt, profiles/kernel_product_pass_mixed_ns3d_N128_M40322.txt).
# Set an entry to None when those kernels change.
SITE_TRAFFIC = {("ns3d_N64_M10082_fp64", "spread"): 6731776.0,
                ("ns3d_N128_M40322_mixed", "nl.rows_product"): 118960128.0}
# What limits a site when it is not its roofline, from the same captures.
SITE_LIMITER = {("ns3d_N128_M40322_mixed", "nl.rows_product"):
                {"unit": "L1/shared memory", "frac": 0.644, "metric": "l1tex__throughput"},
                ("ns3d_N64_M10082_fp64", "spread"):
                {"unit": "instruction issue", "frac": 0.561, "metric": "sm__issue_active"}}


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
    return {"bytes": b, "achieved_gbs": gbs, "frac": gbs / hbm}


def alu_peak_of(arith, fp64_peak, fp32_peak):
    """(GFLOP/s, description) of the arithmetic pipe a transform kernel runs on."""
    if arith == "df64":
        return DF64_PEAK_GFLOPS, (f"double-float multiply-adds: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x "
                                  f"{SM_MAX_GHZ} GHz / {DF64_FP32_INSTR_PER_FMA} instructions x 2 flops")
    if arith == "f64":
        return fp64_peak, "measured FP64 FMA rate (fsib_measure_peak kind 0)"
    return fp32_peak, "measured FP32 FMA rate (fsib_measure_peak kind 1)"


def roofline_of(site, arith, pk, pk_src, fp64_peak, fp32_peak, workload):
    """Binding roofline of one launch site: HBM (algorithmic bytes) or ALU (algorithmic flops
    against the pipe its arithmetic runs on: df64 on the FP32 pipes, f64 on the FP64 pipes,
    f32 on the FP32 pipes)."""
    avg_ms = site["total_ms"] / site["launches"]
    gbs = site["bytes"] / (avg_ms * 1e-3) / 1e9
    gfl = site["flops"] / (avg_ms * 1e-3) / 1e9
    alu_peak, alu_src = alu_peak_of(arith, fp64_peak, fp32_peak)
    t_mem = site["bytes"] / (pk["hbm_gbs"] * 1e9)
    t_alu = site["flops"] / (alu_peak * 1e9)
    if t_alu > t_mem:
        r = {"bound": "alu", "achieved": gfl / 1e3, "peak": alu_peak / 1e3, "unit": "TFLOP/s",
             "frac": gfl / alu_peak, "peak_source": alu_src}
    else:
        r = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
             "peak_source": f"MEASURED_PEAKS hbm_gbs ({pk_src})"}
    r.update({"kernel": site["name"], "avg_launch_ms": avg_ms, "hbm_frac": gbs / pk["hbm_gbs"],
              "traffic": SITE_TRAFFIC.get((workload, site["name"]))})
    lim = SITE_LIMITER.get((workload, site["name"]))
    if lim:
        r["limiter"] = lim
    return r


def timed_steps(torch, pb, X, u, U, steps, flush, stream, label="timed"):
    """Device time (ms) of `steps` single steps, CUDA events on the launching stream around
    each step, L2 flushed between steps (outside the events). The steps sit in an NVTX range
    named `label`, so a profiler can capture them alone (ncu --nvtx --nvtx-include label/)."""
    ev = [_events(torch) for _ in range(steps)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push(label)
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        pb.step(X, u, U, nsteps=1)
        ev[s][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def nufft_rates(torch, pb, X, u, U, M, flush, stream, reps):
    """NUFFT pts/s (M / time of one call) for type-1 and type-2 separately."""
    c = pb.force(X)
    fh = pb.new_spec(device=X.device)
    t = {1: 0.0, 2: 0.0}
    for r in range(reps + 2):
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
                t[kind] += a.elapsed_time(b)
    return M / (t[1] / reps * 1e-3), M / (t[2] / reps * 1e-3)


def site_profile(pb, X, u, U, flush, nprof):
    """Per-launch-site device times (CUDA events around each launch site, direct launches)."""
    pb.profile(True)
    pb.profile_reset()
    Xp, up, Up = X.clone(), u.clone(), U.clone()
    for _ in range(nprof):
        flush.zero_()
        pb.step(Xp, up, Up, nsteps=1)
    sites = pb.profile_entries()
    pb.profile(False)
    return sites


def measure(fsib, torch, prob, prec, steps, warmup, dev, flush, barrier=None, sampler_idx=None,
            nufft_reps=20, nprof=20, native=False, label="timed"):
    """Time one workload: steps/s (CUDA events around each step, L2 flushed between steps),
    NUFFT pts/s for type-1 and type-2, and the per-launch-site breakdown."""
    stream = torch.cuda.current_stream()
    pb = make_problem(fsib, prob, prec, native)
    X = torch.from_numpy(prob.X0.copy()).to(dev)
    u = torch.from_numpy(initial_spectrum(prob)).to(device=dev, dtype=pb.spec_dtype)
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
    if barrier:
        barrier()
    t_begin = time.time()
    ms = timed_steps(torch, pb, X, u, U, steps, flush, stream, label)
    if barrier:
        barrier()
    clocks = sampler.stop(t_begin, time.time()) if sampler else None
    launches = int(pb.info("launches_per_step"))
    pts1, pts2 = nufft_rates(torch, pb, X, u, U, prob.M, flush, stream, nufft_reps)
    sites = site_profile(pb, X, u, U, flush, nprof) if nprof else []
    info = {k: int(pb.info(k)) for k in ("nf", "Nt", "width")}
    return {"pb": pb, "X": X, "u": u, "U": U, "ms": ms, "launches": launches, "clocks": clocks,
            "launch_shapes": dict(shapes, autotune_seconds=round(t_tune, 2)),
            "pts1": pts1, "pts2": pts2, "sites": sites, "nprof": nprof, "info": info}


def breakdown_of(sites, nprof, top=12):
    tot = sum(s["total_ms"] for s in sites)
    rows = sorted(({"site": s["name"], "ms_per_step": s["total_ms"] / nprof, "share": s["total_ms"] / tot,
                    "gbs": s["bytes"] * s["launches"] / (s["total_ms"] * 1e-3) / 1e9,
                    "gflops": s["flops"] * s["launches"] / (s["total_ms"] * 1e-3) / 1e9}
                   for s in sites), key=lambda z: -z["ms_per_step"])
    return rows[:top]


def rel_err(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_steps_from_start(torch, pb, prob, nsteps, dev):
    """(X, u-hat half spectrum as complex128 numpy) after nsteps library steps from the
    workload's initial state."""
    X = torch.from_numpy(prob.X0.copy()).to(dev)
    u = torch.from_numpy(initial_spectrum(prob)).to(device=dev, dtype=pb.spec_dtype)
    U = pb.interp(u, X)
    pb.step(X, u, U, nsteps=nsteps)
    torch.cuda.synchronize()
    return X.cpu().numpy(), u.cpu().numpy().astype(np.complex128)


def error_vs_oracle(prob, Xo, uo, X, u):
    """Relative 2-norm errors of a library state against the oracle's after the same steps:
    the displacement X - X0 and (Navier-Stokes) the spectrum u-hat."""
    from oracle import spectral as sp
    e = {"displacement_rel_l2": rel_err(X - prob.X0, Xo - prob.X0)}
    if uo is not None:
        e["uhat_rel_l2"] = rel_err(sp.half_to_full(u, prob.N, prob.d), uo)
    return e


def native_block(fsib, torch, prob, dev, flush, steps, warmup, pk, pk_src, fp64_peak, fp32_peak):
    """The FP64 form with its transforms in native FP64 arithmetic (same workload, tuned)."""
    m = measure(fsib, torch, prob, "fp64", steps, warmup, dev, flush, nufft_reps=5, nprof=5, native=True,
                label="native_timed")
    top = max(m["sites"], key=lambda s: s["total_ms"])
    r = roofline_of(top, "f64", pk, pk_src, fp64_peak, fp32_peak, None)
    out = {"value": steps / (m["ms"] * 1e-3), "unit": "steps/s", "ms_per_step": m["ms"] / steps, "steps": steps,
           "dtype": "f64", "nufft_pts_per_s": {"type1": m["pts1"], "type2": m["pts2"]},
           "roofline": {k: r[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac")}}
    return out, m


def mixed_block(fsib, torch, dev, flush, pk, pk_src, fp64_peak, fp32_peak, steps, warmup):
    """FP32-mixed workload (N = 128^3, M = 40322) with its error against an FP64 run of the same seed."""
    prob = wl.config_ns3d_mixed()
    m = measure(fsib, torch, prob, "mixed", steps, warmup, dev, flush, nufft_reps=10, nprof=10, label="mixed_timed")
    top = max(m["sites"], key=lambda s: s["total_ms"])
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
    Xa, ua = gpu_steps_from_start(torch, p64, prob, nerr, dev)
    Xb, ub = gpu_steps_from_start(torch, pm, prob, nerr, dev)
    x0 = prob.X0
    errs = {"type1_rel_l2": rel_err(f32, f64), "type2_rel_l2": rel_err(U32, U64),
            f"steps{nerr}_displacement_rel_l2": rel_err(Xb - x0, Xa - x0),
            f"steps{nerr}_uhat_rel_l2": rel_err(ub, ua)}
    p64.close()
    r = roofline_of(top, "f32", pk, pk_src, fp64_peak, fp32_peak, prob.name)
    sr = step_roofline(prob, "mixed", m["info"]["nf"], m["info"]["Nt"], m["ms"] / steps, pk)
    line = {"workload": prob.name, "value": steps / (m["ms"] * 1e-3), "unit": "steps/s",
            "ms_per_step": m["ms"] / steps, "steps": steps, "dtype": "f32",
            "nufft_pts_per_s": {"type1": m["pts1"], "type2": m["pts2"]},
            "error_vs_fp64_run": errs,
            "roofline": {k: r.get(k) for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic")},
            "step_hbm_frac": sr["frac"], "gpu_launches": m["launches"] * steps}
    detail = {"config": {"N": prob.N, "M": prob.M, "tol": prob.tol, **m["info"]}, "launch_shapes": m["launch_shapes"],
              "roofline": r, "step_roofline": sr, "breakdown": breakdown_of(m["sites"], m["nprof"], 10)}
    m["pb"].close()
    return line, detail


def batched_block(fsib, torch, dev, flush, steps, warmup, pk, size=64):
    """64 independent problems (2D/3D, N in {32..128}, M in [128, 20000]), FP32-mixed, autotuned,
    advanced by one CUDA graph launch per step (`size` < 64: the first `size` of them)."""
    probs = wl.config_batched()[:size]
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
    ev = [_events(torch) for _ in range(steps)]
    torch.cuda.nvtx.range_push("batched_timed")
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        B.step(X, u, U, nsteps=1)
        ev[s][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ok = all(bool(torch.isfinite(x).all()) for x in X)
    tuned = {}
    for p, m in zip(probs, B.members):
        k = f"{p.d}d_N{p.N}"
        tuned.setdefault(k, {kk: int(m.info(kk)) for kk in ("fft_tile", "fft_rows", "spread_slice")})
    mtot = sum(p.M for p in probs)
    bytes_step = sum(step_bytes(p, "mixed", int(m.info("nf")), int(m.info("Nt"))) for p, m in zip(probs, B.members))
    gbs = bytes_step / (ms / steps * 1e-3) / 1e9
    launches = int(B.info("launches_per_step"))
    line = {"workload": f"batched{n}_mixed", "problems": n, "value": n * steps / (ms * 1e-3),
            "unit": "problem-steps/s", "ms_per_batch_step": ms / steps,
            "boundary_points_per_s": mtot * steps / (ms * 1e-3), "dtype": "f32",
            "launches_per_batch_step": launches, "gpu_launches": launches * steps,
            "step_hbm_frac": round(gbs / float(pk["hbm_gbs"]), 4), "finite": ok}
    detail = {"total_points": mtot, "n_2d": sum(p.d == 2 for p in probs), "n_3d": sum(p.d == 3 for p in probs),
              "autotune_seconds": tune_s, "tuned_shapes": tuned, "algorithmic_bytes_per_batch_step": bytes_step,
              "achieved_gbs": gbs}
    B.close()
    return line, detail


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


def e2e_of(torch, pb, prob, steps, world):
    """Steps/s through the public API with page-locked host buffers: every step copies
    (X, u-hat, U) in, runs, and copies them back, inside the timed region."""
    Xh = torch.from_numpy(prob.X0.copy()).pin_memory()
    uh = torch.from_numpy(initial_spectrum(prob)).to(dtype=pb.spec_dtype).pin_memory()
    Uh = torch.zeros_like(Xh).pin_memory()
    pb.interp(uh, Xh, out=Uh)
    ke = max(3, min(steps, 30))
    pb.step(Xh, uh, Uh, nsteps=1)
    t0 = time.perf_counter()
    for _ in range(ke):
        pb.step(Xh, uh, Uh, nsteps=1)  # H2D of (X, u-hat, U), step, D2H, synchronous
    te = time.perf_counter() - t0
    nb = Xh.numel() * 8 + uh.numel() * uh.element_size() + Uh.numel() * 8
    return {"value": world * ke / te, "unit": "steps/s", "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
            "steps": ke, "timing": "host wall clock around synchronous fsib_step calls on pinned host arrays"}


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
    native = args.native_fp64 and prec == "fp64"
    arith = "f32" if prec == "mixed" else ("f64" if native else "df64")
    m = measure(fsib, torch, prob, prec, args.steps, args.warmup, dev, flush, barrier, gpu_index, native=native)
    pb = m["pb"]
    ms_max = max_over_ranks(m["ms"], world, dev)
    value = replica_value(args.steps, ms_max, world)

    pk, pk_src = peaks()
    fp64_peak = fsib.measure_peak(0)  # GFLOP/s
    fp32_peak = fsib.measure_peak(1)
    top = max(m["sites"], key=lambda s: s["total_ms"])
    roof = roofline_of(top, arith, pk, pk_src, fp64_peak, fp32_peak, prob.name)
    roof["share"] = top["total_ms"] / sum(s["total_ms"] for s in m["sites"])

    e2e = None if args.no_e2e else e2e_of(torch, pb, prob, args.steps, world)

    detail = {"headline": {"launch_shapes": m["launch_shapes"], "breakdown": breakdown_of(m["sites"], m["nprof"]),
                           "roofline": roof, "fp64_fma_peak_tflops": fp64_peak / 1e3,
                           "fp32_fma_peak_tflops": fp32_peak / 1e3}}

    # error against the oracle and the oracle's own time (the CPU baseline), from one oracle run
    cpu = err = native_err = None
    nat = nat_m = None
    do_native = prec == "fp64" and not native and not args.no_native and prob.d == 3
    if do_native:
        nat, nat_m = native_block(fsib, torch, prob, dev, flush, max(3, min(args.steps, 20)), max(3, args.warmup),
                                  pk, pk_src, fp64_peak, fp32_peak)
        nat["value"] *= world
    if rank == 0 and world == 1 and not args.no_cpu_baseline and prec == "fp64":
        k = 2 if prob.d == 3 else 20
        t, Xo, uo = oracle_steps(prob, k)
        cpu = {"value": k / t, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{k} full oracle steps of the same workload from its initial state "
                         "(direct non-uniform sums, numpy BLAS/FFT)"}
        Xg, ug = gpu_steps_from_start(torch, pb, prob, k, dev)
        err = dict(error_vs_oracle(prob, Xo, uo, Xg, ug), steps=k)
        if nat_m is not None:
            Xn, un = gpu_steps_from_start(torch, nat_m["pb"], prob, k, dev)
            native_err = dict(error_vs_oracle(prob, Xo, uo, Xn, un), steps=k)
    if nat is not None:
        nat["error_vs_oracle"] = native_err
        detail["native_fp64"] = {"launch_shapes": nat_m["launch_shapes"],
                                 "breakdown": breakdown_of(nat_m["sites"], nat_m["nprof"], 8)}
        nat_m["pb"].close()

    mixed = batched = None
    if not args.no_mixed and prec == "fp64" and prob.d == 3:
        mixed, detail["mixed"] = mixed_block(fsib, torch, dev, flush, pk, pk_src, fp64_peak, fp32_peak,
                                             steps=max(3, min(args.steps, 50)), warmup=max(3, args.warmup))
        mixed["value"] *= world
        mixed["nufft_pts_per_s"] = {k: v * world for k, v in mixed["nufft_pts_per_s"].items()}
    if not args.no_batched and prec == "fp64" and prob.d == 3:
        batched, detail["batched"] = batched_block(fsib, torch, dev, flush, steps=max(3, min(args.steps, 20)),
                                                   warmup=max(3, args.warmup), pk=pk, size=args.batch_size)
        for k in ("value", "boundary_points_per_s"):
            batched[k] *= world
    if args.adjoint:
        detail["adjoint"] = adjoint_block(fsib, torch, dev)
    if args.sweep:
        detail["nufft_sweep"] = nufft_sweep(fsib, torch, dev, flush)

    if rank == 0:
        arith_txt = {"df64": "double-float transforms (pairs of floats, ~48-bit significand), FP64 positions/forces",
                     "f64": "FP64 transforms, FP64 positions/forces",
                     "f32": "FP32 transforms, FP64 positions/forces"}[arith]
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": arith, "data": "synthetic",
                "config": {"workload": prob.name, "d": prob.d, "N": prob.N, "M": prob.M, **m["info"],
                           "tol": prob.tol, "arithmetic": arith_txt,
                           "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas{world}"},
                "nufft_pts_per_s": {"type1": world * m["pts1"], "type2": world * m["pts2"]},
                "roofline": {k: roof.get(k) for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                                                      "avg_launch_ms", "share", "hbm_frac", "peak_source", "limiter")},
                "step_roofline": step_roofline(prob, prec, m["info"]["nf"], m["info"]["Nt"], ms_max / args.steps, pk),
                "error_vs_oracle": err, "cpu_baseline": cpu, "e2e": e2e, "clocks": m["clocks"],
                "gpu_launches": m["launches"] * args.steps, "launches_per_step": m["launches"],
                "native_fp64": nat, "mixed": mixed, "batched": batched}
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump(dict(detail, line=line), f, indent=1)
        print(json.dumps(line, separators=(",", ":")), flush=True)
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
