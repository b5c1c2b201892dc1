"""Benchmark: point-steps/s of the periodic TDSE solver on one GB300.

Workload (one bench "step" = one whole solve): the 2D periodic wells problem
on [-pi,pi]^2, 512x512 grid, T = 2, dt = 1e-3 (2000 steps: 7 Richardson
start-up steps + 1993 8th-order Adams steps), pulse A(t) = 2 sin^2(pi t/2)
sin(10 t) (1,0), replicated as a batch of independent seeded instances (64 in
mixed precision, 4 in FP64 by default) so that the per-step working set
(~27 MB per instance in mixed precision) exceeds the 129 MB L2 and the pass
kernels' grids span many waves.  Point-steps = instances x 512^2 x 2000.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                    [--batch B] [--impl reference]
                    [--workload periodic2d|free2d|batch1d|serve]

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.

`--workload batch1d` measures 512 uneven 1D periodic instances (N drawn from
256..16384, T = 1, dt = 1e-3, 1000 steps) stepped as one autotuned persistent
launch per step replayed from a CUDA graph, mixed precision.

`--workload serve` replays a seeded Poisson request stream (200 req/s for
1 s; 1D periodic N 2^10..2^14, 2D periodic 2^7..2^10 per side, 2D free space
2^6..2^8 per side, one third each; T ~ U[0.05, 0.2], dt log-uniform on
[2e-4, 2e-3]) through the request loop (admission by a 64 GB HBM budget,
solves overlapped on their own streams) and reports time-to-solution p50/p99
and aggregate point-steps/s.

`--workload periodic3d` measures the 3D periodic wells workload (128^3,
dt = 1e-3, 500 steps, a batch of 16 mixed / 2 FP64 instances).

`--workload free2d` measures the free-space scheme instead: bump-windowed
Gaussians on [-1,1]^2, 256x256 grid, nu = 2048 per dimension (2058 contour
modes per dimension), p = 8, q = 10, n_r = 1, H for eps = 1e-10, T = 1,
dt = 5e-4 (2000 steps), FP64.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

M = 512
DT = 1e-3
NSTEPS = 2000
ORDER = 8
STARTUP = ORDER - 1
METRIC = "point-steps/s (2D periodic 512^2, 8th-order, T=2)"
# Algorithmic HBM bytes per point-step of the step operator: read u^ (16) and
# 7 history slots, write u^ (16) and one slot; V read once (real).
ALGO_BYTES = {"fp64": 16 + 7 * 16 + 8 + 16 + 16, "mixed": 16 + 7 * 8 + 4 + 16 + 8}
# FP64 FMA throughput of this GB300 pool (register-resident FMA chains, all
# SMs), TFLOP/s: the peak of the FP64-bound free-space step.
FP64_PEAK_TFLOPS = 1.25          # nominal FP64 rate, context only (the lines divide by fp64_peak())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default=None, choices=["mixed", "fp64"],
                    help="default: mixed (periodic2d, batch1d, serve), fp64 (free2d)")
    ap.add_argument("--batch", type=int, default=0,
                    help="instances per GPU (default: 64 periodic mixed, 4 periodic fp64, 1 free space; "
                         "example1: initial states per speed, 2048)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--full-config", action="store_true",
                    help="serve: the request stream at its stated sizes (1D N 2^10..2^16, 2D periodic 2^7..2^10, "
                         "free space 2^6..2^9 with nu = 4n, T ~ U[0.5, 2], 10 s of arrivals)")
    ap.add_argument("--no-fp64-variant", action="store_true",
                    help="skip the complex128 timing of the same workload in the default (mixed) line")
    ap.add_argument("--workload", default="periodic2d",
                    choices=["periodic2d", "free2d", "batch1d", "serve", "example1", "periodic3d", "free_ctype",
                             "free3d"])
    ap.add_argument("--passes-from", type=int, default=16384,
                    help="batch1d: members of n >= this use the four-step layout (0: one CTA per instance for "
                         "all; whole solve 146.4 ms with 0, 140.9 with 8192, 140.6 with 16384)")
    ap.add_argument("--profile-adams", type=int, default=0,
                    help="profiling run: start-up + this many Adams steps of the batch, then exit")
    return ap.parse_args()


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The largest x over the ranks (all_reduce MAX; x itself on one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, t_max: float) -> float:
    """Throughput of the whole job: every rank processed units_per_rank in at
    most t_max seconds (weak scaling)."""
    return ws * units_per_rank / t_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def instances(rank: int, batch: int):
    return [synth.periodic_2d_wells(seed=1000 * rank + 2 + i, M=M, dt=DT, nsteps=NSTEPS) for i in range(batch)]


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (clock, max clock, reasons)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------- GPU arm
def launches_per_solve(dim: int, mixed: bool, path: str = "passes") -> int:
    """Kernel launches of one tdse_step(NSTEPS) call (init, start-up, Adams);
    the cluster path runs all Adams steps of the call in one launch."""
    L = ORDER // 2
    sub = sum(2 ** c for c in range(L))      # trapezoid sub-steps per start-up step
    per_op = 1 if dim == 1 else 3            # kernels per unfused application of the step operator
    startup = STARTUP * (L + sub * per_op + 1 + per_op)   # copy_slot per chain, sub-steps, combine, refresh
    init = 1 if dim == 1 else 2
    k = NSTEPS - STARTUP
    adams = k if dim == 1 else 2 * k + 1     # 2D: col_begin, (row_mid, col_fused) x (k-1), row_mid, col_end
    if dim == 2 and path == "cluster":
        adams = 1
    return init + startup + (1 if mixed else 0) + adams


# DRAM bytes per point-step of the 2D step operator (k_row_mid + k_col_fused_ip)
# from the ncu capture of the 512^2 mixed workload at batch 8 (summarised under
# profiles/); traffic scales with the number of instances.  None = not captured
# for the current kernels.
TRAFFIC_BYTES_PER_POINT_STEP = {("mixed", "passes"): 72.143 + 16.105}
TRAFFIC_NOTE = {("mixed", "passes"): "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_col_fused_ip<512> + "
                "k_row_mid<float2,512>, batch 8 in 4 groups (2 instances per launch), scaled by points: reads "
                "72.1 + 16.1 B per point-step (re-taken on the current kernels); the state, history and intermediate writes (40 B) stayed in L2 "
                "within that capture (profiles/step2d_512x512_mixed_fused.md)"}


def run_gpu(args, ws, rank, local):
    import torch
    from paper_2001_06113_gb300 import Problem

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    insts = instances(rank, args.batch)
    B = len(insts)
    prob = Problem((M, M), DT, NSTEPS, order=ORDER, batch=B, precision=args.precision, stream=stream)
    pinned_V = [torch.from_numpy(it.V0).pin_memory() for it in insts]
    pinned_u = torch.from_numpy(np.stack([it.u0 for it in insts])).pin_memory()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def load_inputs():
        for b, it in enumerate(insts):
            prob.set_potential(pinned_V[b], None, instance=b)
            p = it.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial_batch(pinned_u)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    load_inputs()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            prob.set_initial_batch(pinned_u)
            prob.step(NSTEPS)
        stream.synchronize()

    # ---- device-timed region: K whole solves, inputs resident, L2 flushed between solves
    times = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                prob.set_initial_batch(pinned_u)   # resets the run (H2D outside the events)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                prob.step(NSTEPS)
                e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        barrier()
    t_solve = float(np.mean(times))
    t_solve = max_over_ranks(t_solve, ws, dev)
    points = M * M
    value = ws * B * points * NSTEPS / t_solve

    # ---- step-operator roofline: events around groups of consecutive Adams steps
    #      (2D: per step one row pass + one fused column pass)
    GROUP, NGROUPS = 50, 8
    with torch.cuda.stream(stream):
        prob.set_initial_batch(pinned_u)
        prob.step(STARTUP + 8)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(NGROUPS + 1)]
        evs[0].record(stream)
        for i in range(NGROUPS):
            prob.step(GROUP)
            evs[i + 1].record(stream)
    stream.synchronize()
    dts = np.array([evs[i].elapsed_time(evs[i + 1]) / 1e3 / GROUP for i in range(NGROUPS)])
    t_step = float(np.mean(dts))
    algo = ALGO_BYTES[args.precision] * B * points
    peak, peak_src = hbm_peak()
    achieved = algo / t_step / 1e9
    shape = prob.describe_steps()
    tb = TRAFFIC_BYTES_PER_POINT_STEP.get((args.precision, shape["path"]))
    traffic = None if tb is None else round(tb * B * points)
    kname = {"cluster": "k_step2d_cluster (one 16-CTA cluster per instance, a run of steps per launch)",
             "passes": "k_row_mid + k_col_fused_ip" if args.precision == "mixed" else "k_row_mid + k_col_end (FP64)"}
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "traffic_unit": "bytes per step (all instances)",
                "traffic_note": TRAFFIC_NOTE.get((args.precision, shape["path"])),
                "peak_source": peak_src,
                "kernel": f"2D Adams step operator: {kname[shape['path']]}, timed over groups of {GROUP} steps",
                "launch_shape": shape,
                "algorithmic_bytes_per_point_step": ALGO_BYTES[args.precision],
                "step_ms_p50": round(float(np.percentile(dts, 50)) * 1e3, 4),
                "step_ms_p99": round(float(np.percentile(dts, 99)) * 1e3, 4)}

    # ---- accuracy of this configuration on a sample instance: against the
    #      stored FP64 oracle solution (instance 0) and against the FP64 GPU path
    stated_err = None
    norm_drift = None
    oracle_err = None
    if rank == 0 and args.precision == "fp64":
        with torch.cuda.stream(stream):
            prob.set_initial_batch(pinned_u)
            prob.step(NSTEPS)
        oracle_err = golden_error(insts[0], prob.read_u(0), NSTEPS)
    if args.precision == "mixed" and rank == 0:
        ref = Problem((M, M), DT, NSTEPS, order=ORDER, batch=1, precision="fp64", stream=stream)
        it = insts[0]
        ref.set_potential(it.V0)
        p = it.pulse
        ref.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
        ref.set_initial(it.u0)
        with torch.cuda.stream(stream):
            ref.step(NSTEPS)
            prob.set_initial_batch(pinned_u)
            prob.step(NSTEPS)
        u_ref = ref.read_u(0)
        u_mix = prob.read_u(0)
        stated_err = float(np.sqrt(np.sum(np.abs(u_mix - u_ref) ** 2) / np.sum(np.abs(u_ref) ** 2)))
        norm_drift = float(np.sqrt(np.sum(np.abs(u_mix) ** 2) / np.sum(np.abs(it.u0) ** 2)) - 1.0)
        oracle_err = {"mixed": golden_error(it, u_mix, NSTEPS), "fp64_gpu": golden_error(it, u_ref, NSTEPS)}
        ref.close()

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        out = torch.empty((B, M, M), dtype=torch.complex128).pin_memory()
        e2e_times = []
        with torch.cuda.stream(stream):
            for _ in range(max(1, min(args.steps, 3))):
                flush.zero_()
                stream.synchronize()
                barrier()
                t0 = time.perf_counter()
                load_inputs()
                prob.step(NSTEPS)
                prob.read_u(-1, out=out)
                e2e_times.append(time.perf_counter() - t0)
        te = float(np.mean(e2e_times))
        te = max_over_ranks(te, ws, dev)
        h2d = B * (points * 8 + points * 16 + 2 * (8 * NSTEPS + 1) * 8)
        e2e = {"value": ws * B * points * NSTEPS / te, "unit": "point-steps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": B * points * 16}

    prob.close()
    fp64 = None
    if args.precision == "mixed" and rank == 0 and not args.no_fp64_variant:
        fp64 = fp64_variant(args, insts, stream, dev, value, oracle_err)
    return dict(value=value, t_solve=t_solve, roofline=roofline, e2e=e2e, clocks=clk.summary(),
                stated_err=stated_err, norm_drift=norm_drift, B=B, oracle_err=oracle_err, fp64=fp64)


def fp64_variant(args, insts, stream, dev, mixed_value, oracle_err):
    """The paper's precision (complex128 throughout) on the same workload: a
    batch of 4 instances and one instance alone (the plain one-solve-at-a-time
    FP64 GPU path), whole-solve times, and the Adams step against the FP64
    rate of this GPU (the FP64 step is bound by FP64 arithmetic, not HBM)."""
    import torch
    from paper_2001_06113_gb300 import Problem
    out = {}
    peak, peak_note = fp64_peak(dev)
    for B in (4, 1):
        its = insts[:B]
        prob = Problem((M, M), DT, NSTEPS, order=ORDER, batch=B, precision="fp64", stream=stream)
        for b, it in enumerate(its):
            prob.set_potential(it.V0, None, instance=b)
            p = it.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        u0 = torch.from_numpy(np.stack([it.u0 for it in its])).pin_memory()
        times = []
        with torch.cuda.stream(stream):
            for rep in range(3):
                prob.set_initial_batch(u0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                prob.step(NSTEPS)
                e1.record(stream)
                stream.synchronize()
                if rep:
                    times.append(e0.elapsed_time(e1) / 1e3)
        t = float(np.mean(times))
        entry = {"value": B * M * M * NSTEPS / t, "unit": "point-steps/s", "ms_per_solve": t * 1e3, "batch": B}
        if B == 4:
            GROUP, NGROUPS = 50, 4
            with torch.cuda.stream(stream):
                prob.set_initial_batch(u0)
                prob.step(STARTUP + 8)
                evs = [torch.cuda.Event(enable_timing=True) for _ in range(NGROUPS + 1)]
                evs[0].record(stream)
                for i in range(NGROUPS):
                    prob.step(GROUP)
                    evs[i + 1].record(stream)
            stream.synchronize()
            t_step = float(np.mean([evs[i].elapsed_time(evs[i + 1]) / 1e3 / GROUP for i in range(NGROUPS)]))
            ach = FP64_FLOPS_PER_POINT_STEP * B * M * M / t_step / 1e12
            entry["roofline"] = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 4),
                                 "unit": "TFLOP/s (FP64)", "frac": round(ach / peak, 4), "traffic": None,
                                 "peak_source": peak_note,
                                 "kernel": "k_row_mid<double2,512> + k_col_end<double2,double2,512,1> (FP64 Adams step), "
                                           f"timed over groups of {GROUP} steps",
                                 "algorithmic_flops_per_point_step": FP64_FLOPS_PER_POINT_STEP,
                                 "step_ms": round(t_step * 1e3, 4)}
            entry["rel_l2_vs_oracle"] = oracle_err.get("fp64_gpu") if oracle_err else None
        prob.close()
        out["batch4" if B == 4 else "one_at_a_time"] = entry
    out["mixed_over_fp64_one_at_a_time"] = mixed_value / out["one_at_a_time"]["value"]
    out["mixed_rel_l2_vs_oracle"] = oracle_err.get("mixed") if oracle_err else None
    return out


# ------------------------------------------------------------ free-space arm
FS_M, FS_NU, FS_DT, FS_NSTEPS, FS_Q, FS_NR = 256, 2048, 5e-4, 2000, 10, 1
# target precision eps of Remark Hchoice: FP64 sums (eps_m = 2^-52) and the
# FP32-transform variant (eps_m = 2^-23)
FS_EPS = {"fp64": 1e-10, "mixed": 1e-4}
FS_METRICS = {"fp64": "point-steps/s (2D free space 256^2, nu=2048, 8th-order, T=1, eps=1e-10)",
              "mixed": "point-steps/s (2D free space 256^2, nu=2048, 8th-order, T=1, FP32 transforms, eps=1e-4)"}
# DRAM bytes of one fused k_fs_row launch (end + begin) of one 256^2 instance,
# from the ncu capture summarised in profiles/step2d_free_256x256_fp64.md.
# FP32-transform variant: profiles/step2d_free_256x256_mixed.md (4 CTAs per SM).
FS_ROW_TRAFFIC = {"fp64": 484.806912e6 + 123.36256e6, "mixed": 277.87e6 + 122.29e6}
# FP32 FMA rate: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def free_instances(rank: int, batch: int):
    return [synth.free_bump_gaussians((FS_M, FS_M), seed=1000 * rank + 3 + i, dt=FS_DT, nsteps=FS_NSTEPS,
                                      T_pulse=1.0) for i in range(batch)]


def free_H(insts, precision: str = "fp64") -> float:
    """Remark Hchoice for the batch: ||V||_2 on the grid, max |phi| from the
    sampled pulse (cumulative trapezoid on 20001 points), eps of FS_EPS and
    the machine epsilon of the precision the contour sums run in."""
    from paper_2001_06113_gb300 import free_choose_H
    vnorm = max(math.sqrt(float(np.sum(it.V0 ** 2))) * 2.0 / FS_M for it in insts)
    phimax = 0.0
    t = np.linspace(0.0, FS_NSTEPS * FS_DT, 20001)
    for it in insts:
        A = it.pulse.A(t)
        phi = np.concatenate([np.zeros((1, A.shape[1])), np.cumsum(0.5 * (A[1:] + A[:-1]) * (t[1] - t[0]), axis=0)])
        phimax = max(phimax, float(np.max(np.abs(phi))))
    return free_choose_H(FS_EPS[precision], vnorm, phimax, 2, precision=precision)


def free_mode_count() -> int:
    kappa = 7
    ne = FS_NU // 2 - 2 * kappa + 1
    return 2 * ne + 2 * 8 + FS_Q * max(1, 2 * FS_NR)


def free_flops_per_step() -> float:
    """Real FP64 flops of one 2D free-space Adams step, per instance (complex
    mul 6, complex add 2, length-n FFT 5 n log2 n): the row pass over N0 mode
    rows (forward along axis 1, update, Horner history of 7 terms with
    separable phases, inverse along axis 1) plus the column pass over M1 grid
    columns (inverse along axis 0, implicit solve, V u, forward along axis 0)."""
    M, nu, N = FS_M, FS_NU, free_mode_count()
    R = nu // M
    ne = FS_NU // 2 - 13
    nd = N - 2 * ne
    fft = 2 * R * 5 * M * math.log2(M)
    fwd = 2 * nu * 6 + fft + 2 * ne * 6 + nd * M * 8
    inv = 2 * ne * 6 + fft + 2 * nu * 8 + nd * M * 8
    horner = 7 * 2 + 6 * (6 + 6 + 2) + 6 + 6 + 4
    row = fwd + inv + N * (4 + horner)
    col = inv + fwd + M * 14
    return N * row + M * col


def hbm_peak():
    """(GB/s, "measured" | "fallback"): the machine's measured copy bandwidth."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    return peaks.get("hbm_gbs", 6800.0), ("measured" if "hbm_gbs" in peaks else "fallback")


# FP64 flops of one point-step of the 2D FP64 periodic step (512^2), counted
# from the kernels' arithmetic: four length-512 transforms per point (one per
# axis pass, 5 n log2 n flops each = 45 per point each), the Horner history
# (6 lag phases p_j = q[m0] q[n0+m1] and p_j S: 12 flops each; 7 terms mu_j R_j:
# 4 each; X = u^ - i h S: 4; W = p_0 X with its phase: 12), the implicit solve
# and V product (21), the update (4) and the two 1/n scalings (4).
FP64_FLOPS_PER_POINT_STEP = 4 * 45 + (6 * 12 + 7 * 4 + 4 + 12) + 21 + 4 + 4


def fp64_peak(dev) -> tuple:
    """(TFLOP/s, note): FP64 throughput of this GPU measured here, as the best of
    3 cuBLAS float64 GEMMs of 4096^3 (2 n^3 flops) timed with CUDA events."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    del a, b
    return 2.0 * n ** 3 / best / 1e12, "measured in this run: cuBLAS float64 GEMM 4096^3, best of 3"


GOLDEN_512 = os.path.join(ROOT, "tests", "golden", "periodic_2d_wells_512.npz")


def golden_error(inst, u: np.ndarray, step: int):
    """rel-L2 of u against the stored FP64 oracle solution of the same seeded
    instance at `step` (every 4th grid point; file written by
    tests/golden/make_periodic_goldens.py), or None if not stored."""
    try:
        g = np.load(GOLDEN_512)
    except Exception:
        return None
    p = inst.pulse
    st = int(g["stride"])
    if (str(g["key"]) != inst.name or f"u_{step}" not in g
            or not np.allclose(g["params"], [inst.dt, inst.nsteps, p.A0, p.omega, p.T_pulse, *p.direction])
            or np.max(np.abs(inst.u0[::st, ::st] - g["u0_sample"])) > 1e-13 * np.max(np.abs(g["u0_sample"]))):
        return None
    ref = g[f"u_{step}"]
    sub = u[::st, ::st]
    return float(np.sqrt(np.sum(np.abs(sub - ref) ** 2) / np.sum(np.abs(ref) ** 2)))


def free_algo_bytes(precision: str) -> float:
    """Algorithmic DRAM bytes of one 2D free-space Adams step, per instance:
    per mode the state read and W written (FP64, 32 B), nhist - 1 = 6 ring
    lags read and the new (Vu)^ written (ring element e = 16 B in FP64, 8 B
    FP32); per intermediate value Z (N0 x M1) one write and one read in each
    pass (4 e); per grid point V read (8 B) and u written (16 B)."""
    N, M = free_mode_count(), FS_M
    e = 16 if precision == "fp64" else 8
    return N * N * (32 + 7 * e) + 4 * N * M * e + M * M * 24


def run_free(args, ws, rank, local):
    import torch
    from paper_2001_06113_gb300 import Problem

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    insts = free_instances(rank, args.batch)
    B = len(insts)
    prec = args.precision
    H = free_H(insts, prec)
    prob = Problem((FS_M, FS_M), FS_DT, FS_NSTEPS, order=ORDER, batch=B, precision=prec, stream=stream, bc="free",
                   nu=(FS_NU, FS_NU), H=H, gauss_q=FS_Q, n_r=FS_NR)
    pinned_V = [torch.from_numpy(it.V0).pin_memory() for it in insts]
    pinned_u = torch.from_numpy(np.stack([it.u0 for it in insts])).pin_memory()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def load_inputs():
        for b, it in enumerate(insts):
            prob.set_potential(pinned_V[b], None, instance=b)
            p = it.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial_batch(pinned_u)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def reset():
        prob.set_initial_batch(pinned_u)

    load_inputs()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            reset()
            prob.step(FS_NSTEPS)
        stream.synchronize()
    times = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                reset()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                prob.step(FS_NSTEPS)
                e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        barrier()
    t_solve = float(np.mean(times))
    t_solve = max_over_ranks(t_solve, ws, dev)
    points = FS_M * FS_M
    value = ws * B * points * FS_NSTEPS / t_solve

    GROUP, NGROUPS = 10, 20
    with torch.cuda.stream(stream):
        reset()
        prob.step(STARTUP + 8)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(NGROUPS + 1)]
        evs[0].record(stream)
        for i in range(NGROUPS):
            prob.step(GROUP)
            evs[i + 1].record(stream)
    stream.synchronize()
    dts = np.array([evs[i].elapsed_time(evs[i + 1]) / 1e3 / GROUP for i in range(NGROUPS)])
    t_step = float(np.mean(dts))
    flops = free_flops_per_step() * B
    achieved = flops / t_step / 1e12
    traffic = FS_ROW_TRAFFIC[prec] * B if FS_ROW_TRAFFIC[prec] else None
    timing = {"kernel": "2D free-space Adams step (k_fs_row end+begin + k_fs_phys), timed over groups of 10 steps",
              "algorithmic_flops_per_step": flops,
              "step_ms_p50": round(float(np.percentile(dts, 50)) * 1e3, 4),
              "step_ms_p99": round(float(np.percentile(dts, 99)) * 1e3, 4)}
    if prec == "fp64":
        peak64, src64 = fp64_peak(dev)
        roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak64, 4), "unit": "TFLOP/s",
                    "frac": round(achieved / peak64, 4), "traffic": traffic,
                    "traffic_unit": "DRAM bytes per fused k_fs_row launch (ncu), per instance x instances",
                    "peak_source": src64, "nominal_fp64_tflops": FP64_PEAK_TFLOPS, **timing}
    else:
        # FP32 transforms: both ceilings, the nearer one reported as the bound
        algo = free_algo_bytes(prec) * B
        gbs = algo / t_step / 1e9
        alu = {"achieved": round(achieved, 4), "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s",
               "frac": round(achieved / FP32_PEAK_TFLOPS, 4),
               "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"}
        hpk, hsrc = hbm_peak()
        hbm = {"achieved": round(gbs, 1), "peak": hpk, "unit": "GB/s", "frac": round(gbs / hpk, 4),
               "algorithmic_bytes_per_step": algo, "peak_source": hsrc}
        top, other = ("hbm", "alu") if hbm["frac"] >= alu["frac"] else ("alu", "hbm")
        pick = {"hbm": hbm, "alu": alu}
        roofline = {"bound": top, **pick[top], "traffic": traffic,
                    "traffic_unit": "DRAM bytes per fused k_fs_row launch (ncu), per instance x instances",
                    "other_ceiling": {"bound": other, **pick[other]}, **timing}
    e2e = None
    if not args.no_e2e:
        out = torch.empty((B, FS_M, FS_M), dtype=torch.complex128).pin_memory()
        e2e_times = []
        with torch.cuda.stream(stream):
            for _ in range(max(1, min(args.steps, 2))):
                flush.zero_()
                stream.synchronize()
                barrier()
                t0 = time.perf_counter()
                load_inputs()
                prob.step(FS_NSTEPS)
                prob.read_u(-1, out=out)
                e2e_times.append(time.perf_counter() - t0)
        te = float(np.mean(e2e_times))
        te = max_over_ranks(te, ws, dev)
        h2d = B * (points * 8 + points * 16)
        e2e = {"value": ws * B * points * FS_NSTEPS / te, "unit": "point-steps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": B * points * 16}
    stated_err = None
    if prec == "mixed" and rank == 0:
        # the FP32-transform variant against the FP64 path on the same contour
        NCHK = 40
        ref = Problem((FS_M, FS_M), FS_DT, FS_NSTEPS, order=ORDER, batch=1, precision="fp64", stream=stream,
                      bc="free", nu=(FS_NU, FS_NU), H=H, gauss_q=FS_Q, n_r=FS_NR)
        it = insts[0]
        ref.set_potential(it.V0, None)
        ref.set_pulse(it.pulse.A0, it.pulse.omega, it.pulse.T_pulse, it.pulse.direction)
        ref.set_initial(it.u0)
        with torch.cuda.stream(stream):
            reset()
            prob.step(NCHK)
            ref.step(NCHK)
        stream.synchronize()
        um, ud = prob.read_u(0), ref.read_u(0)
        stated_err = {"rel_l2_vs_fp64_same_contour": float(np.linalg.norm(um - ud) / np.linalg.norm(ud)),
                      "after_steps": NCHK}
        ref.close()
    prob.close()
    return dict(value=value, t_solve=t_solve, roofline=roofline, e2e=e2e, clocks=clk.summary(), stated_err=stated_err,
                B=B, H=H)


def free_launches_per_solve() -> int:
    L = ORDER // 2
    sub = sum(2 ** c for c in range(L))
    startup = STARTUP * (L + sub * 3 + 2 + 2)   # copy_slot per chain, sub-steps, 2 combines, refresh (2)
    init = 4
    k = FS_NSTEPS - STARTUP
    return init + startup + 2 * k + 1


def free_oracle_sample(nadams: int = 2, seed: int = 3):
    """The free-space oracle (as it stands) on `nadams` Adams steps of one
    256^2 instance (direct transform sums); returns point-steps/s."""
    from oracle import fields, gamma
    from oracle.freespace import FreeSpaceOracle
    it = synth.free_bump_gaussians((FS_M, FS_M), seed=seed, dt=FS_DT, nsteps=FS_NSTEPS, T_pulse=1.0)
    H = 2.75
    rules = [gamma.GammaRule.for_nu(FS_M, FS_NU, H, q=FS_Q, n_r=FS_NR) for _ in range(2)]
    orc = FreeSpaceOracle(rules, FS_DT, it.V0, it.vfac, fields.phi_callable(it.pulse, 2))
    uh = orc.fwd(it.u0)
    h0 = orc.fwd(orc.V(0.0) * it.u0)
    n0 = 100
    hist = {n0 - j: h0 for j in range(1, ORDER)}
    t0 = time.perf_counter()
    for k in range(nadams):
        n = n0 + k
        uh, u, hist[n] = orc.adams_step(uh, n * FS_DT, hist, n)
        hist.pop(n - ORDER, None)
    el = time.perf_counter() - t0
    return FS_M * FS_M * nadams / el, el


def profile_run(args):
    """Small fixed launch sequence for ncu: init, start-up, then K Adams steps."""
    import torch
    from paper_2001_06113_gb300 import Problem
    insts = instances(0, args.batch)
    prob = Problem((M, M), DT, NSTEPS, order=ORDER, batch=len(insts), precision=args.precision)
    for b, it in enumerate(insts):
        prob.set_potential(it.V0, None, instance=b)
        p = it.pulse
        prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial(it.u0, instance=b)
    prob.step(STARTUP + args.profile_adams)
    torch.cuda.synchronize()
    prob.check_finite()
    print(json.dumps({"profile_adams": args.profile_adams, "batch": len(insts), "precision": args.precision,
                      "launches_before_adams": launches_per_solve(2, args.precision == "mixed")
                      - (2 * (NSTEPS - STARTUP) + 1)}))
    prob.close()
    return 0


# ---------------------------------------------------------------- CPU oracle arm
def oracle_sample(nadams: int = 6, seed: int = 2):
    """Time the CPU oracle (as it stands) on a bounded sample of the workload:
    `nadams` 8th-order Adams steps of one 512^2 instance, history seeded with
    (Vu)^ of u0 (same cost per step as a real run).  Returns point-steps/s."""
    from oracle.periodic import oracle_for
    it = synth.periodic_2d_wells(seed=seed, M=M, dt=DT, nsteps=NSTEPS)
    orc = oracle_for(it)
    u = it.u0
    h0 = orc.fwd(orc.V(0.0) * u)
    n0 = 100
    hist = {n0 - j: h0 for j in range(1, ORDER)}
    t0 = time.perf_counter()
    for k in range(nadams):
        n = n0 + k
        t = n * DT
        u = orc.adams_step(u, t, hist, n)
        hist[n] = orc.fwd(orc.V(t) * u)
        hist.pop(n - ORDER, None)
    el = time.perf_counter() - t0
    return M * M * nadams / el, el


def oracle_sample_one_core(nadams: int):
    """oracle_sample on one core: a child interpreter with one BLAS / OpenMP
    thread (the thread pools are fixed at import).  None if it fails."""
    import subprocess
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys; sys.argv = ['bench.py']; import bench; "
            f"v, el = bench.oracle_sample(nadams={int(nadams)}); print(v)")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=120)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (subprocess.SubprocessError, ValueError, IndexError, OSError):
        return None


def cpu_cores() -> int:
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        n = [d.get("num_threads") for d in info if d.get("internal_api") in ("openblas", "mkl", "blis")]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


def free_profile_run(args):
    """Small fixed launch sequence for ncu: init, start-up, then K Adams steps (free space)."""
    import torch
    from paper_2001_06113_gb300 import Problem
    insts = free_instances(0, args.batch)
    prob = Problem((FS_M, FS_M), FS_DT, FS_NSTEPS, order=ORDER, batch=len(insts), precision=args.precision,
                   bc="free", nu=(FS_NU, FS_NU), H=free_H(insts, args.precision), gauss_q=FS_Q, n_r=FS_NR)
    for b, it in enumerate(insts):
        prob.set_potential(it.V0, None, instance=b)
        p = it.pulse
        prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial(it.u0, instance=b)
    prob.step(STARTUP + args.profile_adams)
    torch.cuda.synchronize()
    prob.check_finite()
    print(json.dumps({"profile_adams": args.profile_adams, "batch": len(insts), "workload": "free2d",
                      "precision": args.precision,
                      "launches_before_adams": free_launches_per_solve() - (2 * (FS_NSTEPS - STARTUP) + 1)}))
    prob.close()
    return 0


def main_free(args, ws, rank, local):
    import torch
    if args.impl == "reference":
        if rank != 0:
            return 0
        for _ in range(args.warmup):
            free_oracle_sample(nadams=1)
        vals = [free_oracle_sample(nadams=1)[0] for _ in range(args.steps)]
        value = float(np.mean(vals))
        line = {"impl": "reference", "metric": FS_METRICS[args.precision], "value": value, "unit": "point-steps/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * FS_M * FS_M / value, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "2D free space 256x256, nu=2048, dt=5e-4, 8th-order Adams (CPU oracle sample)"},
                "cpu_baseline": {"value": value, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                                 "sample": "1 Adams step of one 256^2 free-space instance per bench step "
                                           "(direct transform sums)"},
                "e2e": {"value": value, "unit": "point-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    if args.profile_adams:
        return free_profile_run(args)
    if ws > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    res = run_free(args, ws, rank, local)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            v, el = free_oracle_sample(nadams=3)
            cpu = {"value": v, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"3 8th-order Adams steps of one 256^2 free-space instance ({el:.1f} s; direct "
                             "transform sums, numpy/OpenBLAS)"}
        prec = args.precision
        line = {
            "metric": FS_METRICS[prec], "value": res["value"], "unit": "point-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["t_solve"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128" if prec == "fp64" else "c64+c128", "data": "synthetic",
            "config": {"workload": f"2D free space 256x256, nu=2048 (N=2058 modes/dim), p=8, q=10, n_r=1, "
                                   f"H={res['H']:.4f} (eps={FS_EPS[prec]:g}), T=1, dt=5e-4 (2000 steps), "
                                   f"8th-order Adams, batch of {res['B']} per GPU, {prec}",
                       "grid": [FS_M, FS_M], "nu": FS_NU, "nsteps": FS_NSTEPS, "dt": FS_DT, "order": ORDER,
                       "batch_per_gpu": res["B"], "precision": prec,
                       "l2": "flushed (256 MB write) before each timed solve; per-step working set > L2",
                       "step": "one whole solve (7 Richardson start-up + 1993 Adams steps)",
                       "parallelism": f"replicas x{ws}"},
            "stated_err": res["stated_err"],
            "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"], "clocks": res["clocks"],
            "gpu_launches": free_launches_per_solve() * args.steps,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------------------ uneven 1D batch arm
B1_COUNT, B1_DT, B1_NSTEPS = 512, 1e-3, 1000
B1_METRIC = "point-steps/s (512 uneven 1D periodic instances, N in 256..16384, 8th-order, T=1, mixed)"
B1_ALGO_BYTES = 16 + 7 * 8 + 4 + 16 + 8      # mixed 1D step: state in/out, 7 ring reads, 1 write, V
# DRAM bytes of one k_periodic1d_multi launch over the 512 instances (ncu capture,
# default launch shape; profiles/batch1d_512_uneven_mixed.md).
B1_MULTI_TRAFFIC = 225.796096e6 + 51.56864e6


def batch1d_instances(rank: int):
    return [synth.periodic_1d_batch_member(i, seed=4 + 1000 * rank, dt=B1_DT, nsteps=B1_NSTEPS)
            for i in range(B1_COUNT)]


def run_batch1d(args, ws, rank, local):
    import torch
    from paper_2001_06113_gb300 import Batch, Problem
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    insts = batch1d_instances(rank)
    groups = {}
    for it in insts:
        groups.setdefault(it.shape[0], []).append(it)
    sizes = sorted(groups)
    pf = args.passes_from
    probs = [Problem((N,), B1_DT, B1_NSTEPS, batch=len(groups[N]), precision="mixed", stream=stream,
                     layout_1d="passes" if pf and N >= pf else "auto") for N in sizes]
    pinned = {N: [(torch.from_numpy(it.V0).pin_memory(), None) for it in groups[N]] for N in sizes}
    pinned_u = {N: torch.from_numpy(np.stack([it.u0 for it in groups[N]])).pin_memory() for N in sizes}

    def load_inputs():
        for N, pr in zip(sizes, probs):
            for b, it in enumerate(groups[N]):
                pr.set_potential(pinned[N][b][0], None, instance=b)
                p = it.pulse
                pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
            pr.set_initial_batch(pinned_u[N])

    def reset():
        for N, pr in zip(sizes, probs):
            pr.set_initial_batch(pinned_u[N])

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    load_inputs()
    batch = Batch(probs, stream=stream)
    default_shape = batch.describe()
    batch.tune(5)
    shape = batch.describe()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=torch.device("cuda", local))
    reset()
    for _ in range(args.warmup):
        reset()
        batch.step(B1_NSTEPS)
    stream.synchronize()
    points = sum(it.shape[0] for it in insts)
    times = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                reset()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                batch.step(B1_NSTEPS)
                e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        barrier()
    t_solve = float(np.mean(times))
    t_solve = max_over_ranks(t_solve, ws, "cuda")
    value = ws * points * B1_NSTEPS / t_solve
    # per-step latency of the fused launch: events around single Adams steps (direct launches)
    reset()
    stream.synchronize()
    dstream = torch.cuda.default_stream()
    batch.step(STARTUP + 8, stream=dstream)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(101)]
    with torch.cuda.stream(dstream):
        evs[0].record(dstream)
        for i in range(100):
            batch.step(1, stream=dstream)
            evs[i + 1].record(dstream)
    dstream.synchronize()
    dts = np.array([evs[i].elapsed_time(evs[i + 1]) / 1e3 for i in range(100)])
    t_step = float(np.mean(dts))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = B1_ALGO_BYTES * points / t_step / 1e9
    fused = shape.get("mode", "fused") == "fused"
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": B1_MULTI_TRAFFIC if fused else None,
                "traffic_unit": "DRAM bytes per k_periodic1d_multi launch (ncu, default launch shape)",
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "kernel": ("k_periodic1d_multi (one persistent launch per Adams step for all 512 instances)" if fused
                           else "k_periodic1d<float2,float2,N> per member size, on parallel streams (tuner's "
                                "choice over the fused launch)") + ", timed per step over 100 steps",
                "algorithmic_bytes_per_point_step": B1_ALGO_BYTES,
                "step_ms_p50": round(float(np.percentile(dts, 50)) * 1e3, 4),
                "step_ms_p99": round(float(np.percentile(dts, 99)) * 1e3, 4)}
    # accuracy and the plain path: one instance per size up to 8192 solved alone in FP64
    reset()
    batch.step(B1_NSTEPS)
    stream.synchronize()
    errs, f64_points, f64_time = {}, 0, 0.0
    for N, pr in zip(sizes, probs):
        if N > 8192:
            continue
        it = groups[N][0]
        ref = Problem((N,), B1_DT, B1_NSTEPS, precision="fp64")
        ref.set_potential(it.V0)
        p = it.pulse
        ref.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
        ref.set_initial(it.u0)
        ref.step(1)                                  # warm
        ref.set_initial(it.u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ref.step(B1_NSTEPS)
        torch.cuda.synchronize()
        f64_time += time.perf_counter() - t0
        f64_points += N * B1_NSTEPS
        u_ref = ref.read_u(0)
        u_mix = pr.read_u(0)
        errs[N] = float(np.sqrt(np.sum(np.abs(u_mix - u_ref) ** 2) / np.sum(np.abs(u_ref) ** 2)))
        ref.close()
    e2e = None
    if not args.no_e2e:
        out = {N: torch.empty((len(groups[N]), N), dtype=torch.complex128).pin_memory() for N in sizes}
        e2e_times = []
        for _ in range(max(1, min(args.steps, 3))):
            stream.synchronize()
            barrier()
            t0 = time.perf_counter()
            load_inputs()
            batch.step(B1_NSTEPS)
            for N, pr in zip(sizes, probs):
                pr.read_u(-1, out=out[N])
            e2e_times.append(time.perf_counter() - t0)
        te = float(np.mean(e2e_times))
        e2e = {"value": ws * points * B1_NSTEPS / te, "unit": "point-steps/s",
               "h2d_bytes_per_step": points * (8 + 16) + 2 * len(insts) * (8 * B1_NSTEPS + 1) * 8,
               "d2h_bytes_per_step": points * 16}
    batch.close()
    for pr in probs:
        pr.close()
    return dict(value=value, t_solve=t_solve, roofline=roofline, e2e=e2e, clocks=clk.summary(), points=points,
                sizes={int(N): len(groups[N]) for N in sizes}, shape=shape, default_shape=default_shape,
                errs=errs, f64_one_at_a_time=f64_points / f64_time if f64_time else None)


def batch1d_launches(shape_members: int) -> int:
    """Launches of one 1000-step batch solve: per member init + start-up
    (7 x (4 copies + 15 sub-steps + combine + refresh)) + change of frame,
    then one fused launch per Adams step."""
    per_member = 1 + STARTUP * (4 + 15 + 1 + 1) + 1
    return shape_members * per_member + (B1_NSTEPS - STARTUP)


def batch1d_oracle_sample(nadams: int = 20):
    from oracle.periodic import oracle_for
    it = synth.periodic_1d_batch_member(0, seed=4, dt=B1_DT, nsteps=B1_NSTEPS, sizes=(1024,))
    orc = oracle_for(it)
    u = it.u0
    h0 = orc.fwd(orc.V(0.0) * u)
    n0 = 100
    hist = {n0 - j: h0 for j in range(1, ORDER)}
    t0 = time.perf_counter()
    for k in range(nadams):
        n = n0 + k
        t = n * B1_DT
        u = orc.adams_step(u, t, hist, n)
        hist[n] = orc.fwd(orc.V(t) * u)
        hist.pop(n - ORDER, None)
    el = time.perf_counter() - t0
    return 1024 * nadams / el, el


def batch1d_profile_run(args):
    """ncu launch sequence: start-up + K fused Adams steps of the uneven batch
    (direct launches), then K Adams steps of every member on its own kernel."""
    import torch
    from paper_2001_06113_gb300 import Batch, Problem
    insts = batch1d_instances(0)
    groups = {}
    for it in insts:
        groups.setdefault(it.shape[0], []).append(it)
    sizes = sorted(groups)
    probs = []
    for N in sizes:
        pr = Problem((N,), B1_DT, B1_NSTEPS, batch=len(groups[N]), precision="mixed")
        for b, it in enumerate(groups[N]):
            pr.set_potential(it.V0, None, instance=b)
            p = it.pulse
            pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
            pr.set_initial(it.u0, instance=b)
        probs.append(pr)
    batch = Batch(probs)
    dstream = torch.cuda.default_stream()
    batch.step(STARTUP + args.profile_adams, stream=dstream)
    for pr in probs:
        pr.step(args.profile_adams)
    torch.cuda.synchronize()
    print(json.dumps({"profile_adams": args.profile_adams, "workload": "batch1d", "shape": batch.describe()}))
    return 0


def main_batch1d(args, ws, rank, local):
    import torch
    if args.impl == "reference":
        if rank != 0:
            return 0
        for _ in range(args.warmup):
            batch1d_oracle_sample(2)
        vals = [batch1d_oracle_sample(20)[0] for _ in range(args.steps)]
        value = float(np.mean(vals))
        print(json.dumps({"impl": "reference", "metric": B1_METRIC, "value": value, "unit": "point-steps/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * 1024 * 20 / value, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "uneven 1D batch (CPU oracle sample: 20 Adams steps, N=1024)"},
                          "cpu_baseline": {"value": value, "unit": "point-steps/s", "cores": cpu_cores(),
                                           "kind": "oracle", "sample": "20 Adams steps of one N=1024 instance"},
                          "e2e": {"value": value, "unit": "point-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    if args.profile_adams:
        return batch1d_profile_run(args)
    if ws > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    res = run_batch1d(args, ws, rank, local)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            v, el = batch1d_oracle_sample(60)
            cpu = {"value": v, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"60 8th-order Adams steps of one N=1024 instance ({el:.1f} s; direct DFT sums)"}
        line = {
            "metric": B1_METRIC, "value": res["value"], "unit": "point-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["t_solve"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
            "data": "synthetic",
            "config": {"workload": f"512 uneven 1D periodic instances per GPU (N histogram {res['sizes']}), "
                                   "T=1, dt=1e-3 (1000 steps), 8th-order Adams, mixed precision, one batch (tuned: "
                                   "one persistent launch per Adams step or the members' kernels on parallel streams), "
                                   "whole solve replayed from a CUDA graph",
                       "points_per_gpu": res["points"], "nsteps": B1_NSTEPS, "dt": B1_DT, "order": ORDER,
                       "launch_shape_tuned": res["shape"], "launch_shape_default": res["default_shape"],
                       "four_step_layout_from_n": args.passes_from or None,
                       "l2": "flushed (256 MB write) before each timed solve; per-step working set "
                             f"{res['points'] * 100 / 1e6:.0f} MB > L2",
                       "step": "one whole solve (init, 7 Richardson start-up steps, 993 Adams steps)",
                       "parallelism": f"replicas x{ws}"},
            "rel_l2_vs_fp64": res["errs"],
            "fp64_one_at_a_time_point_steps_per_s": res["f64_one_at_a_time"],
            "time_to_solution_s": {"p50": res["t_solve"], "p99": res["t_solve"],
                                   "note": "all instances of the batch finish together"},
            "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"], "clocks": res["clocks"],
            "gpu_launches": batch1d_launches(len(res["sizes"])) * args.steps,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------------------ Example 1 arm (moving periodic well)
EX_M, EX_NSTEPS, EX_T, EX_SPEEDS, EX_B = 512, 3200, 2.0 * math.pi / 15.0, (15.0, 30.0, 45.0), 2048
EX_METRIC = ("point-steps/s (Example 1 moving periodic Gaussian well, V0=300, beta=0.2: 3 speeds x 2048 initial "
             "states, M=512, 3200 steps to T=2pi/15, 8th-order, mixed)")
# per point-step: state in/out 32, 7 ring reads 56, 1 ring write 8; the V row
# (one shared table per speed) is read once per step for all instances
EX_ALGO_BYTES = 16 + 7 * 8 + 16 + 8
# DRAM bytes of one k_periodic1d<float2,float2,512> Adams-step launch over 2048
# instances (ncu, profiles/example1_moving_well_512_mixed.md); per step x 3 speeds
EX_LAUNCH_TRAFFIC = 77.75232e6 + 5.611776e6


def example1_oracle_sample(nadams: int = 400):
    """The periodic oracle (as it stands) on `nadams` Adams steps of one
    Example 1 instance (c = 30, M = 512), history seeded with (Vu)^ of u0."""
    from oracle import fields
    from oracle.periodic import PeriodicOracle
    it = synth.moving_well_1d(c=30.0, M=EX_M, nsteps=EX_NSTEPS, T=EX_T)
    orc = PeriodicOracle(it.shape, it.dt, it.Vt, None, fields.phi_callable(None, 1))
    u = it.u0
    h0 = orc.fwd(orc.V(0.0) * u)
    n0 = 100
    hist = {n0 - j: h0 for j in range(1, ORDER)}
    t0 = time.perf_counter()
    for k in range(nadams):
        n = n0 + k
        t = n * it.dt
        u = orc.adams_step(u, t, hist, n)
        hist[n] = orc.fwd(orc.V(t) * u)
        hist.pop(n - ORDER, None)
    el = time.perf_counter() - t0
    return EX_M * nadams / el, el


def run_example1(args, ws, rank, local):
    import torch
    from paper_2001_06113_gb300 import Batch, Problem
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    B = args.batch if args.batch > 0 else EX_B
    sweeps = [synth.example1_sweep(B, c, seed=11 + 1000 * rank, M=EX_M, nsteps=EX_NSTEPS, T=EX_T)
              for c in EX_SPEEDS]
    dt = sweeps[0][0].dt
    probs = [Problem((EX_M,), dt, EX_NSTEPS, batch=B, precision="mixed", stream=stream, potential="shared_table")
             for _ in EX_SPEEDS]
    times_v = probs[0].potential_times()
    tables = [torch.from_numpy(base.potential_table(times_v)).pin_memory() for base, _ in sweeps]
    u0s = [torch.from_numpy(u0).pin_memory() for _, u0 in sweeps]

    def reset():
        for pr, u0 in zip(probs, u0s):
            pr.set_initial_batch(u0)

    def load_inputs():
        for pr, tab in zip(probs, tables):
            pr.set_potential_table(tab)
        reset()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    load_inputs()
    batch = Batch(probs, stream=stream)
    batch.tune(5)
    shape = batch.describe()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=torch.device("cuda", local))
    for _ in range(args.warmup):
        reset()
        batch.step(EX_NSTEPS)
    stream.synchronize()
    points = len(probs) * B * EX_M
    times = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                reset()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                batch.step(EX_NSTEPS)
                e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        barrier()
    t_solve = max_over_ranks(float(np.mean(times)), ws, "cuda")
    value = ws * points * EX_NSTEPS / t_solve
    # per-step latency of the fused launch
    reset()
    stream.synchronize()
    dstream = torch.cuda.default_stream()
    batch.step(STARTUP + 8, stream=dstream)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(101)]
    with torch.cuda.stream(dstream):
        evs[0].record(dstream)
        for i in range(100):
            batch.step(1, stream=dstream)
            evs[i + 1].record(dstream)
    dstream.synchronize()
    dts = np.array([evs[i].elapsed_time(evs[i + 1]) / 1e3 for i in range(100)])
    t_step = float(np.mean(dts))
    peak, peak_src = hbm_peak()
    achieved = EX_ALGO_BYTES * points / t_step / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": EX_LAUNCH_TRAFFIC * len(probs) * B / 2048 if shape.get("mode") == "streams" else None,
                "traffic_unit": "DRAM bytes per Adams step (ncu launch of 2048 instances, scaled by instances)",
                "peak_source": peak_src,
                "kernel": ("k_periodic1d_multi (one persistent launch per Adams step for all instances of the three "
                           "speeds)" if shape.get("mode", "fused") == "fused" else
                           "k_periodic1d<float2,float2,512> per speed on parallel streams (tuner's choice over the "
                           "fused launch)") + ", timed per step over 100 steps",
                "algorithmic_bytes_per_point_step": EX_ALGO_BYTES,
                "step_ms_p50": round(float(np.percentile(dts, 50)) * 1e3, 4),
                "step_ms_p99": round(float(np.percentile(dts, 99)) * 1e3, 4)}
    # accuracy: the first initial state of each speed solved alone in FP64 (its own table), and
    # the FP64 time-discretisation error at c = 30 (3200 against 6400 steps)
    reset()
    batch.step(EX_NSTEPS)
    stream.synchronize()

    def fp64_solve(c, u0, nsteps):
        it = synth.moving_well_1d(c=c, M=EX_M, nsteps=nsteps, T=EX_T)
        ref = Problem((EX_M,), it.dt, nsteps, precision="fp64", potential="table")
        ref.set_potential_fn(it.V_at)
        ref.set_initial(u0)
        ref.step(nsteps)
        u = ref.read_u(0)
        ref.close()
        return u

    errs = {}
    for (base, u0), pr, c in zip(sweeps, probs, EX_SPEEDS):
        ref = fp64_solve(c, u0[0], EX_NSTEPS)
        errs[f"c={c:g}"] = float(np.linalg.norm(pr.read_u(0) - ref) / np.linalg.norm(ref))
        if c == 30.0:
            fine = fp64_solve(c, u0[0], 2 * EX_NSTEPS)
            err_dt = float(np.linalg.norm(ref - fine) / np.linalg.norm(fine))
    e2e = None
    if not args.no_e2e:
        out = [torch.empty((B, EX_M), dtype=torch.complex128).pin_memory() for _ in probs]
        e2e_times = []
        for _ in range(max(1, min(args.steps, 3))):
            stream.synchronize()
            barrier()
            t0 = time.perf_counter()
            load_inputs()
            batch.step(EX_NSTEPS)
            for pr, o in zip(probs, out):
                pr.read_u(-1, out=o)
            e2e_times.append(time.perf_counter() - t0)
        te = max_over_ranks(float(np.mean(e2e_times)), ws, "cuda")
        e2e = {"value": ws * points * EX_NSTEPS / te, "unit": "point-steps/s",
               "h2d_bytes_per_step": points * 16 + sum(int(t.numel()) * 8 for t in tables),
               "d2h_bytes_per_step": points * 16}
    batch.close()
    for pr in probs:
        pr.close()
    return dict(value=value, t_solve=t_solve, roofline=roofline, e2e=e2e, clocks=clk.summary(), points=points,
                B=B, shape=shape, errs=errs, err_dt=err_dt, rows=int(times_v.size))


def example1_profile_run(args):
    """Small fixed launch sequence for ncu: the three speeds' Problems one
    after the other, each init + start-up + K Adams steps (single-size kernels)."""
    import torch
    from paper_2001_06113_gb300 import Problem
    B = args.batch if args.batch > 0 else EX_B
    for c in EX_SPEEDS:
        base, u0 = synth.example1_sweep(B, c, M=EX_M, nsteps=EX_NSTEPS, T=EX_T)
        pr = Problem((EX_M,), base.dt, EX_NSTEPS, batch=B, precision="mixed", potential="shared_table")
        pr.set_potential_fn(base.V_at)
        for b in range(B):
            pr.set_initial(u0[b], instance=b)
        pr.step(STARTUP + args.profile_adams)
        torch.cuda.synchronize()
        pr.check_finite()
        pr.close()
    print(json.dumps({"profile_adams": args.profile_adams, "batch_per_speed": B, "workload": "example1",
                      "k_periodic1d_launches_before_adams": 1 + STARTUP * 16}))
    return 0


def main_example1(args, ws, rank, local):
    import torch
    if args.impl == "reference":
        if rank != 0:
            return 0
        for _ in range(args.warmup):
            example1_oracle_sample(20)
        vals = [example1_oracle_sample(400)[0] for _ in range(args.steps)]
        value = float(np.mean(vals))
        print(json.dumps({"impl": "reference", "metric": EX_METRIC, "value": value, "unit": "point-steps/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * EX_M / value, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "Example 1 moving well (CPU oracle sample: 400 Adams steps of one "
                                                 "M=512 instance, c=30)"},
                          "cpu_baseline": {"value": value, "unit": "point-steps/s", "cores": cpu_cores(),
                                           "kind": "oracle", "sample": "400 Adams steps of one M=512 instance"},
                          "e2e": {"value": value, "unit": "point-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    if args.profile_adams:
        return example1_profile_run(args)
    if ws > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    res = run_example1(args, ws, rank, local)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            v, el = example1_oracle_sample(2000)
            cpu = {"value": v, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"2000 8th-order Adams steps of one M=512 instance ({el:.1f} s; direct DFT sums)"}
        line = {
            "metric": EX_METRIC, "value": res["value"], "unit": "point-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["t_solve"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
            "data": "synthetic",
            "config": {"workload": f"Example 1: periodic Gaussian well V0=300, beta=0.2 moving at c=15, 30, 45; per "
                                   f"speed {res['B']} initial states (ground state shifted and momentum-kicked) "
                                   f"sharing one V(x,t) table ({res['rows']} rows); M=512, T=2pi/15, 3200 steps, "
                                   "8th-order Adams, mixed; the three speeds in one batch (tuned: fused launch or "
                                   "parallel streams)",
                       "grid": [EX_M], "nsteps": EX_NSTEPS, "dt": EX_T / EX_NSTEPS, "order": ORDER,
                       "instances_per_gpu": 3 * res["B"], "launch_shape": res["shape"],
                       "l2": f"flushed (256 MB write) before each timed solve; per-step working set "
                             f"{res['points'] * 80 / 1e6:.0f} MB",
                       "step": "one whole solve (init, 7 Richardson start-up steps, 3193 Adams steps)",
                       "parallelism": f"replicas x{ws}"},
            "rel_l2_vs_fp64": res["errs"], "fp64_dt_error_c30": res["err_dt"],
            "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"], "clocks": res["clocks"],
            "gpu_launches": (3 * (1 + STARTUP * (4 + 15 + 1 + 1) + 1) + (EX_NSTEPS - STARTUP)) * args.steps,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------------------ request loop arm
SV_RATE, SV_DURATION, SV_T, SV_BUDGET = 200.0, 1.0, (0.05, 0.2), 64 << 30
SV_METRICS = {"fp64": "aggregate point-steps/s of a served request stream (1D/2D periodic mixed, 2D free space FP64)",
              "mixed": "aggregate point-steps/s of a served request stream (1D/2D periodic mixed, 2D free space "
                       "FP32 transforms)"}


def main_serve(args, ws, rank, local):
    import torch
    from paper_2001_06113_gb300.serve import (FREE_EPS, Request, Server, TorchBackend, free_contour_params,
                                              requests_from_trace)
    fprec = args.precision          # free-space requests: "mixed" (FP32 transforms) or "fp64"
    if args.impl == "reference":
        if rank != 0:
            return 0
        # the oracle on the 1D part of the stream: a bounded sample of Adams steps
        for _ in range(args.warmup):
            batch1d_oracle_sample(2)
        vals = [batch1d_oracle_sample(20)[0] for _ in range(args.steps)]
        value = float(np.mean(vals))
        print(json.dumps({"impl": "reference", "metric": SV_METRICS[fprec], "value": value, "unit": "point-steps/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * 1024 * 20 / value, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "served stream (CPU oracle sample: 20 Adams steps, 1D N=1024)"},
                          "cpu_baseline": {"value": value, "unit": "point-steps/s", "cores": cpu_cores(),
                                           "kind": "oracle", "sample": "20 Adams steps of one N=1024 instance"},
                          "e2e": {"value": value, "unit": "point-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    # warm-up: a short stream of small solves (kernel attributes, allocator)
    warm = synth.serve_requests(seed=99, rate=100.0, duration=0.1, T_range=(0.005, 0.01), sizes_1d=(1024,),
                                sizes_2d=(128,), sizes_free=(64,))
    Server(TorchBackend(), SV_BUDGET).run(requests_from_trace(warm, free_precision=fprec))
    if args.full_config:
        dur, T_range, R = 10.0, (0.5, 2.0), 8
        trace = synth.serve_requests(seed=5, rate=SV_RATE, duration=dur, T_range=T_range,
                                     sizes_1d=tuple(2 ** p for p in range(10, 17)),
                                     sizes_free=tuple(2 ** p for p in range(6, 10)))
    else:
        dur, T_range, R = SV_DURATION, SV_T, 8
        trace = synth.serve_requests(seed=5, rate=SV_RATE, duration=SV_DURATION, T_range=SV_T)
    reqs = requests_from_trace(trace, free_precision=fprec, free_R=R)
    srv = Server(TorchBackend(), SV_BUDGET, max_active=64)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        st = srv.run(reqs)
        torch.cuda.synchronize()
    by_kind = {}
    for (t, kind, inst), r in zip(trace, reqs):
        d = by_kind.setdefault(kind, {"n": 0, "point_steps": 0.0, "lat": []})
        d["n"] += 1
        d["point_steps"] += r.points * r.nsteps
        d["lat"].append(r.latency)
    classes = {k: {"requests": v["n"], "point_steps": v["point_steps"],
                   "p50_s": float(np.percentile(v["lat"], 50)), "p99_s": float(np.percentile(v["lat"], 99))}
               for k, v in by_kind.items()}
    # stated accuracy: mixed results vs the FP64 path, solved alone (also timed: the plain path);
    # free space against FP64 on the eps = 1e-10 contour
    # the error sample: the four cheapest requests (points x steps) of each class
    def cheapest(kind, n):
        cls = [(r, k) for r, (t, k, inst) in zip(reqs, trace) if k == kind]
        return sorted(cls, key=lambda x: x[0].points * x[0].nsteps)[:n]
    per = cheapest("1d", 4) + cheapest("2d", 4)
    fre = cheapest("free", 4) if fprec == "mixed" else []
    errs, ferrs, f64_work, f64_time = [], [], 0.0, 0.0
    for r, kind in per + fre:
        if kind == "free":
            ref = Request(r.rid, 0.0, r.inst, bc="free", precision="fp64",
                          free=free_contour_params(r.inst, FREE_EPS["fp64"]))
        else:
            ref = Request(r.rid, 0.0, r.inst, precision="fp64")
        be = TorchBackend()
        h = be.prepare(ref)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        be.start(h)
        torch.cuda.synchronize()
        f64_time += time.perf_counter() - t0
        f64_work += r.points * r.nsteps
        u = be.finish(h)
        e = float(np.sqrt(np.sum(np.abs(r.result - u) ** 2) / np.sum(np.abs(u) ** 2)))
        (ferrs if kind == "free" else errs).append(e)
    line = {
        "metric": SV_METRICS[fprec], "value": st["point_steps_per_s"], "unit": "point-steps/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": st["makespan_s"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64+f64 (periodic), " + ("c64+c128 (free space)" if fprec == "mixed" else "c128 (free space)"),
        "data": "synthetic",
        "config": {"workload": f"Poisson stream {SV_RATE:.0f} req/s for {dur:.1f} s ({len(reqs)} requests): "
                               f"1D periodic N 2^10..2^{16 if args.full_config else 14}, 2D periodic 2^7..2^10, "
                               f"2D free space 2^6..2^{9 if args.full_config else 8} (nu = {R}n, "
                               f"{'FP32 transforms, eps = 1e-4' if fprec == 'mixed' else 'FP64, eps = 1e-10'}), "
                               f"one third each; T ~ U[{T_range[0]}, {T_range[1]}], dt log-uniform [2e-4, 2e-3]"
                               + (" (the stated request-stream configuration)" if args.full_config else
                                  " (a reduced stream: T scaled by 0.1, 1 s of arrivals, smaller 1D and "
                                  "free-space sizes)"),
                   "hbm_budget_bytes": SV_BUDGET, "max_active": 64,
                   "step": "the whole stream from the first arrival to the last result on the host"},
        "time_to_solution_s": {"p50": st["p50_s"], "p99": st["p99_s"], "mean": st["mean_s"]},
        "classes": classes, "peak_active": st["peak_active"], "peak_workspace_bytes": st["peak_bytes"],
        "completed": st["completed"], "failed": st["failed"],
        "rel_l2_vs_fp64_max": max(errs) if errs else None,
        "free_rel_l2_vs_fp64_eps1e-10_max": max(ferrs) if ferrs else None,
        "error_sample": "the four cheapest requests of each class, solved alone by the FP64 path (free space: FP64 "
                        "transforms on the eps = 1e-10 contour, nu = 8n); the GPU test suite checks the cheapest "
                        "requests of the stated stream against the CPU oracle",
        "fp64_one_at_a_time_point_steps_per_s": f64_work / f64_time if f64_time else None,
        "roofline": None, "cpu_baseline": None,
        "e2e": {"value": st["point_steps_per_s"], "unit": "point-steps/s",
                "h2d_bytes_per_step": sum(r.points * 24 for r in reqs),
                "d2h_bytes_per_step": sum(r.points * 16 for r in reqs)},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------ 3D periodic
M3, DT3, NSTEPS3 = 128, 1e-3, 500


def oracle_sample_3d(nadams: int = 1):
    """The CPU oracle on one 128^3 instance of the 3D workload: `nadams`
    Adams steps with a seeded history (direct O(M^2) sums per axis)."""
    from oracle.periodic import oracle_for
    it = synth.periodic_3d_wells(seed=2, M=M3, dt=DT3, nsteps=NSTEPS3)
    orc = oracle_for(it)
    u = it.u0
    h0 = orc.fwd(orc.V(0.0) * u)
    n0 = 100
    hist = {n0 - j: h0 for j in range(1, ORDER)}
    t0 = time.perf_counter()
    for k in range(nadams):
        n = n0 + k
        u = orc.adams_step(u, n * DT3, hist, n)
        hist[n] = orc.fwd(orc.V(n * DT3) * u)
        hist.pop(n - ORDER, None)
    el = time.perf_counter() - t0
    return M3 ** 3 * nadams / el, el


def launches_per_solve_3d(mixed: bool, groups: int) -> int:
    """Kernel launches of one tdse_step(NSTEPS3) call on a 3D context: one
    unfused application of the step operator is 5 kernels (column pass,
    axis-1 pass, row pass, axis-1 pass, column pass); each Adams step of a
    group chain is 4 (row pass, axis-1, fused column pass, axis-1)."""
    L = ORDER // 2
    sub = sum(2 ** c for c in range(L))
    startup = STARTUP * (L + sub * 5 + 1 + 5)
    k = NSTEPS3 - STARTUP
    adams = groups * (2 + (k - 1) * 4 + 3)
    return 4 + startup + (1 if mixed else 0) + adams


def main_periodic3d(args, ws, rank, local):
    """3D periodic wells (128^3, dt = 1e-3, 500 steps, 8th order), a batch of
    seeded instances: whole-solve throughput, the Adams step against HBM
    (mixed) or the FP64 rate, and the error against the FP64 GPU path."""
    import torch
    from paper_2001_06113_gb300 import Problem
    if args.impl == "reference":
        if rank != 0:
            return 0
        for _ in range(args.warmup):
            oracle_sample_3d(1)
        vals = [oracle_sample_3d(1)[0] for _ in range(args.steps)]
        v = float(np.mean(vals))
        print(json.dumps({"impl": "reference", "metric": "point-steps/s (3D periodic 128^3, 8th-order)", "value": v,
                          "unit": "point-steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * M3 ** 3 / v, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "3D periodic wells 128^3, dt=1e-3, 8th-order Adams (CPU oracle sample)"},
                          "cpu_baseline": {"value": v, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                                           "sample": "1 Adams step of one 128^3 instance per bench step"},
                          "e2e": {"value": v, "unit": "point-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    if ws > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    B = args.batch if args.batch > 0 else (8 if args.precision == "mixed" else 2)
    insts = [synth.periodic_3d_wells(seed=1000 * rank + 2 + i, M=M3, dt=DT3, nsteps=NSTEPS3) for i in range(B)]
    P3 = M3 ** 3
    prob = Problem((M3, M3, M3), DT3, NSTEPS3, order=ORDER, batch=B, precision=args.precision, stream=stream)
    pinned_V = [torch.from_numpy(it.V0).pin_memory() for it in insts]
    pinned_u = torch.from_numpy(np.stack([it.u0 for it in insts])).pin_memory()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def load_inputs():
        for b, it in enumerate(insts):
            prob.set_potential(pinned_V[b], None, instance=b)
            p = it.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial_batch(pinned_u)

    load_inputs()
    if args.profile_adams:      # launch sequence for ncu: start-up + K Adams steps, untimed
        with torch.cuda.stream(stream):
            prob.step(STARTUP + args.profile_adams)
        stream.synchronize()
        prob.close()
        print(json.dumps({"profile_adams": args.profile_adams, "workload": "periodic3d", "batch": B,
                          "precision": args.precision}))
        return 0
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            prob.set_initial_batch(pinned_u)
            prob.step(NSTEPS3)
    stream.synchronize()
    times = []
    with ClockSampler(local) as clk:
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                prob.set_initial_batch(pinned_u)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                prob.step(NSTEPS3)
                e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
    t_solve = max_over_ranks(float(np.mean(times)), ws, dev)
    value = ws * B * P3 * NSTEPS3 / t_solve
    GROUP, NGROUPS = 25, 8
    with torch.cuda.stream(stream):
        prob.set_initial_batch(pinned_u)
        prob.step(STARTUP + 8)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(NGROUPS + 1)]
        evs[0].record(stream)
        for i in range(NGROUPS):
            prob.step(GROUP)
            evs[i + 1].record(stream)
    stream.synchronize()
    dts = np.array([evs[i].elapsed_time(evs[i + 1]) / 1e3 / GROUP for i in range(NGROUPS)])
    t_step = float(np.mean(dts))
    if args.precision == "mixed":
        peak, src = hbm_peak()
        ach = ALGO_BYTES["mixed"] * B * P3 / t_step / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": None, "peak_source": src, "algorithmic_bytes_per_point_step": ALGO_BYTES["mixed"],
                "kernel": "3D Adams step operator: column pass (axis 0), axis-1 passes, row pass (axis 2), "
                          f"timed over groups of {GROUP} steps"}
    else:
        peak, src = fp64_peak(dev)
        fl = 6 * 35 + (6 * 18 + 7 * 4 + 4 + 18) + 21 + 4 + 6   # six 128-point transforms per point, 3-axis phases
        ach = fl * B * P3 / t_step / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 4), "unit": "TFLOP/s (FP64)",
                "frac": round(ach / peak, 4), "traffic": None, "peak_source": src,
                "algorithmic_flops_per_point_step": fl,
                "kernel": f"3D FP64 Adams step operator, timed over groups of {GROUP} steps"}
    roof["step_ms_p50"] = round(float(np.percentile(dts, 50)) * 1e3, 4)
    roof["step_ms_p99"] = round(float(np.percentile(dts, 99)) * 1e3, 4)
    err = None
    if args.precision == "mixed" and rank == 0:
        ref = Problem((M3, M3, M3), DT3, NSTEPS3, order=ORDER, batch=1, precision="fp64", stream=stream)
        it = insts[0]
        ref.set_potential(it.V0)
        p = it.pulse
        ref.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
        ref.set_initial(it.u0)
        with torch.cuda.stream(stream):
            ref.step(NSTEPS3)
            prob.set_initial_batch(pinned_u)
            prob.step(NSTEPS3)
        a, r = prob.read_u(0), ref.read_u(0)
        err = float(np.sqrt(np.sum(np.abs(a - r) ** 2) / np.sum(np.abs(r) ** 2)))
        ref.close()
    out = torch.empty((B,) + (M3,) * 3, dtype=torch.complex128).pin_memory()
    e2e_t = []
    with torch.cuda.stream(stream):
        for _ in range(max(1, min(args.steps, 2))):
            flush.zero_()
            stream.synchronize()
            t0 = time.perf_counter()
            load_inputs()
            prob.step(NSTEPS3)
            prob.read_u(-1, out=out)
            e2e_t.append(time.perf_counter() - t0)
    te = max_over_ranks(float(np.mean(e2e_t)), ws, dev)
    shape = prob.describe_steps()
    prob.close()
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            v, el = oracle_sample_3d(1)
            cpu = {"value": v, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"1 Adams step of one 128^3 instance ({el:.1f} s; direct O(M^2) sums per axis)"}
        print(json.dumps({
            "metric": "point-steps/s (3D periodic 128^3, 8th-order, T=0.5)", "value": value, "unit": "point-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_solve * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+f64" if args.precision == "mixed" else "c128", "data": "synthetic",
            "config": {"workload": f"3D periodic wells 128^3, T=0.5, dt=1e-3 (500 steps), 8th-order Adams, "
                                   f"batch of {B} seeded instances per GPU, {args.precision}",
                       "l2": "flushed (256 MB write) before each timed solve", "launch_shape": shape,
                       "step": "one whole solve (7 Richardson start-up + 493 Adams steps) of the batch"},
            "rel_l2_vs_fp64": err, "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": ws * B * P3 * NSTEPS3 / te, "unit": "point-steps/s",
                    "h2d_bytes_per_step": B * (P3 * 8 + P3 * 16), "d2h_bytes_per_step": B * P3 * 16},
            "clocks": clk.summary(),
            "gpu_launches": launches_per_solve_3d(args.precision == "mixed", shape.get("groups", 1)) * args.steps}))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main_free_ctype(args, ws, rank, local):
    """Cost of the C-type transforms against the dyadic refinement n_r of the
    Gauss panels (N^C = 2 q n_r modes; n_r = O(log T) for long runs, Sec. 6):
    ms per Adams step of the 2D free-space workload (256^2, nu = 2048, FP64)
    with the C block as direct sums and through the Chebyshev interpolant
    (Sec. 4.1), n_r = 1..4, timed over 40 steps after the start-up."""
    import torch
    from paper_2001_06113_gb300 import Problem
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    inst = free_instances(0, 1)[0]
    H = free_H([inst], "fp64")
    rows = []
    for n_r in (1, 2, 3, 4):
        for ct in ("direct", "chebyshev"):
            prob = Problem((FS_M, FS_M), FS_DT, FS_NSTEPS, order=ORDER, precision="fp64", stream=stream, bc="free",
                           nu=(FS_NU, FS_NU), H=H, gauss_q=FS_Q, n_r=n_r, c_transform=ct)
            prob.set_potential(inst.V0, None)
            p = inst.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
            prob.set_initial(inst.u0)
            with torch.cuda.stream(stream):
                prob.step(STARTUP + 4)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                prob.step(40)
                e1.record(stream)
            stream.synchronize()
            rows.append({"n_r": n_r, "NC": FS_Q * 2 * n_r, "c_transform": ct, "N_T": prob.cheb_terms(0),
                         "ms_per_step": round(e0.elapsed_time(e1) / 40, 4)})
            prob.close()
    print(json.dumps({"workload": "free-space C-type transform cost vs n_r (2D 256^2, nu = 2048, FP64, H for "
                                  "eps = 1e-10)", "unit": "ms per Adams step", "rows": rows}))
    return 0


# ------------------------------------------------------------ 3D free space
F3_M, F3_NU, F3_DT, F3_NSTEPS, F3_Q, F3_NR = 64, 256, 1e-3, 200, 10, 1
F3_EPS = {"fp64": 1e-10, "mixed": 1e-4}
F3_DIR = (1.0, -0.5, 0.3)


def free3d_instance(seed: int = 3):
    return synth.free_bump_gaussians((F3_M,) * 3, seed=seed, dt=F3_DT, nsteps=F3_NSTEPS, A0=2.0, omega=10.0,
                                     direction=F3_DIR)


def free3d_H(inst, precision: str) -> float:
    from paper_2001_06113_gb300 import free_choose_H
    vnorm = math.sqrt(float(np.sum(inst.V0 ** 2)) * (2.0 / F3_M) ** 3)
    t = np.linspace(0.0, F3_NSTEPS * F3_DT, 4001)
    A = inst.pulse.A(t)
    phi = np.concatenate([np.zeros((1, A.shape[1])), np.cumsum(0.5 * (A[1:] + A[:-1]) * (t[1] - t[0]), axis=0)])
    return free_choose_H(F3_EPS[precision], vnorm, float(np.max(np.abs(phi))), 3, precision=precision)


def free3d_flops_per_step(N: int) -> float:
    """Real FP64 flops of one 3D free-space Adams step (64^3, nu = 256), per
    instance, counted as for 2D (complex mul 6, add 2, FFT 5 n log2 n): the
    row pass over the N0 N1 mode rows (forward and inverse along axis 2 and
    the per-mode update and Horner history), the axis-1 passes over the N0 M2
    lines (one inverse, one forward), the grid pass over the M1 M2 columns
    (inverse and forward along axis 0, implicit solve and V u)."""
    M, nu = F3_M, F3_NU
    R = nu // M
    ne = nu // 2 - 13
    nd = N - 2 * ne
    fft = 2 * R * 5 * M * math.log2(M)
    fwd = 2 * nu * 6 + fft + 2 * ne * 6 + nd * M * 8
    inv = 2 * ne * 6 + fft + 2 * nu * 8 + nd * M * 8
    horner = 7 * 2 + 6 * (6 + 6 + 2) + 6 + 6 + 4 + 6          # + the product of the two row phases
    row = N * N * (fwd + inv + N * (4 + horner))
    mid = N * M * (inv + fwd)
    col = M * M * (inv + fwd + M * 14)
    return row + mid + col


def free3d_algo_bytes(N: int, e: int) -> float:
    """Algorithmic DRAM bytes of one 3D free-space Adams step (e = ring and
    intermediate element bytes): per mode the FP64 state read and W written
    (32 B), 6 ring lags read and the new (Vu)^ written (7 e); Z [N0][N1][M2]
    and Y [N0][M1][M2] each written and read twice (once per direction); per
    grid point V read (8 B) and u written (16 B)."""
    M = F3_M
    return N ** 3 * (32 + 7 * e) + 4 * N * N * M * e + 4 * N * M * M * e + M ** 3 * 24


# DRAM bytes of one fused k_fs_row<float2, 64, 4> launch of the 64^3 step (ncu
# launch list, read 1169.4 MB + write 445.5 MB).
F3_ROW_TRAFFIC_MIXED = 1169.4e6 + 445.5e6


def free3d_oracle_sample(N_adams: int = 1):
    """point-steps/s of the CPU oracle: Adams steps of one 64^3 instance from a
    synthetic history (dense transform matrices per axis)."""
    from oracle import fields, gamma
    from oracle.freespace import FreeSpaceOracle
    inst = free3d_instance()
    H = free3d_H(inst, "fp64")
    rules = [gamma.GammaRule.for_nu(F3_M, F3_NU, H, q=F3_Q, n_r=F3_NR) for _ in range(3)]
    orc = FreeSpaceOracle(rules, F3_DT, inst.V0, inst.vfac, fields.phi_callable(inst.pulse, 3), order=ORDER)
    uh = orc.fwd(inst.u0)
    h0 = orc.fwd(orc.V(0.0) * inst.u0)
    n0 = 20
    hist = {n0 - j: h0 for j in range(1, ORDER)}
    t0 = time.perf_counter()
    for k in range(N_adams):
        n = n0 + k
        uh, _, hist[n] = orc.adams_step(uh, n * F3_DT, hist, n)
        hist.pop(n - ORDER, None)
    el = time.perf_counter() - t0
    return F3_M ** 3 * N_adams / el, el


def main_free3d(args, ws, rank, local):
    """3D free space (Sec. 4.3): one 64^3 instance, nu = 256 per axis (N = 266
    modes per axis, 1.9e7 modes), q = 10, n_r = 1, 8th-order Adams, T = 0.2
    (200 steps), A along (1, -0.5, 0.3).  Whole-solve throughput in grid
    point-steps/s; the Adams step against the FP64 rate measured here (FP64)
    or against the FP32 rate (mixed), with the error of the mixed path against
    the FP64 path on the same contour."""
    import torch
    from paper_2001_06113_gb300 import Problem
    prec = args.precision
    metric = f"point-steps/s (3D free space 64^3, nu=256, 8th-order, T=0.2, {prec})"
    if args.impl == "reference":
        if rank != 0:
            return 0
        for _ in range(args.warmup):
            free3d_oracle_sample(1)
        vals = [free3d_oracle_sample(1)[0] for _ in range(args.steps)]
        v = float(np.mean(vals))
        print(json.dumps({"impl": "reference", "metric": metric, "value": v, "unit": "point-steps/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * F3_M ** 3 / v, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "3D free space 64^3, nu=256 (CPU oracle sample)"},
                          "cpu_baseline": {"value": v, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                                           "sample": "1 Adams step of one 64^3 instance per bench step"},
                          "e2e": {"value": v, "unit": "point-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    inst = free3d_instance()
    H = free3d_H(inst, prec)

    def make(precision, Hh):
        pr = Problem((F3_M,) * 3, F3_DT, F3_NSTEPS, order=ORDER, precision=precision, stream=stream, bc="free",
                     nu=(F3_NU,) * 3, H=Hh, gauss_q=F3_Q, n_r=F3_NR)
        pr.set_potential(inst.V0, None)
        p = inst.pulse
        pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
        pr.set_initial(inst.u0)
        return pr

    prob = make(prec, H)
    N = prob.mode_shape[0]
    if args.profile_adams:      # launch sequence for ncu: start-up + K Adams steps, untimed
        with torch.cuda.stream(stream):
            prob.step(STARTUP + args.profile_adams)
        stream.synchronize()
        prob.close()
        print(json.dumps({"profile_adams": args.profile_adams, "workload": "free3d", "precision": prec}))
        return 0
    pinned_u = torch.from_numpy(inst.u0.copy()).pin_memory()
    pinned_V = torch.from_numpy(inst.V0.copy()).pin_memory()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            prob.set_initial(pinned_u)
            prob.step(F3_NSTEPS)
    stream.synchronize()
    times = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                prob.set_initial(pinned_u)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                prob.step(F3_NSTEPS)
                e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    t_solve = float(np.mean(times))
    points = F3_M ** 3
    value = points * F3_NSTEPS / t_solve
    GROUP, NGROUPS = 5, 10
    with torch.cuda.stream(stream):
        prob.set_initial(pinned_u)
        prob.step(STARTUP + 4)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(NGROUPS + 1)]
        evs[0].record(stream)
        for i in range(NGROUPS):
            prob.step(GROUP)
            evs[i + 1].record(stream)
    stream.synchronize()
    dts = np.array([evs[i].elapsed_time(evs[i + 1]) / 1e3 / GROUP for i in range(NGROUPS)])
    t_step = float(np.mean(dts))
    flops = free3d_flops_per_step(N)
    achieved = flops / t_step / 1e12
    timing = {"kernel": "3D free-space Adams step (k_fs_row end+begin, k_fs_mid inverse, k_fs_phys, k_fs_mid "
                        "forward), timed over groups of 5 steps",
              "algorithmic_flops_per_step": flops, "modes_per_axis": N,
              "step_ms_p50": round(float(np.percentile(dts, 50)) * 1e3, 4)}
    if prec == "fp64":
        peak, src = fp64_peak(dev)
        roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 4), "traffic": None, "peak_source": src, **timing}
    else:
        # FP32 transforms: both ceilings, the nearer one reported as the bound
        algo = free3d_algo_bytes(N, 8)
        hpk, hsrc = hbm_peak()
        gbs = algo / t_step / 1e9
        hbm = {"achieved": round(gbs, 1), "peak": hpk, "unit": "GB/s", "frac": round(gbs / hpk, 4),
               "algorithmic_bytes_per_step": algo, "peak_source": hsrc}
        alu = {"achieved": round(achieved, 4), "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s",
               "frac": round(achieved / FP32_PEAK_TFLOPS, 4), "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"}
        top, other = ("hbm", "alu") if hbm["frac"] >= alu["frac"] else ("alu", "hbm")
        pick = {"hbm": hbm, "alu": alu}
        roofline = {"bound": top, **pick[top], "traffic": F3_ROW_TRAFFIC_MIXED,
                    "traffic_unit": "DRAM bytes per fused k_fs_row launch (ncu), the step's dominant kernel",
                    "other_ceiling": {"bound": other, **pick[other]}, **timing}
    e2e = None
    if not args.no_e2e:
        out = torch.empty((F3_M,) * 3, dtype=torch.complex128).pin_memory()
        with torch.cuda.stream(stream):
            stream.synchronize()
            t0 = time.perf_counter()
            prob.set_potential(pinned_V, None)
            prob.set_initial(pinned_u)
            prob.step(F3_NSTEPS)
            prob.read_u(0, out=out)
            te = time.perf_counter() - t0
        e2e = {"value": points * F3_NSTEPS / te, "unit": "point-steps/s", "h2d_bytes_per_step": points * 24,
               "d2h_bytes_per_step": points * 16}
    err = None
    if prec == "mixed":
        ref = make("fp64", H)
        with torch.cuda.stream(stream):
            prob.set_initial(pinned_u)
            prob.step(40)
            ref.step(40)
        stream.synchronize()
        um, ud = prob.read_u(0), ref.read_u(0)
        err = {"rel_l2_vs_fp64_same_contour": float(np.linalg.norm(um - ud) / np.linalg.norm(ud)), "after_steps": 40}
        ref.close()
    ws_bytes = prob.workspace_bytes
    prob.close()
    cpu = None
    if not args.no_cpu_baseline:
        v, el = free3d_oracle_sample(1)
        cpu = {"value": v, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"1 8th-order Adams step of the 64^3 instance ({el:.1f} s; dense transforms per axis)"}
    print(json.dumps({
        "metric": metric, "value": value, "unit": "point-steps/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128" if prec == "fp64" else "c64+c128", "data": "synthetic",
        "config": {"workload": f"3D free space 64^3, nu=256 (N={N} modes/axis), p=8, q=10, n_r=1, H={H:.4f} "
                               f"(eps={F3_EPS[prec]:g}), dt=1e-3, 200 steps, 8th-order Adams, {prec}",
                   "workspace_bytes": ws_bytes, "l2": "flushed (256 MB write) before each timed solve",
                   "step": "one whole solve (7 Richardson start-up + 193 Adams steps)"},
        "stated_err": err, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary()}))
    return 0


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.precision is None:
        args.precision = "fp64" if args.workload == "free2d" else "mixed"
    if args.batch <= 0 and args.workload == "periodic3d":
        args.batch = 16 if args.precision == "mixed" else 2
    if args.batch <= 0 and args.workload != "example1":
        args.batch = 1 if args.workload == "free2d" else (64 if args.precision == "mixed" else 4)
    if args.workload == "free2d":
        return main_free(args, ws, rank, local)
    if args.workload == "batch1d":
        return main_batch1d(args, ws, rank, local)
    if args.workload == "serve":
        return main_serve(args, ws, rank, local)
    if args.workload == "example1":
        return main_example1(args, ws, rank, local)
    if args.workload == "periodic3d":
        return main_periodic3d(args, ws, rank, local)
    if args.workload == "free_ctype":
        return main_free_ctype(args, ws, rank, local)
    if args.workload == "free3d":
        return main_free3d(args, ws, rank, local)
    if args.impl == "reference":
        if rank != 0:
            return 0
        vals = []
        for _ in range(args.warmup):
            oracle_sample(nadams=2)
        for _ in range(args.steps):
            v, _ = oracle_sample(nadams=20)
            vals.append(v)
        value = float(np.mean(vals))
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "point-steps/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * M * M * 20 / value, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "2D periodic wells 512x512, dt=1e-3, 8th-order Adams (CPU oracle sample)",
                           "grid": [M, M], "dt": DT, "order": ORDER},
                "cpu_baseline": {"value": value, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                                 "sample": "20 Adams steps of one 512^2 instance per bench step (direct O(M^2) DFT sums)"},
                "e2e": {"value": value, "unit": "point-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if args.profile_adams:
        return profile_run(args)
    if ws > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    res = run_gpu(args, ws, rank, local)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            # spawn-free: the oracle runs in this process after all GPU work is done
            v, el = oracle_sample(nadams=60)
            cpu = {"value": v, "unit": "point-steps/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"60 8th-order Adams steps of one 512^2 instance ({el:.1f} s; direct O(M^2) DFT sums, "
                             "numpy/OpenBLAS)",
                   "value_1core": oracle_sample_one_core(10),
                   "sample_1core": "10 Adams steps of the same instance with one BLAS/OpenMP thread"}
        line = {
            "metric": METRIC, "value": res["value"], "unit": "point-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["t_solve"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+f64" if args.precision == "mixed" else "c128",
            "data": "synthetic",
            "config": {"workload": f"2D periodic wells 512x512, T=2, dt=1e-3 (2000 steps), 8th-order Adams, "
                                   f"batch of {res['B']} seeded instances per GPU, {args.precision}",
                       "grid": [M, M], "nsteps": NSTEPS, "dt": DT, "order": ORDER, "batch_per_gpu": res["B"],
                       "precision": args.precision, "l2": "flushed (256 MB write) before each timed solve; "
                                                         "per-step working set > L2",
                       "step": "one whole solve (7 Richardson start-up + 1993 Adams steps) of the batch",
                       "parallelism": f"replicas x{ws}"},
            "rel_l2_vs_fp64": res["stated_err"], "norm_drift_T": res["norm_drift"],
            "rel_l2_vs_oracle": (res["oracle_err"] or {}).get("mixed") if isinstance(res["oracle_err"], dict)
            else res["oracle_err"],
            "fp64_variant": res["fp64"],
            "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"], "clocks": res["clocks"],
            "gpu_launches": launches_per_solve(2, args.precision == "mixed",
                                               res["roofline"]["launch_shape"]["path"]) * args.steps,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
