#!/usr/bin/env python3
"""Benchmark of the matrix-free H*psi hot path on the sinc-DVR workload.

Workload: the Colbert-Miller sinc-DVR harmonic oscillator on D = 131072 grid
points (L = 0.9 sqrt(2D)), one vector (a Gaussian wavepacket at x = 2),
FP32 entry generation with FP64 Chebyshev recurrence.  One step = one
64-term Chebyshev step of exp(-i tau H) (63 matrix-free H*psi applies plus
the FP64 recurrence/accumulation), tau the longest sub-step that 64 terms
resolve at coefficient tolerance 1e-7.  The dense operator would need
275 GB in complex128; it is never stored.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mf|reference]

Under torchrun (N > 1) every rank propagates an independent wavepacket
(parameter-parallel tasks, no collective on the data path) and the job value
is the sum of work over the max time across ranks.  ``--impl reference``
times the CPU oracle on bounded row samples of the same product.

At N = 1 the line also carries, under "workloads", the other
configurations, each timed on its own with its roofline, CPU oracle baseline
and error against the FP64 form: the Philox ensemble at D = 4096 in the FP64
form (one product and a 32-term step), Philox generation at D = 131072 (one
vector, procedural, with the per-pipe roofline against the pipe rates
measured in the same run, "pipe_rates"), the 64-vector Philox workload at
D = 262144 with its 120 GB cache (BF16X2 and FP32 forms, one Chebyshev step),
the 256 batched problems (one step) and the planner comparison on the
shipped sweep records (surrogates trained on the GPU).  --headline-only
leaves them out.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H psi matrix entries applied/s and Chebyshev steps/s at stated error vs FP64 form"
D = 131072
TERMS = 64
TOL = 1e-7
DT_CONFIG = 0.1  # the workload's nominal dt; tau sub-steps cover it
WORKLOAD = "sinc-DVR harmonic oscillator D=131072, 1 vector, 64-term Chebyshev steps"


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ----------------------------------------------------------- multi-rank ---
# N ranks run N independent propagations (weak scaling, no data-path
# collective); the only cross-rank steps are the barriers around the timed
# region and the max-over-ranks job time.
def rank_task(rank):
    """Centre x0 of rank's coherent state (an independent problem per rank)."""
    return 2.0 + 0.25 * rank


def job_seconds(t_local, world, device=None):
    """The slowest rank's seconds (all ranks get the same value)."""
    import torch
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, entries_per_step, t_job):
    """Whole-job entries/s: the units all ranks processed over the job time."""
    return world * steps * entries_per_step / t_job


# ------------------------------------------------------------------ clocks ---
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
            os.unlink(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            busy = [s for s in sm if s > 0.5 * max(sm)] or sm
            out = {"sm_mhz": float(np.median(busy)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# -------------------------------------------------------------- roofline ---
def traffic_from_profile():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, valid only while the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "dvr_rows_f32_D131072.md")
    src = os.path.join(ROOT, "paper_2606_31598_gb300", "csrc", "k_dvr.cu")
    try:
        txt = open(path).read()
        want = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt).group(1)
        traffic = float(re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt).group(1))
    except Exception:
        return None
    have = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return traffic if have == want else None


# ------------------------------------------------------------ CPU oracle ---
def cpu_oracle_sample(target_s=10.0, max_rows=None):
    """Oracle FP64 product on evenly spaced output rows; returns entries/s."""
    from oracle import oracle as O
    import workloads as W
    op = O.make_op(O.GEN_SINC_DVR_HO, D)
    x = W.wavepacket(D)
    O.apply_rows(op, x, np.arange(64, dtype=np.int64))  # thread pool start-up
    rows = np.linspace(0, D - 1, 1024).astype(np.int64)
    t0 = time.perf_counter()
    O.apply_rows(op, x, rows)
    t = time.perf_counter() - t0
    n = int(min(max_rows or D, max(1024, 1024 * target_s / max(t, 1e-6))))
    rows = np.linspace(0, D - 1, n).astype(np.int64)
    t0 = time.perf_counter()
    O.apply_rows(op, x, rows)
    t = time.perf_counter() - t0
    return n * D / t, n, t


def cpu_threads():
    try:
        from oracle import oracle as O  # noqa: F401
        import ctypes
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_get_max_threads.restype = ctypes.c_int
        return int(gomp.omp_get_max_threads())
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    per_step_s = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_sample(target_s=min(per_step_s, 5.0))
    vals, times, nrows = [], [], 0
    for _ in range(args.steps):
        v, nrows, t = cpu_oracle_sample(target_s=per_step_s)
        vals.append(v)
        times.append(t)
    value = float(np.sum([n for n in [nrows * D] * len(times)]) / np.sum(times))
    cores = cpu_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "D": D, "nvec": 1},
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle",
                         "sample": "%d of %d output rows of one FP64 H psi per step" % (nrows, D)},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- GPU ---
def substep_tau(plan):
    """Longest tau whose expansion needs at most TERMS terms at TOL."""
    lo, hi = 1e-7, 1e-2
    for _ in range(50):
        mid = np.sqrt(lo * hi)
        if plan.cheb_terms(mid) <= TERMS:
            lo = mid
        else:
            hi = mid
    return lo


def coherent_state(x, x0, t):
    """Exact unit harmonic oscillator coherent state at time t (psi(x, 0) a
    Gaussian of unit width at x0, zero momentum)."""
    return (np.pi ** -0.25 * np.exp(-0.5j * t) * np.exp(-0.5 * (x - x0 * np.cos(t)) ** 2 - 1j * x0 * np.sin(t) * x
                                                       + 0.25j * x0 * x0 * np.sin(2 * t)))


def run_mf(args):
    import torch
    import torch.distributed as dist

    import paper_2606_31598_gb300 as mf
    import workloads as W

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream().cuda_stream
    props = torch.cuda.get_device_properties(dev)
    x0 = rank_task(rank)

    plan = mf.Plan(D, mf.MF_GEN_SINC_DVR_HO, precision=mf.MF_PREC_FP32, stream=stream, device=local)
    desc = plan.describe()
    emin, emax = plan.bounds()
    tau = substep_tau(plan)
    nterms = plan.cheb_terms(tau)
    assert nterms <= TERMS
    psi0 = W.wavepacket(D, x0=x0)
    psi = torch.from_numpy(psi0).to(dev)
    applies = TERMS - 1
    entries_per_step = applies * float(D) * float(D)

    for _ in range(args.warmup):
        plan.cheb_propagate(psi, 1, tau, TERMS)
    torch.cuda.synchronize()

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clock = ClockSampler(local)
    psi.copy_(torch.from_numpy(psi0).to(dev))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clock.start()
    plan.profile(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record()
        plan.cheb_propagate(psi, 1, tau, TERMS)
        stops[k].record()
    torch.cuda.synchronize()
    kern_ms, kern_n = plan.profile_read()
    plan.profile(False)
    if world > 1:
        dist.barrier()
    clocks = clock.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    t_local = sum(step_ms) / 1e3
    t_job = job_seconds(t_local, world, dev)
    value = job_value(world, args.steps, entries_per_step, t_job)
    psi_timed = psi.cpu().numpy()

    # end to end through the public call: pinned host psi in, result out
    host_in = torch.from_numpy(psi0.copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e_a = torch.cuda.Event(enable_timing=True)
    e_b = torch.cuda.Event(enable_timing=True)
    dpsi = torch.empty_like(psi)
    torch.cuda.synchronize()
    e_a.record()
    for k in range(args.steps):
        dpsi.copy_(host_in, non_blocking=True)
        plan.cheb_propagate(dpsi, 1, tau, TERMS)
        host_out.copy_(dpsi, non_blocking=True)
        host_in, host_out = host_out, host_in
    e_b.record()
    torch.cuda.synchronize()
    t_e2e = job_seconds(e_a.elapsed_time(e_b) / 1e3, world, dev)
    e2e_value = job_value(world, args.steps, entries_per_step, t_e2e)

    # stated error: one step of the FP32 form vs the FP64 form and vs the
    # closed-form coherent state
    err = {}
    if rank == 0:
        plan64 = mf.Plan(D, mf.MF_GEN_SINC_DVR_HO, precision=mf.MF_PREC_FP64, stream=stream, device=local)
        plan64.set_bounds(emin, emax)
        a = torch.from_numpy(psi0).to(dev)
        b = torch.from_numpy(psi0).to(dev)
        plan.cheb_propagate(a, 1, tau, TERMS)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        plan64.cheb_propagate(b, 1, tau, TERMS)
        ev1.record()
        torch.cuda.synchronize()
        fp64_step_s = ev0.elapsed_time(ev1) / 1e3
        a, b = a.cpu().numpy(), b.cpu().numpy()
        L = W.dvr_default_L(D)
        xg = -L + (2 * L / (D - 1)) * np.arange(D)
        exact = coherent_state(xg, x0, tau)
        exact = exact / np.linalg.norm(exact)
        # the BF16 hi+lo split form of the same step (tcgen05 kernel)
        plan16 = mf.Plan(D, mf.MF_GEN_SINC_DVR_HO, precision=mf.MF_PREC_BF16X2, stream=stream, device=local)
        plan16.set_bounds(emin, emax)
        c16 = torch.from_numpy(psi0).to(dev)
        plan16.cheb_propagate(c16, 1, tau, TERMS)
        torch.cuda.synchronize()
        plan16.sync()
        c16 = c16.cpu().numpy()
        # the same step timed in the BF16X2 form (one vector padded to the
        # tensor cores' smallest N of 8 vectors)
        d16 = torch.from_numpy(psi0).to(dev)
        ev0.record()
        plan16.cheb_propagate(d16, 1, tau, TERMS)
        ev1.record()
        torch.cuda.synchronize()
        plan16.sync()
        bf16x2_step_s = ev0.elapsed_time(ev1) / 1e3
        plan16.close()
        err = {"fp32_vs_fp64_form": float(np.linalg.norm(a - b)), "fp32_vs_closed_form": float(np.linalg.norm(a - exact)),
               "bf16x2_vs_fp64_form": float(np.linalg.norm(c16 - b)),
               "fp64_vs_closed_form": float(np.linalg.norm(b - exact)),
               "norm_drift_after_timed_steps": float(abs(np.linalg.norm(psi_timed) - 1.0)),
               "measure": "2-norm of the state difference after one step (unit-norm states)"}
        fp64_entries_per_s = entries_per_step / fp64_step_s
        plan64.close()

    if rank == 0:
        sm_mhz = clocks.get("sm_mhz") or 0.0
        nsm = props.multi_processor_count
        peak = nsm * 128 * 2 * sm_mhz * 1e6 / 1e12 if sm_mhz else None  # TFLOP/s FP32 FMA pipe
        per_launch_s = kern_ms / 1e3 / max(kern_n, 1)
        achieved = 4.0 * D * D / per_launch_s / 1e12
        traffic = traffic_from_profile()
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_job * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "D": D, "nvec": 1, "terms_per_step": TERMS, "applies_per_step": applies,
                       "tau": tau, "substeps_per_dt_0.1": int(np.ceil(DT_CONFIG / tau)),
                       "precision": "fp32 entries and tile sums, fp64 recurrence", "storage": desc["storage"],
                       "path": desc["path"], "launch": [desc["dvr_rows"], desc["dvr_cols"]],
                       "l2": "flushed between timed steps (256 MiB write, outside the step events)",
                       "bounds": [emin, emax]},
            "cheb_terms_per_s": world * args.steps * applies / t_job,
            "cheb_steps_per_s": world * args.steps / t_job,
            "dt_steps_per_s": world * args.steps / t_job / np.ceil(DT_CONFIG / tau),
            "fp64_form_entries_per_s": fp64_entries_per_s,
            "bf16x2_form_entries_per_s": entries_per_step / bf16x2_step_s,
            "error": err,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": (achieved / peak) if peak else None, "traffic": traffic,
                         "kernel": "dvr_rows_f32", "flop_per_launch": 4.0 * D * D,
                         "peak_basis": "%d SMs x 128 FP32 lanes x 2 FLOP x median sampled SM clock" % nsm,
                         "kernel_ms": per_launch_s * 1e3, "kernel_launches_timed": kern_n},
            "e2e": {"value": e2e_value, "unit": "entries/s", "h2d_bytes_per_step": D * 16, "d2h_bytes_per_step": D * 16},
            "gpu_launches": args.steps * (2 + 2 * applies),
            "clocks": clocks,
        }
        cb_value, cb_rows, cb_t = cpu_oracle_sample(target_s=10.0)
        line["cpu_baseline"] = {"value": cb_value, "unit": "entries/s", "cores": cpu_threads(), "kind": "oracle",
                                "sample": "%d of %d output rows of one FP64 H psi (%.1f s)" % (cb_rows, D, cb_t)}
        plan.close()
        plan = None
        if world == 1 and not args.headline_only:
            # the other configurations, each with its own timing, roofline,
            # CPU oracle baseline and error (one GPU, after the headline)
            peaks = measured_peaks()
            rates = mf.mf_pipe_rates(local, stream)
            line["pipe_rates"] = {"ops_per_s": rates,
                                  "per_sm_per_clock_at_max_clock": {
                                      k: v / (props.multi_processor_count * 2.07e9) for k, v in rates.items()},
                                  "source": "mf_pipe_rates: register-only chains, 8 CTAs x 256 threads per SM"}
            line["workloads"] = {}
            for key, fn in (("philox_D4096_fp64", lambda: sub_small_philox(stream, rates)),
                            ("philox_D131072_generation", lambda: sub_philox_generation(stream, rates)),
                            ("philox_D262144_64vec_120GB", lambda: sub_multivector(stream, peaks, rates)),
                            ("batch_256_problems", lambda: sub_batch(stream, rates)),
                            ("planner_sweep_regret", sub_planner)):
                t0 = time.perf_counter()
                line["workloads"][key] = fn()
                line["workloads"][key]["wall_s"] = time.perf_counter() - t0
                torch.cuda.empty_cache()
        print(json.dumps(line))
    if plan is not None:
        plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def measured_peaks():
    """HBM copy GB/s and BF16 TFLOP/s (burst, sustained) measured on this
    pool's GPUs (MEASURED_PEAKS.json beside this file), else the fallback
    figures; the dict says which."""
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return {"hbm_gbs": float(m["hbm_gbs"]), "bf16_tflops": float(m["bf16_tflops"]),
                "bf16_tflops_sustained": float(m["bf16_tflops_sustained"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def events_time(fn, reps):
    """Mean seconds of fn() over reps calls (CUDA events, synchronised)."""
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


# FP64 arithmetic operations of the definition per canonical entry of the
# FP64 Philox form (division and square root counted as one each, so the
# bound is a lower one): the two uniforms (2 each), the log with its
# division and 10-term polynomial (18), -2 log (1), the square root (1),
# sin/cos reduction and two 9-term polynomials (24), sigma scaling (3); plus
# 8 FP64 FMAs per vector for H and H^dagger.  All run on the FP64 pipe.
PHILOX64_DFMA_OPS = 2 + 2 + 18 + 1 + 1 + 24 + 3


def sub_small_philox(stream, rates=None):
    """Plain method, small size: Philox ensemble D = 4096 (seed 1) in the FP64
    form (complex128), block 512, procedural; one H psi plus one 32-term
    Chebyshev step of t = 1 per step, psi random (seed 1).  GPU and CPU
    oracle run the same step in full; the error is against the oracle."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    from oracle import oracle as O
    D, B, NT = 4096, 512, 32
    plan = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=B, precision=mf.MF_PREC_FP64,
                   storage=mf.MF_STORE_PROCEDURAL, stream=stream)
    emin, emax = plan.bounds()
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    psi0 = W.random_state(D, 1, seed=1)
    x = torch.from_numpy(psi0).cuda()
    y = torch.empty_like(x)
    psi = torch.empty_like(x)

    def step():
        plan.apply(y, x, 1)
        psi.copy_(x)
        plan.cheb_propagate(psi, 1, 1.0, NT)

    step()
    plan.profile(True)
    reps = 10
    t = events_time(step, reps)
    kern_ms, kern_n = plan.profile_read()
    plan.profile(False)
    op = O.make_op(O.GEN_PHILOX_GUE, D, seed=1)
    t0 = time.perf_counter()
    ref_y = O.apply(op, psi0, block=B)
    ref_psi = O.cheb_step(op, psi0, 1.0, c, R, NT, block=B)
    t_cpu = time.perf_counter() - t0
    yh, ph = y.cpu().numpy(), psi.cpu().numpy()
    entries = float(NT) * D * D  # one product plus 31 in the step
    plan.close()
    return {"workload": "Philox GUE D=4096 (seed 1), FP64 form, block 512, procedural, 1 vector; one H psi "
                        "plus one 32-term Chebyshev step of t=1",
            "step_s": t, "entries_per_s": entries / t, "products_per_step": NT, "steps_per_s": 1.0 / t,
            "kernel_ms_per_launch": kern_ms / max(1, kern_n),
            "error": {"apply_rel_vs_oracle": float(np.max(np.abs(yh - ref_y)) / np.max(np.abs(ref_y))),
                      "step_abs_vs_oracle": float(np.max(np.abs(ph - ref_psi))),
                      "measure": "FP64 form against the CPU oracle's FP64 statement (same bounds and terms)"},
            "roofline": fp64_roofline(D * (D + 1) / 2.0, kern_ms / 1e3 / max(1, kern_n), rates),
            "cpu_baseline": {"value": entries / t_cpu, "unit": "entries/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": "the whole step (one product plus the 32-term step) in FP64 (%.2f s)" % t_cpu}}


def sub_philox_generation(stream, rates):
    """Seeded generation at the roofline's finest grain: Philox D = 131072
    (seed 1), FP32 form, procedural, one vector (seed 3): every canonical
    entry generated once per product and applied as H and H^dagger.  The
    roofline is per pipe (operations of the definition over the measured
    rate of each pipe); the oracle's FP32 statement of about 4100 rows (tile
    and block boundaries, and evenly spaced ones) is both the CPU baseline
    and the error reference."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    from oracle import oracle as O
    D = 131072
    x0 = W.random_state(D, 1, seed=3)
    x = torch.from_numpy(x0).cuda()
    y = torch.empty_like(x)
    plan = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=2048, precision=mf.MF_PREC_FP32,
                   storage=mf.MF_STORE_PROCEDURAL, stream=stream)
    plan.apply(y, x, 1)
    plan.profile(True)
    t = events_time(lambda: plan.apply(y, x, 1), 5)
    kern_ms, kern_n = plan.profile_read()
    plan.profile(False)
    plan.sync()
    per = kern_ms / 1e3 / max(1, kern_n)
    canon = D * (D + 1) / 2.0
    # rows at tile and block boundaries and 4096 evenly spaced ones: the
    # oracle computes them once, as the CPU baseline and the error reference
    edge = np.array([0, 1, 127, 128, 2047, 2048, 65535, 65536, 100000, 131071])
    rows = np.unique(np.concatenate([edge, np.linspace(0, D - 1, 4096).astype(np.int64)]))
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    plan.close()
    op32 = O.make_op(O.GEN_PHILOX_GUE, D, seed=1, form=O.FORM_FP32)
    t0 = time.perf_counter()
    ref = O.apply_rows(op32, x0.reshape(D, 1), rows)
    t_cpu = time.perf_counter() - t0
    roof = pipe_roofline(canon / per, rates)
    roof["issue_frac"] = canon / per * PHILOX_INSTR_PER_ENTRY / (152 * 128 * 2.07e9)
    return {"workload": "Philox GUE D=131072 (seed 1), FP32 form, procedural, 1 vector (seed 3)",
            "apply_s": t, "kernel_ms": per * 1e3, "entries_per_s": float(D) * D / t,
            "canonical_entries_per_s": canon / per,
            "error": {"rows_rel_vs_oracle": float(np.max(np.abs(got.reshape(-1) - ref.reshape(-1))) /
                                                  np.max(np.abs(ref))),
                      "measure": "%d sampled output rows against the oracle's FP32 statement" % len(rows)},
            "roofline": roof,
            "cpu_baseline": {"value": len(rows) * float(D) / t_cpu, "unit": "entries/s", "cores": cpu_threads(),
                             "kind": "oracle", "sample": "%d of 131072 output rows of one FP32-form H psi "
                                                        "(%.2f s), rate extrapolated" % (len(rows), t_cpu)}}


def sub_multivector(stream, peaks, rates):
    """The 64-vector workload: Philox D = 262144 (seed 1), 64 unit vectors
    (seed 2), block 2048, 120 GB partial cache (3576 of 8256 canonical
    pairs), BF16X2 (tcgen05, Hermitian reuse) and FP32 forms; one Chebyshev
    step of dt = 1 at tolerance 1e-12 in the BF16X2 form.  Errors against the
    FP64 form on 1024 sampled rows computed by the oracle; the CPU baseline
    is the oracle's FP64 product on those rows, extrapolated to all D rows."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    from oracle import oracle as O
    D, R, B, BUDGET = 262144, 64, 2048, int(120e9)
    X = torch.from_numpy(W.random_state(D, R, seed=2)).cuda()
    Y = torch.empty_like(X)
    rows = np.unique(np.concatenate([np.linspace(0, D - 1, 1020).astype(np.int64),
                                     np.array([2047, 2048, 63488, 212992], dtype=np.int64)]))
    out = {"workload": "Philox GUE D=262144 (seed 1), 64 vectors (seed 2), block 2048, 120 GB partial cache"}
    res = {}
    for name, prec in (("bf16x2", mf.MF_PREC_BF16X2), ("fp32", mf.MF_PREC_FP32)):
        t0 = time.perf_counter()
        plan = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=B, cache_budget_bytes=BUDGET, precision=prec,
                       storage=mf.MF_STORE_PARTIAL, nvec_hint=R, stream=stream, cheb_tol=1e-12)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        desc = plan.describe()
        plan.apply(Y, X, R)
        plan.profile(True)
        reps = 3 if name == "bf16x2" else 1
        t = events_time(lambda: plan.apply(Y, X, R), reps)
        kern_ms, kern_n = plan.profile_read()
        plan.profile(False)
        plan.sync()
        r = {"apply_s": t, "entries_per_s": float(D) * D * R / t, "kernel_ms": kern_ms / max(1, kern_n),
             "create_s": t_create, "pairs_cached": desc["pairs_cached"], "walk": desc.get("tc_walk")}
        r["_rows"] = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
        if name == "bf16x2":
            nt = plan.cheb_terms(1.0)
            psi = X.clone()
            t_step = events_time(lambda: plan.cheb_propagate(psi, R, 1.0, 0), 1)
            plan.sync()
            r.update({"cheb_terms": nt, "cheb_step_s": t_step, "cheb_steps_per_s": 1.0 / t_step,
                      "cheb_terms_per_s": (nt - 1) / t_step})
            del psi
        res[name] = r
        plan.close()
        torch.cuda.empty_cache()
    Xh = X.cpu().numpy()
    del X, Y
    torch.cuda.empty_cache()
    op64 = O.make_op(O.GEN_PHILOX_GUE, D, seed=1)
    t0 = time.perf_counter()
    ref = O.apply_rows(op64, Xh, rows)
    t_cpu = time.perf_counter() - t0
    scale = np.max(np.abs(ref))
    for name in res:
        res[name]["err_vs_fp64_form"] = float(np.max(np.abs(res[name].pop("_rows") - ref)) / scale)
    # composite bound of the BF16X2 product (Sec. IV.B runtime model with
    # measured rates): tensor work, cached bytes, generation
    npair, pc = 8256, res["bf16x2"]["pairs_cached"]
    canon = D * (D + 1) / 2.0
    cached = pc * float(B) * B
    t_tc = 24.0 * R * D * D / (peaks["bf16_tflops_sustained"] * 1e12)
    t_hbm = 8.0 * cached / (peaks["hbm_gbs"] * 1e9)
    # generation: the procedural canonical entries at the per-pipe bound of
    # the generator (the contraction runs on the tensor cores, so no FP32
    # apply FMAs are counted)
    gen = pipe_bound(rates, apply_ffma_per_entry=0)
    t_gen = (canon - cached) * gen["t_bound"]
    bound = max(t_tc, t_hbm, t_gen)
    tb = res["bf16x2"]["kernel_ms"] / 1e3
    # the instruction-shape bound: the Hermitian walk issues N = 2 x 64 = 128
    # MMAs (M = 128, K = 16): per off-diagonal 128 x 128 tile 8 K steps x 6
    # split products for H and as many for H^dagger (96), per diagonal tile
    # 48, at the measured N = 128 instruction rate
    T = D // 128
    n_mma = 96.0 * (T * (T + 1) / 2 - T) + 48.0 * T
    t_tc_shape = n_mma / rates["mma128"] if rates.get("mma128") else None
    out.update(res)
    out["roofline"] = {
        "bound": {t_tc: "tensor", t_hbm: "hbm", t_gen: "generation"}[bound], "t_bound_s": bound,
        "t_tensor_s": t_tc, "t_hbm_s": t_hbm, "t_generation_s": t_gen, "achieved_s": tb, "frac": bound / tb,
        "tensor_tflops": 24.0 * R * D * D / tb / 1e12, "peak_tensor_tflops": peaks["bf16_tflops_sustained"],
        "peak_source": peaks["source"],
        "generation_bound_pipe": gen["bound_pipe"],
        "t_tensor_shape_s": t_tc_shape,
        "frac_of_shape_bound": (max(t_tc_shape, t_hbm, t_gen) / tb) if t_tc_shape else None,
        "shape_note": "one tcgen05.mma M=128 K=16 instruction takes the same time at N=128 as at N=256 "
                      "(mf_pipe_rates), so the 64-vector product (N=128) can reach at most half of the dense "
                      "BF16 rate; t_tensor_shape_s is its MMA instructions at the measured N=128 rate",
        "basis": "tensor: 3 bf16 products x 8 real FLOP x 64 vectors x D^2 at the sustained BF16 peak; hbm: the "
                 "cached canonical entries (8 B each) at the measured copy rate; generation: the procedural "
                 "canonical entries at the slowest pipe's measured rate (operations of the FP32 Philox "
                 "definition per entry, mf_pipe_rates)"}
    out["speedup_bf16x2_vs_fp32"] = res["fp32"]["apply_s"] / res["bf16x2"]["apply_s"]
    out["cpu_baseline"] = {"value": len(rows) * float(D) * R / t_cpu, "unit": "entries/s", "cores": cpu_threads(),
                           "kind": "oracle", "sample": "%d of %d output rows of one FP64 H X with 64 vectors "
                                                      "(%.1f s), rate extrapolated to all rows" % (len(rows), D, t_cpu)}
    return out


def sub_planner():
    """The planner comparison of Algorithms 1-3 on the GB300 sweep records
    shipped with the package (475 problems, 4275 candidate plans measured
    with the current kernels, scored by the library's Algorithm 1): the
    held-out regret (seed-0 split by problem) of the analytic ranking and of
    the direct and residual surrogates, trained here on the GPU (3000 Adam
    epochs each).  CPU baseline: the oracle's FP64 training of the same
    network, epochs per second over 50 epochs."""
    import math
    from oracle import mlp_oracle as MO
    from paper_2606_31598_gb300 import planner_sweep as ps
    recs = ps.load(ps.RECORDS_GB300)
    t0 = time.perf_counter()
    res = ps.evaluate(recs, epochs=3000)
    t_fit = time.perf_counter() - t0
    train, _ = ps.split(recs, 0.2, 0)
    X = ps.surrogate_inputs(train).astype(np.float64)
    Y = np.zeros((len(train), 3))
    M = np.zeros((len(train), 3))
    for i, r in enumerate(train):
        k = ps.STRATEGIES.index(r["storage"])
        Y[i, k] = math.log(r["t_mv"])
        M[i, k] = 1.0
    F, H, O = X.shape[1], 64, 3
    rng = np.random.default_rng(0)
    p0 = np.concatenate([rng.standard_normal(F * H) / np.sqrt(F), np.zeros(H), rng.standard_normal(H * H) / np.sqrt(H),
                         np.zeros(H), rng.standard_normal(H * O) / np.sqrt(H), np.zeros(O)])
    mu, sd = MO.zscore(X)
    t0 = time.perf_counter()
    MO.train_adam(p0, mu, sd, X, Y, M, F, H, O, epochs=50, lr=3e-3)
    t_cpu = time.perf_counter() - t0
    return {"workload": "planner sweep records (GB300, current kernels): %d problems, %d candidate plans; seed-0 "
                        "80/20 split by problem" % (len({r["problem"] for r in recs}), len(recs)),
            "held_out_regret": {"analytic": res["analytic_test"], "learned_direct": res["learned_test"],
                                "learned_residual": res["residual_test"],
                                "no_planner_procedural_b2048": res["fixed_procedural_test"],
                                "no_planner_max_cache_b2048": res["fixed_max_cache_test"]},
            "train_regret": {"analytic": res["analytic_train"], "learned_direct": res["learned_train"],
                             "learned_residual": res["residual_train"]},
            "score_drift": res["score_drift"],
            "fit_s_two_surrogates": t_fit, "gpu_epochs_per_s": 2 * 3000 / t_fit,
            "cpu_baseline": {"value": 50 / t_cpu, "unit": "epochs/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": "50 FP64 Adam epochs of the direct surrogate on the training records "
                                       "(%.2f s)" % t_cpu}}


def sub_batch(stream, rates=None):
    """256 batched Philox problems (the workload draw: D log-uniform in
    [1024, 32768] rounded to 128, 1..16 vectors, seeds 0..255), plans chosen
    per problem by the measured autotuner, FP32 form, one persistent launch
    per Chebyshev term under a captured CUDA graph; one step of dt = 1.  The
    error is problem 0's step against the oracle (same bounds and terms); the
    CPU baseline is the oracle's FP64 product of the first 8 problems."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    from oracle import oracle as O
    probs = W.batch_problems(256)
    Ds = [p[0] for p in probs]
    nv = [p[1] for p in probs]
    seeds = [p[2] for p in probs]
    t0 = time.perf_counter()
    b = mf.Batch(Ds, nv, seeds, mf.MF_GEN_PHILOX_GUE, cache_budget_bytes=int(200e9), precision=mf.MF_PREC_FP32,
                 planner_mode=mf.MF_PLANNER_AUTOTUNE, autotune_k=4, autotune_repeats=2, stream=stream)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    parts = [W.random_state(D, k, seed=100 + i).reshape(D, k) for i, (D, k) in enumerate(zip(Ds, nv))]
    host = torch.from_numpy(np.concatenate([q.ravel() for q in parts]))
    packed = host.cuda()
    nt = b.propagate(packed, 1.0, 1)  # captures the graph for this buffer; later calls replay it
    torch.cuda.synchronize()
    t = events_time(lambda: b.propagate(packed, 1.0, 1), 3)
    packed.copy_(host)
    b.propagate(packed, 1.0, 1)
    torch.cuda.synchronize()
    got0 = packed[int(b.offsets[0]):int(b.offsets[1])].cpu().numpy().reshape(Ds[0], nv[0])
    NCPU = 4  # problems of the CPU baseline (their bounds, before the batch is closed)
    bounds = [mf.mf_spectral_bounds(b.plan(i)) for i in range(NCPU)]
    entries = float(sum(D * D * k for D, k in zip(Ds, nv)))
    hbm_bytes = hbm_bytes_once = gen_entries = flops = 0.0
    n_herm = 0
    stores = {}
    for i, (D, k) in enumerate(zip(Ds, nv)):
        d = mf.mf_plan_describe(b.plan(i))
        stores[d["storage"]] = stores.get(d["storage"], 0) + 1
        cached = min(float(D) * D, 2.0 * d["pairs_cached"] * d["block"] ** 2)
        herm = b.hermitian(i)
        n_herm += herm
        hbm_bytes += (4.0 if herm else 8.0) * cached
        hbm_bytes_once += 4.0 * cached
        gen_entries += (0.5 if herm else 1.0) * (float(D) * D - cached)
        flops += 8.0 * D * D * k
    n_items, grid = b.info()
    b.close()
    # CPU baseline: the oracle's Chebyshev step (FP32 form, the batch's
    # bounds and term count) of the first problems; problem 0's result is
    # also the error reference
    applies = nt - 1
    t0 = time.perf_counter()
    cpu_entries = 0.0
    for i in range(NCPU):
        lo, hi = bounds[i]
        ref = O.cheb_step(O.make_op(O.GEN_PHILOX_GUE, Ds[i], seed=seeds[i], form=O.FORM_FP32), parts[i], 1.0,
                          0.5 * (hi + lo), 0.5 * (hi - lo), nt)
        if i == 0:
            ref0 = ref
        cpu_entries += float(applies) * Ds[i] * Ds[i] * nv[i]
    t_cpu = time.perf_counter() - t0
    return {"workload": "256 batched Philox problems, D in [1024, 32768], 1-16 vectors, FP32, autotuned plans",
            "create_s": t_create, "terms_per_step": nt, "step_s": t, "steps_per_s": 1.0 / t,
            "entries_per_s": entries * applies / t, "sum_D2_nvec": entries, "work_items": n_items,
            "persistent_grid": grid, "storage_chosen": stores, "hermitian_reuse_problems": n_herm,
            "error": {"problem0_step_abs_vs_oracle": float(np.max(np.abs(got0 - ref0))),
                      "measure": "FP32 form against the oracle's statement of the same form, same bounds/terms"},
            "roofline": batch_roofline(hbm_bytes, gen_entries, flops, t / applies, rates, hbm_bytes_once),
            "cpu_baseline": {"value": cpu_entries / t_cpu, "unit": "entries/s", "cores": cpu_threads(),
                             "kind": "oracle", "sample": "the FP32-form Chebyshev step of the first %d problems "
                                                        "(%.1f s)" % (NCPU, t_cpu)}}


def time_applies(plan, x, y, nvec, reps):
    """Mean seconds of one apply (CUDA events on the current stream)."""
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    plan.apply(y, x, nvec)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        plan.apply(y, x, nvec)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def run_dvrmv(args):
    """Sinc-DVR D = 131072, FP32 form, procedural, 1..16 vectors: the
    one-vector row-split kernel and the multi-vector window kernel (vector
    buckets 2, 4, 8, 16).  Algorithmic work 4 FLOP per kinetic entry and
    vector (real entry times complex x); peak 152 SMs x 128 FMA lanes x 2 x
    the SM clock sampled during the run."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    D = 131072
    stream = torch.cuda.current_stream().cuda_stream
    props = torch.cuda.get_device_properties(0)
    out = {"workload": "sinc-DVR D=%d, FP32 form, procedural, several vectors" % D}
    nvecs = [args.dvrmv_nvec] if args.dvrmv_nvec else [1, 2, 4, 8, 16]
    t1 = None
    for nv in nvecs:
        plan = mf.Plan(D, mf.MF_GEN_SINC_DVR_HO, seed=1, precision=mf.MF_PREC_FP32, nvec_hint=nv, stream=stream)
        x = torch.from_numpy(W.random_state(D, nv, seed=4)).cuda()
        y = torch.empty_like(x)
        clock = ClockSampler(0)
        clock.start()
        plan.profile(True)
        t = time_applies(plan, x, y, nv, max(1, args.steps))
        kern_ms, kern_n = plan.profile_read()
        clk = clock.stop()
        plan.profile(False)
        per = kern_ms / 1e3 / max(1, kern_n)
        mhz = clk.get("sm_mhz") or 2070.0
        peak = props.multi_processor_count * 128 * 2 * mhz * 1e6
        flops = 4.0 * D * D * nv
        if nv == 1:
            t1 = t
        out["nvec_%d" % nv] = {"apply_s": t, "kernel_s": per, "kernel_tflops": flops / per / 1e12,
                               "fp32_fma_peak_tflops": peak / 1e12, "frac": flops / per / peak,
                               "vs_one_vector_products": (nv * t1 / t) if t1 else None, "clocks": clk}
        plan.close()
    print(json.dumps(out))
    return 0


def run_multivector(args):
    """Philox ensemble D = 262144, 64 vectors, block 2048, 120 GB partial
    cache (P_cache = 3576 of 8256 canonical pairs): BF16X2 on tcgen05 against
    the FP32 and FP64 SIMT forms; Chebyshev steps of dt = 1 (order from tol
    1e-12) in the BF16X2 form."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    D, R, B = args.mv_dim, 64, 2048
    nblk = (D + B - 1) // B
    # the same cached fraction of canonical pairs as 120 GB at D = 262144
    # (--mv-cache none: every block generated)
    BUDGET = int(120e9 if D == 262144 else 3576 / 8256 * nblk * (nblk + 1) / 2 * B * B * 8 + 1)
    if args.mv_cache == "none":
        BUDGET = 0
    stream = torch.cuda.current_stream().cuda_stream
    X = torch.from_numpy(W.random_state(D, R, seed=2)).cuda()
    Y = torch.empty_like(X)
    out = {"workload": "Philox GUE D=%d, 64 vectors, block 2048, %.1f GB partial cache" % (D, BUDGET / 1e9)}
    plan = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=B, cache_budget_bytes=BUDGET, precision=mf.MF_PREC_BF16X2,
                   storage=mf.MF_STORE_PARTIAL if BUDGET else mf.MF_STORE_PROCEDURAL, nvec_hint=R, stream=stream,
                   cheb_tol=1e-12, hermitian_reuse=0 if args.mv_rowowner else -1)
    desc = plan.describe()
    t_bf = time_applies(plan, X, Y, R, 3)
    Ybf = Y.clone()
    plan.profile(True)
    psi = X.clone()
    for _ in range(args.warmup):
        plan.cheb_propagate(psi, R, 1.0, 0)
    torch.cuda.synchronize()
    plan.profile_read()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.cheb_propagate(psi, R, 1.0, 0)
    e1.record()
    torch.cuda.synchronize()
    kern_ms, kern_n = plan.profile_read()
    t_steps = e0.elapsed_time(e1) / 1e3
    nterms = plan.cheb_terms(1.0)
    plan.close()
    p32 = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=B, cache_budget_bytes=BUDGET, precision=mf.MF_PREC_FP32,
                  storage=mf.MF_STORE_PARTIAL if BUDGET else mf.MF_STORE_PROCEDURAL, nvec_hint=R, stream=stream)
    t_32 = time_applies(p32, X, Y, R, 1)
    Y32 = Y.clone()
    p32.close()
    entries = float(D) * D * R
    flops_tc = 24.0 * D * D * R  # 3 split products x 8 real FLOP per complex MAC
    out.update({
        "plan": desc, "nterms_per_step": nterms,
        "bf16x2": {"apply_s": t_bf, "entries_per_s": entries / t_bf, "tensor_tflops": flops_tc / t_bf / 1e12,
                   "kernel_ms": kern_ms / max(1, kern_n),
                   "cheb_steps_per_s": args.steps / t_steps, "cheb_terms_per_s": args.steps * (nterms - 1) / t_steps},
        "fp32": {"apply_s": t_32, "entries_per_s": entries / t_32},
        "speedup_bf16x2_vs_fp32": t_32 / t_bf,
        "bf16x2_vs_fp32_rel": float((Ybf - Y32).abs().max() / Y32.abs().max()),
    })
    if args.fp64:
        p64 = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=B, precision=mf.MF_PREC_FP64,
                      storage=mf.MF_STORE_PROCEDURAL, nvec_hint=R, stream=stream)
        t_64 = time_applies(p64, X, Y, R, 1)
        p64.close()
        m = Y.abs().max()
        out["fp64_procedural"] = {"apply_s": t_64, "entries_per_s": entries / t_64}
        out["bf16x2"]["err_vs_fp64_form"] = float((Ybf - Y).abs().max() / m)
        out["fp32"]["err_vs_fp64_form"] = float((Y32 - Y).abs().max() / m)
        out["speedup_bf16x2_vs_fp64_procedural"] = t_64 / t_bf
    print(json.dumps(out))
    return 0


def run_philox(args):
    """Seeded generation and cached streaming: the Philox ensemble at
    D = 131072 (FP32 form), one vector (or --philox-nvec 2), procedural
    (every canonical entry generated once per apply, used for H and
    H^dagger) and fully cached (each canonical entry read once from HBM,
    8 bytes); Chebyshev steps of dt = 1."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    D, nv = args.philox_dim, args.philox_nvec
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.from_numpy(W.random_state(D, nv, seed=3)).cuda()
    y = torch.empty_like(x)
    canon = D * (D + 1) / 2.0
    out = {"workload": "Philox GUE D=%d, %d vector%s, FP32 form" % (D, nv, "s" if nv > 1 else "")}
    props = torch.cuda.get_device_properties(0)
    rates = mf.mf_pipe_rates(0, stream)
    out["pipe_rates"] = rates
    for name, storage, budget in [("procedural", mf.MF_STORE_PROCEDURAL, 0),
                                  ("full_cache", mf.MF_STORE_FULL, int(canon * 8 * 1.02) + (1 << 30))]:
        plan = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=2048, cache_budget_bytes=budget,
                       precision=mf.MF_PREC_FP32, storage=storage, stream=stream, nvec_hint=nv)
        desc = plan.describe()
        clock = ClockSampler(0)
        clock.start()
        plan.profile(True)
        t = time_applies(plan, x, y, nv, args.steps)
        kern_ms, kern_n = plan.profile_read()
        clk = clock.stop()
        plan.profile(False)
        per = kern_ms / 1e3 / max(1, kern_n)
        res = {"apply_s": t, "kernel_s": per, "entries_per_s": D * float(D) * nv / t,
               "canonical_entries_per_s": canon / per,
               "pairs_cached": desc["pairs_cached"], "clocks": clk}
        if storage == mf.MF_STORE_FULL:
            gbs = canon * 8 / per / 1e9
            hbm = measured_peaks()["hbm_gbs"]
            res["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                               "note": "8 B per canonical entry read once per apply; peak of measured copy"}
        else:
            res["roofline"] = pipe_roofline(canon / per, rates, apply_ffma_per_entry=8 * nv)
            mhz = clk.get("sm_mhz") or 2070.0
            issue = props.multi_processor_count * 128 * mhz * 1e6  # thread instructions / s
            if nv == 1:  # the ncu instruction count is the one-vector kernel's
                res["roofline"]["issue_frac"] = canon / per * PHILOX_INSTR_PER_ENTRY / issue
        if name == "procedural":
            nt = plan.cheb_terms(1.0)
            psi = x.clone()
            plan.cheb_propagate(psi, nv, 1.0, 0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(args.steps):
                plan.cheb_propagate(psi, nv, 1.0, 0)
            e1.record()
            torch.cuda.synchronize()
            res["cheb_steps_per_s"] = args.steps / (e0.elapsed_time(e1) / 1e3)
            res["terms_per_step"] = nt
        out[name] = res
        plan.close()
    print(json.dumps(out))
    return 0


# Operations of the definition per canonical entry of the FP32 Philox form,
# by the pipe that executes them (half of one Philox4x32-10 call and one
# complex Gaussian entry; each packed FP32 instruction counts as two FP32
# operations):
#   imad_hi  10: 2 high 32x32 products per round, 10 rounds, per 2 entries
#   imad     10: the 2 low products per round
#   lop3     17: 2 three-input XORs per round (10), the two uniforms' masks
#                (4), exponent and mantissa extraction of the log argument
#                (2), the quadrant index of sin/cos (1)
#   iadd3    11: the key schedule (9 bumps x 2 keys per 2 entries) and the
#                exponent bias and reduction step of the log (2)
#   ffma     46: uniforms (6), log with its division and polynomial (15),
#                -2 log (1), square root with its correction (4), sin/cos
#                reduction and polynomials (17), sigma scaling (3)
#   mufu      2: the reciprocal (division) and reciprocal square root
#   i2f       7: integer-float conversions (4 in the uniforms, the log's
#                exponent, the quadrant's truncation and its float)
# plus, for the product itself, 8 FP32 FMAs per vector (H and H^dagger).
PHILOX_GEN_PIPE_OPS = {"imad_hi": 10, "imad": 10, "lop3": 17, "iadd3": 11, "ffma": 46, "mufu": 2, "i2f": 7}
PHILOX_OPS_PER_ENTRY = sum(PHILOX_GEN_PIPE_OPS.values()) + 8
# Thread instructions per canonical entry of the FP32 Philox generator as ncu
# counted them in the one-vector kernel (generation plus the 8 FMAs).
PHILOX_INSTR_PER_ENTRY = 108


def fp64_roofline(canon, t_launch, rates):
    """Roofline of one FP64-form product launch against the measured FP64
    pipe: the FP64 operations of the definition per canonical entry plus the
    8 apply FMAs, over the DFMA rate of mf_pipe_rates."""
    out = {"bound": "fp64", "achieved_canonical_entries_per_s": canon / t_launch, "kernel_s": t_launch,
           "ops_per_entry": PHILOX64_DFMA_OPS + 8,
           "note": "FP64 Philox-to-Gaussian arithmetic on GB300's FP64 pipe (about 1/75 of the FP32 FMA rate); "
                   "division and square root counted as one operation each, so the bound is a lower one"}
    if rates and rates.get("dfma"):
        t_bound = canon * (PHILOX64_DFMA_OPS + 8) / rates["dfma"]
        out.update({"bound_pipe": "dfma", "t_bound_s": t_bound, "frac": t_bound / t_launch,
                    "peak_dfma_per_s": rates["dfma"]})
    return out


def pipe_bound(rates, apply_ffma_per_entry=8):
    """Per-pipe bound of procedural Philox generation (seconds per canonical
    entry): each pipe's operations per entry over that pipe's measured rate
    (mf_pipe_rates); the bound is the slowest pipe, the sum of all pipes'
    times a pessimistic (no overlap) bound."""
    ops = dict(PHILOX_GEN_PIPE_OPS)
    ops["ffma"] += apply_ffma_per_entry
    t = {k: ops[k] / rates[k] for k in ops}
    worst = max(t, key=t.get)
    return {"ops_per_entry": ops, "s_per_entry": t, "bound_pipe": worst, "t_bound": t[worst],
            "t_sum": sum(t.values())}


def pipe_roofline(canon_per_s, rates, apply_ffma_per_entry=8):
    """Roofline record of a measured canonical-entry rate against the
    per-pipe bound: frac = bound time / measured time per entry (the
    fraction of the slowest pipe's measured peak the kernel keeps busy);
    sum_frac the same against the no-overlap sum."""
    b = pipe_bound(rates, apply_ffma_per_entry)
    t_meas = 1.0 / canon_per_s
    return {"bound": "alu", "bound_pipe": b["bound_pipe"], "frac": b["t_bound"] / t_meas,
            "sum_frac": b["t_sum"] / t_meas,
            "per_pipe_frac": {k: v / t_meas for k, v in b["s_per_entry"].items()},
            "ops_per_entry": b["ops_per_entry"],
            "achieved_canonical_entries_per_s": canon_per_s,
            "peak_canonical_entries_per_s": 1.0 / b["t_bound"],
            "basis": "operations of the FP32 Philox definition per canonical entry by pipe, over the pipe rates "
                     "measured by mf_pipe_rates (register-only chains) in this run"}


def batch_roofline(hbm_bytes, gen_entries, flops, t_apply, rates=None, hbm_bytes_once=None):
    """Lower bounds of one batched product from its three resources, each at
    its measured peak: HBM (the measured copy rate), the FP32 FMA pipe (the
    FFMA rate of mf_pipe_rates, else 152 x 128 lanes x 2070 MHz) and entry
    generation (the generated entries at the slowest generator pipe of
    mf_pipe_rates, else the 1.5e11 entries/s of the Philox row-owner kernel);
    achieved fraction = largest bound / measured time.  hbm_bytes are the
    stored bytes the chosen forms read (a stored pair once in the
    Hermitian-reuse form, twice in the row-owner form); hbm_bytes_once, if
    given, every stored pair read once (the bound of canonical-pair reuse for
    every problem), reported beside it."""
    t_hbm = hbm_bytes / (measured_peaks()["hbm_gbs"] * 1e9)
    if rates and rates.get("ffma"):
        t_fma = flops / (2.0 * rates["ffma"])
        t_gen = gen_entries * pipe_bound(rates, apply_ffma_per_entry=0)["t_bound"]
    else:
        t_fma = flops / (152 * 128 * 2 * 2.07e9)
        t_gen = gen_entries / 1.5e11
    bound = max(t_hbm, t_fma, t_gen)
    name = {t_hbm: "hbm", t_fma: "fma", t_gen: "generation"}[bound]
    out = {"t_apply_s": t_apply, "t_hbm_s": t_hbm, "t_fma_s": t_fma, "t_gen_s": t_gen, "bound": name,
           "frac": bound / t_apply, "sum_of_bounds_frac": (t_hbm + t_fma + t_gen) / t_apply,
           "rates": "measured in this run" if rates else "unit counts"}
    if hbm_bytes_once is not None:
        t_once = hbm_bytes_once / (measured_peaks()["hbm_gbs"] * 1e9)
        out["t_hbm_pairs_once_s"] = t_once
        out["frac_of_pairs_once_bound"] = max(t_once, t_fma, t_gen) / t_apply
    return out


def run_batch(args):
    """256 independent Philox problems (D log-uniform in [1024, 32768] rounded
    to 128, 1..16 vectors, seeds 0..255), plans chosen per problem by the
    measured autotuner with a shared 200 GB cache budget, FP32 form,
    Chebyshev steps of dt = 1: one persistent launch per term under a CUDA
    graph, against the same problems propagated one after another through
    their own plans."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    if args.batch_uniform:
        # uniform problems (D, vectors, count): one vector bucket, for profiling
        D, k, n = (int(v) for v in args.batch_uniform.split(","))
        probs = [(D, k, i) for i in range(n)]
    else:
        probs = W.batch_problems(args.batch_n)
    Ds = [p[0] for p in probs]
    nv = [p[1] for p in probs]
    seeds = [p[2] for p in probs]
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    b = mf.Batch(Ds, nv, seeds, mf.MF_GEN_PHILOX_GUE, cache_budget_bytes=int(args.batch_budget_gb * 1e9),
                 precision=mf.MF_PREC_FP32, planner_mode=mf.MF_PLANNER_AUTOTUNE, autotune_k=4, autotune_repeats=2,
                 stream=stream)
    t_create = time.perf_counter() - t0
    n_items, grid = b.info()
    parts = [W.random_state(D, k, seed=100 + i).reshape(D, k) for i, (D, k) in enumerate(zip(Ds, nv))]
    packed = torch.from_numpy(np.concatenate([q.ravel() for q in parts])).cuda()
    nt = b.propagate(packed, 1.0, args.steps)  # capture the graph once, warm
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    b.propagate(packed, 1.0, args.steps)
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    stores = {}
    entries = 0.0
    hbm_bytes = 0.0       # stored bytes read per product by the chosen forms
    hbm_bytes_once = 0.0  # every stored pair read once
    gen_entries = 0.0     # entries generated per product
    flops = 0.0           # 8 real FLOP per entry and vector
    n_herm = 0
    for i, (D, k) in enumerate(zip(Ds, nv)):
        d = mf.mf_plan_describe(b.plan(i))
        stores[d["storage"]] = stores.get(d["storage"], 0) + 1
        entries += float(D) * D * k
        cached = min(float(D) * D, 2.0 * d["pairs_cached"] * d["block"] ** 2)
        herm = b.hermitian(i)
        n_herm += herm
        hbm_bytes += (4.0 if herm else 8.0) * cached
        hbm_bytes_once += 4.0 * cached
        gen_entries += (0.5 if herm else 1.0) * (float(D) * D - cached)
        flops += 8.0 * D * D * k
    # the same problems one by one through their own plans (same term count;
    # the plans run on the batch's stream, so time with device syncs)
    seq = [torch.from_numpy(q.copy()).cuda() for q in parts]
    for _ in range(args.steps):
        for i, k in enumerate(nv):
            mf.mf_cheb_propagate(b.plan(i), seq[i], k, 1.0, nt)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        for i, k in enumerate(nv):
            mf.mf_cheb_propagate(b.plan(i), seq[i], k, 1.0, nt)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t1
    applies = args.steps * (nt - 1)
    what = ("D = %d, %d vectors each" % (Ds[0], nv[0])) if args.batch_uniform else "D in [1024, 32768], 1-16 vectors"
    out = {"workload": "%d batched Philox problems, %s, FP32" % (len(Ds), what),
           "sum_D2_nvec": entries, "terms_per_step": nt, "create_s": t_create, "work_items": n_items,
           "persistent_grid": grid, "storage_chosen": stores, "hermitian_reuse_problems": n_herm,
           "batched": {"steps_per_s": args.steps / t_batch, "entries_per_s": entries * applies / t_batch},
           "sequential": {"steps_per_s": args.steps / t_seq, "entries_per_s": entries * applies / t_seq},
           "speedup_batched_vs_sequential": t_seq / t_batch,
           "roofline": batch_roofline(hbm_bytes, gen_entries, flops, t_batch / applies, None, hbm_bytes_once),
           "max_diff_batched_vs_sequential": float(max((packed[int(b.offsets[i]):int(b.offsets[i + 1])]
                                                        - seq[i].reshape(-1)).abs().max() for i in range(len(Ds))))}
    print(json.dumps(out))
    b.close()
    return 0


def run_sysbath(args):
    """The system-bath shape of Sec. VII: d_S = 4 (two system qubits),
    d_B = 65536 (16 bath qubits), D = 262144, one interaction term (n_op = 2
    dense bath operators H_B, B_1, Philox-generated on demand, never stored),
    random Hermitian H_S and A_1 (numpy seed 0), g = 1, FP32 form.  Reports
    the time per H psi, entries applied/s (n_op d_B^2 d_S per product), real
    FLOP/s by Eq. generic_matvec_flops (8 n_op d_B^2 d_S), an imaginary-time
    filter of 80 terms (the paper's TPQ order) and the FP32 form's error
    against the FP64 form on one product."""
    import torch
    import paper_2606_31598_gb300 as mf
    d_S, d_B, n_int, g = args.sb_ds, args.sb_db, 1, 1.0
    rng = np.random.default_rng(0)

    def herm(n):
        m = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        return 0.5 * (m + m.conj().T)

    H_S = herm(d_S)
    A = np.stack([herm(d_S) for _ in range(n_int)])
    seeds = [1 + k for k in range(n_int + 1)]
    nop = n_int + 1
    stream = torch.cuda.current_stream().cuda_stream
    X = torch.from_numpy(np.ascontiguousarray(
        (rng.standard_normal((d_B, d_S)) + 1j * rng.standard_normal((d_B, d_S))) / np.sqrt(2.0 * d_B * d_S))).cuda()
    Y = torch.empty_like(X)
    p32 = mf.Plan.sysbath(d_S, d_B, seeds, H_S, A, g, precision=mf.MF_PREC_FP32, stream=stream)
    clock = ClockSampler(0)
    clock.start()
    t_apply = time_applies(p32, X, Y, d_S, args.steps)
    Y32 = Y.clone()
    emin, emax = p32.bounds()
    psi = X.clone()
    p32.cheb_filter(psi, d_S, 0.1, 80, True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    p32.cheb_filter(psi, d_S, 0.1, 80, True)
    e1.record()
    torch.cuda.synchronize()
    t_filter = e0.elapsed_time(e1) / 1e3
    clk = clock.stop()
    p32.close()
    entries = float(nop) * d_B * d_B * d_S
    out = {"workload": "system-bath d_S=%d d_B=%d n_int=%d (D=%d), Philox bath operators, FP32 form"
                       % (d_S, d_B, n_int, d_S * d_B),
           "apply_s": t_apply, "entries_per_s": entries / t_apply, "real_flops_per_s": 8.0 * entries / t_apply,
           "tpq_filter_80_terms_s": t_filter, "bounds": [emin, emax], "clocks": clk,
           "paper_context": "0.104089 s per H psi on 8 L40S GPUs with a full cache (Sec. VII)"}
    if args.fp64:
        p64 = mf.Plan.sysbath(d_S, d_B, seeds, H_S, A, g, precision=mf.MF_PREC_FP64, stream=stream)
        t64 = time_applies(p64, X, Y, d_S, 1)
        p64.close()
        out["fp64"] = {"apply_s": t64, "entries_per_s": entries / t64}
        out["fp32_vs_fp64_form"] = float((Y32 - Y).abs().max() / Y.abs().max())
    print(json.dumps(out))
    return 0


def run_external(args):
    """The storage hierarchy on one operator: the Philox ensemble at D (FP32
    form) written out as externally stored canonical blocks (b = 2048) in host
    memory, applied with all pairs read from host memory over the host link,
    with half of them in the HBM cache, and with all of them in HBM; beside
    it, the same operator generated procedurally.  Host-link bandwidth =
    host-resident block bytes / apply time."""
    import torch
    import paper_2606_31598_gb300 as mf
    import workloads as W
    D, b = args.ext_dim, 2048
    stream = torch.cuda.current_stream().cuda_stream
    nblk = -(-D // b)
    pairs = [(n, m) for n in range(nblk) for m in range(n, nblk)]
    gen = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=b, precision=mf.MF_PREC_FP32,
                  storage=mf.MF_STORE_PROCEDURAL, stream=stream)
    t0 = time.perf_counter()
    blocks = np.zeros((len(pairs), b, b), dtype=np.complex64)
    for k, (n, m) in enumerate(pairs):
        rows, cols = min(b, D - n * b), min(b, D - m * b)
        blocks[k, :rows, :cols] = gen.entries(n * b, m * b, rows, cols)
    t_fill = time.perf_counter() - t0
    x = torch.from_numpy(W.random_state(D, 1, seed=3)).cuda()
    y = torch.empty_like(x)
    out = {"workload": "externally stored blocks: Philox D=%d as %d canonical %dx%d complex64 blocks (%.1f GB) "
                       "in host memory" % (D, len(pairs), b, b, blocks.nbytes / 1e9),
           "fill_s": t_fill}
    t_gen = time_applies(gen, x, y, 1, args.steps)
    y_gen = y.clone()
    out["procedural"] = {"apply_s": t_gen}
    gen.close()
    blk = 8.0 * b * b
    for name, npc in [("host_all", 0), ("host_half", len(pairs) // 2), ("hbm_all", len(pairs))]:
        plan = mf.Plan.external(D, b, blocks, cache_budget_bytes=int(npc * blk), precision=mf.MF_PREC_FP32,
                                stream=stream)
        t = time_applies(plan, x, y, 1, args.steps)
        host_bytes = (len(pairs) - npc) * blk
        res = {"apply_s": t, "pairs_in_hbm": npc, "host_bytes": host_bytes,
               "max_rel_diff_vs_procedural": float((y - y_gen).abs().max() / y_gen.abs().max())}
        if host_bytes > 0:
            res["host_link_gbs"] = host_bytes / t / 1e9
        if npc == len(pairs):
            res["hbm_gbs"] = npc * blk / t / 1e9
        out[name] = res
        plan.close()
    # the host link's copy-engine rate for context: one pinned 2 GB buffer
    h = torch.empty(1 << 28, dtype=torch.complex64).pin_memory()
    dbuf = torch.empty(1 << 28, dtype=torch.complex64, device="cuda")
    dbuf.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        dbuf.copy_(h, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    out["h2d_copy_engine_gbs"] = 3 * h.numel() * 8 / (e0.elapsed_time(e1) / 1e3) / 1e9
    del h, dbuf
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mf", choices=["mf", "reference"])
    ap.add_argument("--batch-n", type=int, default=256, help="batch: number of problems")
    ap.add_argument("--batch-uniform", default="", help="batch: 'D,nvec,count' uniform problems instead of the draw")
    ap.add_argument("--philox-dim", type=int, default=131072, help="philox: D")
    ap.add_argument("--philox-nvec", type=int, default=1, choices=[1, 2], help="philox: vectors")
    ap.add_argument("--batch-budget-gb", type=float, default=200.0, help="batch: shared cache budget")
    ap.add_argument("--sb-ds", type=int, default=4, help="sysbath: system dimension d_S")
    ap.add_argument("--sb-db", type=int, default=65536, help="sysbath: bath dimension d_B")
    ap.add_argument("--ext-dim", type=int, default=65536, help="external: D")
    ap.add_argument("--workload", default="dvr",
                    choices=["dvr", "dvrmv", "multivector", "batch", "philox", "sysbath", "external"],
                    help="dvr: the benchmark line; dvrmv: the DVR product for 1..16 vectors; "
                         "multivector: the 64-vector tensor-core workload report")
    ap.add_argument("--dvrmv-nvec", type=int, default=0, help="dvrmv: one vector count only (0: 1, 2, 4, 8, 16)")
    ap.add_argument("--fp64", action="store_true", help="multivector: also time the FP64 procedural form")
    ap.add_argument("--mv-cache", default="partial", choices=["partial", "none"],
                    help="multivector: the 120 GB-share partial cache, or every block generated")
    ap.add_argument("--mv-rowowner", action="store_true",
                    help="multivector: the row-owner tcgen05 kernel (hermitian_reuse = 0) for the BF16X2 form")
    ap.add_argument("--mv-dim", type=int, default=262144, help="multivector: D (smaller D keeps the cached fraction)")
    ap.add_argument("--headline-only", action="store_true",
                    help="dvr: the headline line alone, without the other configurations' sub-results")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "dvrmv":
        return run_dvrmv(args)
    if args.workload == "multivector":
        return run_multivector(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "philox":
        return run_philox(args)
    if args.workload == "sysbath":
        return run_sysbath(args)
    if args.workload == "external":
        return run_external(args)
    return run_mf(args)


if __name__ == "__main__":
    sys.exit(main())
