#!/usr/bin/env python3
"""Throughput of the cut-cell MAC projection step on GB300, in MAC cell-steps/s.

Workload (one GPU): the 1024x512 Re 100 cylinder on [-4,12]x[-4,4] in FP64 with the seeded
N(0, 1e-3) velocity perturbation, Jacobi-PCG to 1e-10 (the configuration the metric is
quoted on); each Poisson solve starts from the projection of its solution onto the last 32
solutions (--guess-history; 0 starts from the previous Phi, as the oracle does), and stops
at the same relative residual.  A "step" is one whole PmII projection step (predictor with
AB2 convection and Crank-Nicolson viscosity, Helmholtz PCG, divergence, Poisson PCG,
projection and pressure update) over the case.  The state is device resident; L2 is flushed (256 MiB write)
between timed steps, outside each step's CUDA-event interval.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank advances its own replica of the case
(the case is not split: replicas only) and ``value`` is the sum over ranks.
``--impl reference`` times the FP64 CPU oracle on this machine's host cores: whole steps of
the same workload's trajectory, the same warm-up and timed step counts.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MAC cell-steps/s single & batched; HBM GB/s frac; p50/p99 solve latency"
UNIT = "cell-steps/s"
WORKLOAD = "cylinder_re100_1024x512"

# Algorithmic cost of one Jacobi-PCG iteration per cell (FP64): K p (4 differences, 4
# products, 3 sums), p.q, x += a p, r -= a q, z = D^-1 r, r.z, r.r, p = z + b p.
PCG_FLOPS_PER_CELL_ITER = 24
# x, r and p each read and written once per iteration (8-byte words).
PCG_BYTES_PER_CELL_ITER = 48
# Solutions kept for the projected initial guess of the Poisson solves (the largest basis the
# library takes; 24 and 32 were both about 3 % faster than 16 on the headline workload).
GUESS_L = 32
# FP64 peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA/clock x 2 flop x
# 2.07 GHz; reported beside the rate ccm_measure_fp64_rate measures, which is the denominator.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-full", action="store_true",
                    help="also time one whole headline step of the oracle on one thread")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the measurements that follow the headline")
    ap.add_argument("--extras", default="mixed,configs,batched,serving",
                    help="comma-separated subset of the measurements that follow the headline")
    ap.add_argument("--launch-plan", default="",
                    help="headline case: this launch shape instead of the set-up autotuner's (the seven "
                         "comma-separated values of ccm_launch_plan), e.g. for a profiler run")
    ap.add_argument("--configs", default="",
                    help="comma-separated names of the single-case configurations to run (default: all)")
    ap.add_argument("--guess-history", type=int, default=GUESS_L,
                    help="headline case: initial guess of each Poisson solve by projection onto the last L "
                         "solutions (0: the previous Phi); the stopping test is the same")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="headline case's precision (the configuration is FP64; mixed for profiling the "
                         "mixed-precision kernels on the same workload)")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "chebyshev"])
    ap.add_argument("--cheb-degree", type=int, default=3)
    ap.add_argument("--batch-cases", type=int, default=64,
                    help="cases of the batched measurement (the first N of the seeded 64-case mix)")
    ap.add_argument("--serving-window", default="32,100",
                    help="NREQ,DIV: the serving measurement takes the first NREQ requests of the "
                         "stream with their step counts divided by DIV")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_time_ms(t_ms, world, device="cuda"):
    """Length of the timed region for the whole job: every rank's own total (ms), reduced with
    MAX over the ranks (the slowest replica sets the job's time)."""
    if world <= 1:
        return t_ms
    import torch

    t = torch.tensor([t_ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, cells, steps, t_ms):
    """Whole-job throughput in cell-steps/s: the cells every replica advanced, over the slowest
    replica's time (replicas: no data moves between ranks)."""
    return world * cells * steps / (t_ms * 1e-3)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


# The FP64 Poisson CG on the Jacobi-scaled system takes one of three launch shapes, chosen by the
# set-up autotuner: tiles with one barrier per iteration, their vectors in global memory (f1) or
# resident in shared memory (f2), or, on small grids, one thread-block cluster.
KERNEL_SOURCES = {
    "k_pcg_poisson_m1": ("ccm_internal.cuh", "pcg_common.cuh", "pcg_cheb.cuh", "pcg_mixed1.cu"),
    "k_pcg_poisson_m2": ("ccm_internal.cuh", "pcg_common.cuh", "pcg_cheb.cuh", "pcg_mixed1.cu"),
    "k_pcg_poisson_mixed": ("ccm_internal.cuh", "pcg_common.cuh", "pcg_cheb.cuh", "pcg_quad.cuh", "pcg_mixed.cu"),
    "k_pcg_poisson_f1": ("ccm_internal.cuh", "pcg_common.cuh", "pcg_fixed.cuh", "pcg_fused.cu"),
    "k_pcg_poisson_f2": ("ccm_internal.cuh", "pcg_common.cuh", "pcg_fixed.cuh", "pcg_fused.cu"),
    "k_pcg_poisson_cluster": ("pcg_common.cuh", "pcg_cluster.cu"),
}


def kernel_of(plan):
    """The Poisson kernel a launch plan (bench's _plan_dict) runs."""
    if plan.get("kind") == "cluster":
        return "k_pcg_poisson_cluster"
    if plan.get("kind") == "tiles, one barrier per iteration":
        return "k_pcg_poisson_m2" if plan.get("resident") else "k_pcg_poisson_m1"
    if plan.get("kind") in ("blocks", "built-in") and plan.get("precision") == "mixed":
        return "k_pcg_poisson_mixed"
    return "k_pcg_poisson_f2" if plan.get("resident") else "k_pcg_poisson_f1"


def kernel_source_hash(kernel="k_pcg_poisson_f2"):
    import hashlib

    csrc = os.path.join(ROOT, "paper_2211_10698_gb300", "csrc")
    return hashlib.sha256(b"".join(open(os.path.join(csrc, f), "rb").read()
                                   for f in KERNEL_SOURCES[kernel])).hexdigest()[:16]


def _traffic_from_profile(kernel="k_pcg_poisson_f2"):
    """DRAM bytes per launch of the Poisson PCG from the committed ncu summary, if it covers
    this kernel and the kernel source still matches the hash recorded with the counters."""
    path = os.path.join(ROOT, "profiles", "pcg_poisson_fp64_cylinder.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    vals = {}
    for line in text.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel") != kernel or vals.get("kernel source sha256") != kernel_source_hash(kernel):
        return None, None
    try:
        return float(vals["dram bytes per iteration per cell"]), vals
    except (KeyError, ValueError):
        return None, None


class Clocks:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
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
        rows = []
        with open(self.f.name) as fh:
            for r in csv.reader(fh):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def oracle_steps(case, steps, threads, warmup=0):
    """Whole steps of the FP64 oracle on this machine's cores: the seeded initial state (with
    the case's velocity perturbation), ``warmup`` untimed steps, then ``steps`` steps each timed
    on the wall clock.  Every solve runs to the case's tolerance (nothing is capped).  Returns
    the thread count used, the seconds and the Poisson iterations of each timed step."""
    import oracle
    from paper_2211_10698_gb300 import inputs

    used = oracle.set_threads(threads)
    o = oracle.Oracle(case)
    pu, pv = inputs.perturbation(case)
    st = o.init_state(pu, pv)
    if warmup:
        o.step(st, warmup)
    secs, iters = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        hist, _ = o.step(st, 1)
        secs.append(time.perf_counter() - t0)
        iters.append(hist[0]["iters_p"])
    return dict(threads=used, seconds=secs, iters_p=iters)


FIELDS = (("u", 0), ("v", 1), ("p", 2))  # ccm.CCM_F_U, CCM_F_V, CCM_F_P


def gpu_state(g):
    """A case's whole state (U, V, P, Phi, conv^{n-1}, step count) in the oracle's layout."""
    from paper_2211_10698_gb300 import ccm

    get = g.get_field
    return dict(u=get(ccm.CCM_F_U).copy(), v=get(ccm.CCM_F_V).copy(), p=get(ccm.CCM_F_P).copy(),
                phi=get(ccm.CCM_F_PHI).copy(), cu=get(ccm.CCM_F_CONV_U).copy(), cv=get(ccm.CCM_F_CONV_V).copy(),
                n=int(get(ccm.CCM_F_STEP)[0, 0]))


def gpu_next_step(g):
    """The state, one more step of the case on the GPU (its own settings) and that step's u, v, P."""
    state = gpu_state(g)
    g.step(1)
    return state, {name: g.get_field(f).copy() for name, f in FIELDS}


def oracle_step_from(case, state, threads):
    """One whole oracle step from a given state, timed; returns the timing record and u, v, P."""
    import numpy as np

    import oracle

    used = oracle.set_threads(threads)
    o = oracle.Oracle(case)
    st = {k: (np.array(v, dtype=np.float64, order="C") if isinstance(v, np.ndarray) else v) for k, v in state.items()}
    t0 = time.perf_counter()
    hist, _ = o.step(st, 1)
    sec = time.perf_counter() - t0
    return dict(threads=used, seconds=[sec], iters_p=[hist[0]["iters_p"]]), {name: st[name] for name, _ in FIELDS}


def _rel_errors(got, want):
    import numpy as np

    return {name: float(np.linalg.norm(got[name] - want[name]) / max(np.linalg.norm(want[name]), 1e-300))
            for name, _ in FIELDS}


def _window_summary(case, w):
    t = sum(w["seconds"])
    return dict(cells=case.cells, steps=len(w["seconds"]), threads=w["threads"], seconds=t,
                value=case.cells * len(w["seconds"]) / t, unit=UNIT,
                poisson_iters_per_step=sum(w["iters_p"]) / len(w["iters_p"]))


def cpu_baseline(case, head_next, c3_next=None, full=False):
    """The FP64 oracle timed on this machine's cores, whole steps only, each solve to its
    configured tolerance:
    - the headline workload: one whole step from the GPU run's state after its timed steps, on
      all cores (the value); the GPU's own step from the same state gives the error of each
      field against the oracle;
    - the 2048x1024 airfoil (``c3_next``): likewise one step from the GPU's state after its
      timed window, the GPU step in mixed precision;
    - the 128x64 Re 40 cylinder: all 100 steps from the seeded start, on all cores and on one
      thread;
    - with ``full``, also a headline step on one thread (a minute or more)."""
    from paper_2211_10698_gb300 import inputs

    nproc = os.cpu_count()
    state, gnext = head_next
    w, onext = oracle_step_from(case, state, 0)
    windows = {f"{WORKLOAD} all cores": dict(_window_summary(case, w), from_step=state["n"])}
    parity = {WORKLOAD: dict(step=state["n"] + 1, precision="fp64", rel_l2=_rel_errors(gnext, onext))}
    if c3_next is not None:
        c3case, c3state, c3gpu = c3_next
        w3, o3 = oracle_step_from(c3case, c3state, 0)
        windows[f"{c3case.name} all cores"] = dict(_window_summary(c3case, w3), from_step=c3state["n"])
        parity[c3case.name] = dict(step=c3state["n"] + 1, precision="mixed on the GPU, FP64 oracle",
                                   rel_l2=_rel_errors(c3gpu, o3))
    c1 = inputs.cylinder_re40_128x64()
    windows[f"{c1.name} all cores"] = _window_summary(c1, oracle_steps(c1, c1.steps, 0))
    windows[f"{c1.name} 1 thread"] = _window_summary(c1, oracle_steps(c1, c1.steps, 1))
    if full:
        w1, _ = oracle_step_from(case, state, 1)
        windows[f"{WORKLOAD} 1 thread"] = dict(_window_summary(case, w1), from_step=state["n"])
    h = windows[f"{WORKLOAD} all cores"]
    return dict(value=h["value"], unit=UNIT, cores=h["threads"], kind="oracle",
                sample=(f"{WORKLOAD}: one whole oracle step from the GPU run's state at step {state['n']} (every "
                        f"solve to its 1e-10 tolerance, {h['poisson_iters_per_step']:.0f} Poisson iterations) on "
                        f"{h['threads']} threads, {h['seconds']:.1f} s"),
                nproc=nproc, cpu_model=_cpu_model(), windows=windows,
                parity=dict(note="relative L2 error of the GPU's step against the oracle's step from the same "
                                 "state, both at the configured tolerances", **parity))


def run_reference(args):
    """The FP64 CPU oracle as the reference arm: the headline workload's own trajectory
    (seeded initial state, ``warmup`` untimed whole steps, then ``steps`` whole steps each
    timed), on all of this machine's cores.  Rank 0 alone runs it."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_2211_10698_gb300 import inputs

    case = inputs.cylinder_re100_1024x512()
    w = oracle_steps(case, args.steps, 0, warmup=args.warmup)
    secs = sum(w["seconds"])
    value = case.cells * args.steps / secs
    iters = sum(w["iters_p"]) / len(w["iters_p"])
    sample = (f"{WORKLOAD}: steps {args.warmup + 1}..{args.warmup + args.steps} of the seeded run after "
              f"{args.warmup} untimed steps, whole oracle steps (every solve to its 1e-10 tolerance, "
              f"{iters:.0f} Poisson iterations per step) on {w['threads']} threads")
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * secs / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD, nx=case.nx, ny=case.ny, cells=case.cells, precision="fp64",
                            precond="jacobi", tol_p=case.tol_p, tol_h=case.tol_h,
                            poisson_iters_per_step=iters),
                cpu_baseline=dict(value=value, unit=UNIT, cores=w["threads"], kind="oracle", sample=sample,
                                  nproc=os.cpu_count(), cpu_model=_cpu_model()),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def _timed_steps(torch, stream, step_fn, steps, flush):
    """CUDA-event time of `steps` calls of step_fn, L2 flushed between calls (untimed)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        step_fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def measure_variant(torch, stream, flush, precision="mixed", precond="jacobi", degree=3, guess=0, steps=20,
                    warmup=5):
    """The headline workload with another solver setting at the same accuracy target (every
    Poisson solve to a relative residual of 1e-10): the mixed-precision solve (FP32 CG with
    FP64 residual replacements), the Chebyshev preconditioner, or the projected initial guess.
    Its fields after the steps are compared with the plain FP64 Jacobi path's."""
    import numpy as np

    from paper_2211_10698_gb300 import ccm, inputs

    case = inputs.cylinder_re100_1024x512()
    case.precision, case.precond, case.cheb_degree, case.guess_history = precision, precond, degree, guess
    g = ccm.Case(case, stream=stream.cuda_stream, allocator=ccm.TorchAllocator())
    pu, pv = inputs.perturbation(case)
    g.set_field(ccm.CCM_F_U, g.get_field(ccm.CCM_F_U) + pu)
    g.set_field(ccm.CCM_F_V, g.get_field(ccm.CCM_F_V) + pv)
    g.step(warmup)
    g.enable_kernel_timing(True)
    ms = _timed_steps(torch, stream, lambda: g.step_async(1), steps, flush)
    st = g.read_stats()
    kt = g.kernel_timing()
    plan = _plan_dict(g, precision)
    fields = [g.get_field(f) for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P)]
    g.close()
    ref_case = inputs.cylinder_re100_1024x512()
    ref = ccm.Case(ref_case, stream=stream.cuda_stream, allocator=ccm.TorchAllocator())
    ref.set_field(ccm.CCM_F_U, ref.get_field(ccm.CCM_F_U) + pu)
    ref.set_field(ccm.CCM_F_V, ref.get_field(ccm.CCM_F_V) + pv)
    ref.step(warmup + steps)
    err = {}
    for name, f, a in zip(("u", "v", "p"), (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P), fields):
        b = ref.get_field(f)
        err[name] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    ref.close()
    t = sum(ms)
    desc = ("mixed (FP32 CG on the Jacobi-scaled system, FP64 residual replacements to 1e-10)"
            if precision == "mixed" else "fp64")
    return dict(workload=WORKLOAD, precision=desc,
                precond=precond + (f" degree {degree}" if precond == "chebyshev" else ""),
                initial_guess=(f"projection onto the last {guess} solutions" if guess else "previous Phi"),
                value=case.cells * steps / (t * 1e-3), unit=UNIT, ms_per_step=t / steps, steps=steps,
                poisson_iters_per_step=st["iters_p"] / steps, final_rel_res=st["last_res_p"],
                poisson_ms_per_step=kt["poisson_ms"] / steps,
                us_per_iteration=1e3 * kt["poisson_ms"] / max(kt["poisson_iters"], 1),
                max_div=st["max_div"], converged=bool(st["converged"]), launch_plan=plan,
                rel_l2_vs_plain_fp64_path=err)


def _measure_case(torch, stream, flush, case, steps, warmup, precision=None, precond=None, keep=None):
    """Steps of one case timed with CUDA events; with ``keep`` (a dict), keep["next"] receives
    the state after the timed steps and the GPU's next step from it."""
    from paper_2211_10698_gb300 import ccm

    g = ccm.Case(case, precision=precision, precond=precond, stream=stream.cuda_stream,
                 allocator=ccm.TorchAllocator())
    g.step(warmup)
    g.read_stats()
    ms = _timed_steps(torch, stream, lambda: g.step_async(1), steps, flush)
    st = g.read_stats(allow_not_converged=True)
    plan = _plan_dict(g, precision or case.precision)
    if keep is not None:
        keep["next"] = gpu_next_step(g)
    g.close()
    t = sum(ms)
    return dict(value=case.cells * steps / (t * 1e-3), unit=UNIT, ms_per_step=t / steps, steps=steps,
                poisson_iters_per_step=st["iters_p"] / steps, helmholtz_iters_per_step=st["iters_h"] / steps,
                last_rel_res_p=st["last_res_p"], converged=bool(st["converged"]), launch_plan=plan)


def _plan_dict(g, precision="fp64"):
    """The launch shape the set-up autotuner chose for the case's Poisson solve (a mixed case's
    tiles are those of the solve with one barrier per iteration)."""
    tx, ty, nbx, ntiles, mb, cl, res = g.launch_plan()
    if cl:
        return dict(kind="cluster", ctas=cl)
    if tx and precision == "mixed":
        return dict(kind="tiles, one barrier per iteration", tile=[tx, ty], tiles=ntiles, resident=bool(res))
    if tx:
        return dict(kind="tiles", tile=[tx, ty], tiles=ntiles, resident=bool(res))
    if mb:
        return dict(kind="blocks", blocks=mb, precision=precision)
    return dict(kind="built-in", precision=precision)


def measure_configs(torch, stream, flush, only=None, keep=None):
    """The other single-case configurations: the 128x64 cylinder at Re 40 (FP64), and the
    2048x1024 NACA0012 at Re 1000 in the mixed setting, with its configured Chebyshev
    preconditioner and with Jacobi (both one-launch solves).  `only`: names to run."""
    from paper_2211_10698_gb300 import inputs

    def want(name):
        return not only or name in only

    out = {}
    if want("cylinder_re40_128x64"):
        c1 = inputs.cylinder_re40_128x64()
        out["cylinder_re40_128x64"] = dict(precision="fp64", **_measure_case(torch, stream, flush, c1, 20, 3))
    c3 = inputs.naca0012_re1000_2048x1024()
    if want("naca0012_re1000_2048x1024"):
        out["naca0012_re1000_2048x1024"] = dict(
            precision="mixed", precond=f"chebyshev degree {c3.cheb_degree}",
            **_measure_case(torch, stream, flush, c3, 10, 1, keep=keep))
    if want("naca0012_re1000_2048x1024_projected"):
        c3p = inputs.naca0012_re1000_2048x1024()
        c3p.guess_history = GUESS_L
        out["naca0012_re1000_2048x1024_projected"] = dict(
            precision="mixed", precond=f"chebyshev degree {c3p.cheb_degree}",
            initial_guess=f"projection onto the last {GUESS_L} solutions",
            **_measure_case(torch, stream, flush, c3p, 10, 1))
    if want("naca0012_re1000_2048x1024_jacobi"):
        out["naca0012_re1000_2048x1024_jacobi"] = dict(
            precision="mixed", precond="jacobi (one launch, FP64 residual replacements)",
            **_measure_case(torch, stream, flush, c3, 2, 1, precond="jacobi"))
    return out


def measure_batch(torch, stream, flush, ncases=64, steps=10, warmup=4):
    """The 64-case batch (cylinders and NACA00tt sections, 256..1024 cells wide, mixed
    precision, Chebyshev degree 4 as configured): all cases advance together, one batched
    Poisson solve per step.  The warm-up covers the cases' first step and the three steps that
    tune the Poisson launch's block split."""
    from paper_2211_10698_gb300 import ccm, inputs

    specs = inputs.batch_cases(ncases)
    alloc = ccm.TorchAllocator()
    cases = [ccm.Case(c, stream=stream.cuda_stream, allocator=alloc) for c in specs]
    b = ccm.Batch(ncases, stream=stream.cuda_stream)
    for c in cases:
        b.add(c)
    b.step(warmup)
    last = []
    ms = _timed_steps(torch, stream, lambda: last.append(b.step(1)), steps, flush)
    cells = sum(c.cells for c in specs)
    t = sum(ms)
    its = [st["last_iters_p"] for st in last[-1]]
    its_window = [sum(st["last_iters_p"] for st in sts) / len(sts) for sts in last]
    conv = all(st["converged"] for sts in last for st in sts)
    graph_steps = b.graph_steps()
    split_a, split_tuned = b.split()
    b.close()
    for c in cases:
        c.close()
    pcs = sorted({f"{c.precond}" + (f" degree {c.cheb_degree}" if c.precond == "chebyshev" else "") for c in specs})
    return dict(workload=f"batch of {ncases} cases ({cells} cells)", precision="mixed", cells=cells,
                value=cells * steps / (t * 1e-3), unit=UNIT, ms_per_step=t / steps, steps=steps,
                precond=", ".join(pcs), poisson_iters_last_step={"max": max(its), "mean": sum(its) / len(its)},
                poisson_iters_mean_per_step=its_window, window=f"steps {warmup + 1}..{warmup + steps} of each case",
                converged=conv, graph_steps=graph_steps,
                poisson_split=dict(weights=f"cells x nx^{split_a:g}", tuned=split_tuned),
                note="every stage of a step is one launch for all cases: explicit stages, the Helmholtz "
                     "solves and the Poisson solves (cooperative); steps after the first replay captured "
                     "CUDA graphs")


def measure_serving(precision, nreq=32, step_div=100, budget_gb=150.0, max_batch=64, chunk=5):
    """A bounded window of the request stream (exponential arrivals at 20/s; cylinders and
    NACA00tt sections 128..2048 cells wide; the first ``nreq`` requests, their step counts
    divided by ``step_div``): requests are submitted when their arrival time has passed and the
    loop runs rounds until all are done.  Latency runs from arrival to completion."""
    import numpy as np

    from paper_2211_10698_gb300 import ccm, inputs

    reqs = inputs.serving_requests(nreq)
    srv = ccm.Server(int(budget_gb * 1e9), max_batch=max_batch, chunk_steps=chunk)
    pending = list(reqs)
    ids = []
    t0 = time.monotonic()
    active = 0
    peak_bytes = 0
    while pending or active:
        now = time.monotonic() - t0
        if not active and pending and pending[0][0] > now:
            time.sleep(pending[0][0] - now)
            now = time.monotonic() - t0
        while pending and pending[0][0] <= now:
            arr, c = pending.pop(0)
            n = max(1, c.steps // step_div)
            ids.append((arr, c, n, srv.submit(c, nsteps=n, precision=precision,
                                              precond="jacobi" if precision == "fp64" else None)))
        active = srv.run(1)
        peak_bytes = max(peak_bytes, srv.bytes_in_use())
    lat, cell_steps, t_end, fails = [], 0, 0.0, 0
    for arr, c, n, rid in ids:
        p = srv.poll(rid)
        fails += p["state"] != "done" or not p["converged"]
        lat.append(p["t_done"] - (t0 + arr))
        cell_steps += c.cells * n
        t_end = max(t_end, p["t_done"] - t0)
        srv.release(rid)
    srv.close()
    lat = np.array(lat)
    return dict(precision=precision, requests=len(ids), value=cell_steps / t_end, unit=UNIT,
                p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                makespan_s=t_end, cell_steps=cell_steps, failed=int(fails), peak_hbm_bytes=int(peak_bytes))


def run_ours(args):
    import numpy as np
    import torch

    from paper_2211_10698_gb300 import ccm, inputs

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    case = inputs.cylinder_re100_1024x512()
    case.guess_history = args.guess_history
    case.precision, case.precond, case.cheb_degree = args.precision, args.precond, args.cheb_degree
    stream = torch.cuda.current_stream()
    if args.launch_plan:
        case.autotune = 0
    g = ccm.Case(case, stream=stream.cuda_stream, allocator=ccm.TorchAllocator())
    if args.launch_plan:
        g.set_launch_plan(tuple(int(x) for x in args.launch_plan.split(",")))
    pu, pv = inputs.perturbation(case)
    g.set_field(ccm.CCM_F_U, g.get_field(ccm.CCM_F_U) + pu)
    g.set_field(ccm.CCM_F_V, g.get_field(ccm.CCM_F_V) + pv)
    g.step(args.warmup)
    launch_plan = _plan_dict(g, case.precision)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    g.enable_kernel_timing(True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = Clocks(local)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        g.step_async(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    st = g.read_stats()
    kt = g.kernel_timing()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = job_time_ms(sum(step_ms), world)
    value = job_value(world, case.cells, args.steps, t_ms)
    iters_p = st["iters_p"] / args.steps
    iters_h = st["iters_h"] / args.steps

    # end to end through the C ABI with host (pinned) buffers: upload U, V, P, one step,
    # download U, V, P
    shape = case.shape
    hb = [torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(3)]
    fields = (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P)
    for f, buf in zip(fields, hb):
        g.get_field(f, out=buf)
    g.enable_kernel_timing(False)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(args.e2e_steps):
        for f, buf in zip(fields, hb):
            g.set_field(f, buf)
        e2e_iters += g.step(1)["iters_p"]
        for f, buf in zip(fields, hb):
            g.get_field(f, out=buf)
    e2e_s = time.perf_counter() - e0
    e2e_val = world * case.cells * args.e2e_steps / e2e_s if args.e2e_steps > 0 else None
    nbytes = 3 * shape[0] * shape[1] * 8

    peaks, peak_kind = _peaks()
    # the FP64 FMA rate of this GPU, measured (independent FMA chains, CUDA events)
    import ctypes as _ct

    fp64_meas = _ct.c_double(0.0)
    fp64_peak, fp64_src = FP64_PEAK_TFLOPS, "FP64 unit count x clock (152 SMs x 2 FMA/clk x 2 x 2.07 GHz)"
    if ccm.lib().ccm_measure_fp64_rate(_ct.byref(fp64_meas)) == ccm.CCM_OK and fp64_meas.value > 0:
        fp64_peak = fp64_meas.value
        fp64_src = ("measured FP64 FMA rate of this GPU (ccm_measure_fp64_rate: independent FMA chains, "
                    "CUDA events, best of 3)")
    launches = max(kt["poisson_launches"], 1)
    avg_ms = kt["poisson_ms"] / launches
    iters_per_launch = kt["poisson_iters"] / launches
    flops = PCG_FLOPS_PER_CELL_ITER * case.cells * iters_per_launch
    bytes_alg = PCG_BYTES_PER_CELL_ITER * case.cells * iters_per_launch
    achieved_tf = flops / (avg_ms * 1e-3) / 1e12
    achieved_gbs = bytes_alg / (avg_ms * 1e-3) / 1e9
    frac_alu = achieved_tf / fp64_peak
    frac_hbm = achieved_gbs / peaks["hbm_gbs"]
    kernel = kernel_of(launch_plan)
    traffic_pc, prof = _traffic_from_profile(kernel)
    traffic = traffic_pc * case.cells * iters_per_launch if traffic_pc is not None else None
    if frac_alu >= frac_hbm:
        roof = dict(bound="alu", achieved=achieved_tf, peak=fp64_peak, unit="TFLOP/s", frac=frac_alu,
                    traffic=traffic, kernel=kernel, peak_source=fp64_src)
    else:
        roof = dict(bound="hbm", achieved=achieved_gbs, peak=peaks["hbm_gbs"], unit="GB/s", frac=frac_hbm,
                    traffic=traffic, kernel=kernel, peak_source=f"{peak_kind} hbm_gbs")
    roof_alt = dict(hbm_achieved_gbs=achieved_gbs, hbm_peak_gbs=peaks["hbm_gbs"], hbm_frac=frac_hbm,
                    fp64_achieved_tflops=achieved_tf, fp64_peak_tflops=fp64_peak, fp64_frac=frac_alu,
                    fp64_unit_count_peak_tflops=FP64_PEAK_TFLOPS,
                    fp64_frac_of_unit_count_peak=achieved_tf / FP64_PEAK_TFLOPS,
                    avg_launch_ms=avg_ms, iters_per_launch=iters_per_launch,
                    us_per_iteration=1e3 * avg_ms / max(iters_per_launch, 1), peak_kind=peak_kind)

    head_next = gpu_next_step(g) if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    extras = {}
    c3_keep = {}
    want = set() if args.no_extras else set(args.extras.split(","))
    if rank == 0 and "mixed" in want:
        variants = {"mixed_same_accuracy": dict(precision="mixed", precond="jacobi"),
                    "mixed_chebyshev": dict(precision="mixed", precond="chebyshev", degree=3),
                    "mixed_chebyshev_projected": dict(precision="mixed", precond="chebyshev", degree=3, guess=GUESS_L)}
        if args.guess_history:
            variants["fp64_previous_phi"] = dict(precision="fp64", precond="jacobi", guess=0)
        else:
            variants["fp64_projected_guess"] = dict(precision="fp64", precond="jacobi", guess=GUESS_L)
        for name, kw in variants.items():
            try:
                extras[name] = measure_variant(torch, stream, flush, **kw)
            except Exception as e:  # report, do not lose the headline line
                extras[name] = {"error": str(e)}
    if rank == 0 and "configs" in want:
        try:
            extras["configs"] = measure_configs(torch, stream, flush,
                                                set(filter(None, args.configs.split(","))), keep=c3_keep)
        except Exception as e:
            extras["configs"] = {"error": str(e)}
    if rank == 0 and "batched" in want:
        try:
            extras["batched"] = measure_batch(torch, stream, flush, ncases=args.batch_cases)
        except Exception as e:
            extras["batched"] = {"error": str(e)}
    if rank == 0 and "serving" in want:
        try:
            torch.cuda.synchronize()
            nreq, sdiv = (int(x) for x in args.serving_window.split(","))
            sv = dict(workload=f"request stream window: first {nreq} requests at 20/s, steps/{sdiv}, "
                               f"budget 150 GB, batches of up to 64, chunks of 5 steps")
            sv["mixed"] = measure_serving("mixed", nreq=nreq, step_div=sdiv)
            sv["fp64"] = measure_serving("fp64", nreq=nreq, step_div=sdiv)
            extras["serving"] = sv
        except Exception as e:
            extras["serving"] = {"error": str(e)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c3_next = None
        if "next" in c3_keep:
            c3_next = (inputs.naca0012_re1000_2048x1024(),) + tuple(c3_keep["next"])
        cpu = cpu_baseline(case, head_next, c3_next, full=args.cpu_baseline_full)
    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=t_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="f64" if case.precision == "fp64" else "f32+f64", data="synthetic",
                    config=dict(workload=WORKLOAD, nx=case.nx, ny=case.ny, cells=case.cells, precision=case.precision,
                                precond=case.precond + (f" degree {case.cheb_degree}" if case.precond == "chebyshev" else ""), tol_p=case.tol_p, tol_h=case.tol_h, parallelism=f"replicas{world}",
                                initial_guess=(f"projection onto the last {case.guess_history} solutions"
                                               if case.guess_history else "previous Phi"),
                                l2="flushed between timed steps (256 MiB write, outside the step events)",
                                poisson_iters_per_step=iters_p, helmholtz_iters_per_step=iters_h,
                                launch_plan=launch_plan),
                    roofline=roof, roofline_detail=roof_alt, cpu_baseline=cpu,
                    e2e=dict(value=e2e_val, unit=UNIT, h2d_bytes_per_step=nbytes, d2h_bytes_per_step=nbytes,
                             steps=args.e2e_steps,
                             # the steps after the timed ones, later on the trajectory: their Poisson
                             # iteration count sets their cost, as iters_per_step does the headline's
                             poisson_iters_per_step=(e2e_iters / args.e2e_steps) if args.e2e_steps > 0 else None),
                    gpu_launches=int(kt["kernel_launches"]), clocks=clocks,
                    wall_s=wall, step_ms_min=min(step_ms), step_ms_max=max(step_ms),
                    max_div=st["max_div"], kinetic=st["kinetic"], converged=bool(st["converged"]))
        line.update(extras)
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
