"""Benchmark: time per load step of the semismooth-Newton TFETI solver (Algorithm 4).

Workload: unit cube of 64^3 trilinear bricks torn into 8x8x8 = 512 boxes of 8^3
elements (2187 dofs each, 308 544 multipliers), the Sec. 5 material, u = 0 on z = 0,
uniform x-traction on z = 1 ramped linearly to 1.5 x the first-yield load over 20
load steps; eps_PCGP = 1e-8 (dual relative residual), eps_Newton = 1e-6.

One bench step = one load step (ssn_time_step): every Newton iteration runs the
return mapping, the tangent assembly, the subdomain factorisations, the PCGP
dual solve with its F-applies and projections, and the recovery.  The K timed steps
are load steps 1..K of the ramp (K = 20: the whole ramp; beyond step 20 the load
would keep rising at the same rate).  The W warm-up steps run before them on the same
context as a coarser ramp to the same final load (0 -> 1.5 t_y in W steps, so the
plastic code paths and pools are warm) and are discarded: the state is reset to zero
and the start history and network restart.  Inputs (factors 2.5 GB) are larger than
L2, so no flush is needed between steps.

Arms: default = the CUDA path; ``--impl reference`` = the FP64 CPU oracle: one full
Newton iteration of load step 1 timed live (single core, and concurrently on every core),
scaled by the oracle's Newton iterations per step (see ``oracle_newton_sample``).  For
N > 1 (torchrun) each rank solves an independent replica of the workload (weak
scaling; the solver itself runs on one GPU).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "time per load step @1e-8 dual res: FP64 vs mixed+learned; F-apply % HBM peak"
UNIT = "s/load_step"
FP64_NOMINAL_TFLOPS = 1.25    # GB300 FP64 rate as published; the roofline uses the rate measured in the run


# DRAM traffic per launch of the banded F-apply kernel at the 64^3 benchmark size, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum; the launch-list summary under profiles/ gives the
# command).  Valid only while the kernel source is the one measured.
MEASURED_TRAFFIC = {"k_sub_solve": {"workload": "cube64_8x8x8", "bytes": 34.37e6,
                                    "src": "paper_1205_1926_gb300/csrc/kernels_band.cu",
                                    "sha256": "5f8f884233206d10cad9c65b326615a3ce4106e7bd603f2808adf1301e97fb6d"}}


def measured_traffic(kernel, workload):
    rec = MEASURED_TRAFFIC.get(kernel)
    if rec is None or rec["workload"] != workload:
        return None
    try:
        with open(os.path.join(ROOT, rec["src"]), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != rec["sha256"]:
                return None
    except OSError:
        return None
    return rec["bytes"]


def algorithmic_fapply(w):
    """Algorithmic FP64 work and bytes of one banded F-apply: for every box its factor of n (bw + 1)
    entries (n dofs, half bandwidth bw of the lexicographic order), read by a forward and a backward
    sweep at 2 flops per entry; bytes as stored (8 per entry and sweep)."""
    entries = 0
    for k in range(len(w.cuts[2]) - 1):
        for j in range(len(w.cuts[1]) - 1):
            for i in range(len(w.cuts[0]) - 1):
                ax = w.cuts[0][i + 1] - w.cuts[0][i]
                ay = w.cuts[1][j + 1] - w.cuts[1][j]
                az = w.cuts[2][k + 1] - w.cuts[2][k]
                n = 3 * (ax + 1) * (ay + 1) * (az + 1)
                bw = 3 * ((ax + 1) * (ay + 1) + (ax + 1) + 1) + 2
                entries += n * (bw + 1)
    return {"flops": 4.0 * entries, "bytes": 16.0 * entries, "factor_entries": entries}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def workload_config(w, steps, warmup, precond="lumped"):
    sched = "cyclic (load, unload, reverse, unload) to +-" if w.cyclic else "ramp to "
    return {"workload": f"{w.name}: {w.nel[0]}x{w.nel[1]}x{w.nel[2]} hex8 bricks, "
                        f"{len(w.cuts[0]) - 1}x{len(w.cuts[1]) - 1}x{len(w.cuts[2]) - 1} subdomains, "
                        f"{w.n_steps}-step {sched}{w.load_factor} x first-yield x-traction on z=1",
            "newton_tol": w.newton_tol, "pcg_rtol": w.pcg_rtol, "preconditioner": precond,
            "kdag": "fixing-node banded Cholesky (shared elastic factor per box shape)",
            "load_steps_timed": f"1..{steps} of the {w.n_steps}-step schedule",
            "warmup": f"{warmup} load steps of a coarser ramp to the schedule's peak load on the same context, "
                      "then the state reset to zero (discarded)",
            "l2": "inputs larger than L2 (subdomain factors 2.5 GB), no flush"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples go to BENCH_CLOCKS_DIR (default: the system's temporary directory)
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------------------- oracle
def oracle_newton_sample(w):
    """Time one full Newton iteration of the FP64 oracle on load step 1 of the workload.

    The sample is the body of Algorithm 4 once, on every subdomain: Algorithm 5 (return map and
    tangent assembly), the fixing-node factorisations and the coarse matrix (the solver set-up),
    Algorithm 3 to eps_PCGP with its recovery, and the Newton update; then the commit (the return
    map at the increment).  The model's mesh, B and R set-up is excluded like the GPU's set-up.
    The first-yield traction comes from the oracle's record of this workload when it has one.
    """
    import numpy as np
    from oracle.ssn import ElastoplasticModel
    model = ElastoplasticModel(w)
    t_y = None
    rec_path = os.path.join(ROOT, "tests", "golden", "cube64_oracle_record.json")
    if w.name == "cube64_8x8x8" and os.path.exists(rec_path):
        with open(rec_path) as fh:
            t_y = json.load(fh)["t_y"]
    if t_y is None:
        t_y = model.first_yield_traction(rtol=1e-10)
    df = w.load_fractions()[0] * t_y * model.traction_load(w.traction_dir)
    du = np.zeros(model.dec.n_dof)
    t0 = time.perf_counter()
    K_blocks, f, _ = model.assemble(du, df)
    t1 = time.perf_counter()
    solver = model.tfeti(K_blocks)
    t2 = time.perf_counter()
    sol = solver.solve(f, rtol=w.pcg_rtol, maxit=w.pcg_maxit)
    du_new = du + sol["u"]
    np.linalg.norm(du_new - du) / (np.linalg.norm(du_new) + np.linalg.norm(du))
    t3 = time.perf_counter()
    model.return_map(du_new)
    t4 = time.perf_counter()
    return {"newton_s": t3 - t0, "assembly_s": t1 - t0, "setup_s": t2 - t1, "solve_s": t3 - t2,
            "commit_s": t4 - t3, "pcg_iterations": sol["iterations"], "cores": 1}


THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
              "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")
SAMPLE_KEYS = ("newton_s", "assembly_s", "setup_s", "solve_s", "commit_s")


def _single_thread_env():
    env = dict(os.environ)
    for k in THREAD_ENV:
        env[k] = "1"
    return env


def oracle_sample_subprocess(workload_name):
    """oracle_newton_sample in a fresh interpreter whose BLAS/OpenMP pools hold one thread."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", workload_name],
                       env=_single_thread_env(), capture_output=True, text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def _mem_available_bytes():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def oracle_sample_all_cores(workload_name, n_proc=None, bytes_per_proc=8e9):
    """The same sample run as concurrent single-thread oracle processes, one per host core (fewer if
    host memory would not hold them): their mean is the oracle's time per core with every core busy.
    Dividing a step's time by the process count estimates the oracle with its subdomain work split
    over all cores (the parallelism of Sec. 4.3); the coarse problem and the reductions would not
    split that well, so this is a lower bound on its time."""
    n_proc = n_proc or os.cpu_count() or 1
    avail = _mem_available_bytes()
    if avail is not None:
        n_proc = max(1, min(n_proc, int(0.8 * avail // bytes_per_proc)))
    procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-sample", workload_name],
                              env=_single_thread_env(), stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
             for _ in range(n_proc)]
    outs = []
    for pr in procs:
        out, _ = pr.communicate()
        if pr.returncode == 0:
            outs.append(json.loads(out.strip().splitlines()[-1]))
    if not outs:
        return None
    return {k: statistics.mean(o[k] for o in outs) for k in SAMPLE_KEYS} | {"cores": len(outs)}


def oracle_step_seconds(s, newton_per_step):
    """Seconds per load step: Newton iterations per step x one full Newton iteration, plus the commit.
    Every Newton solve of the 64^3 ramp takes about the same number of PCGP iterations (24-25 in the
    oracle's record of all 20 steps), so a Newton iteration costs about the same in every step."""
    return newton_per_step * s["newton_s"] + s["commit_s"]


def oracle_record_newton(first, last):
    path = os.path.join(ROOT, "tests", "golden", "cube64_oracle_record.json")
    with open(path) as fh:
        rec = json.load(fh)
    steps = [s for s in rec["steps"] if first <= s["step"] <= last] or rec["steps"]
    return statistics.mean(s["newton"] for s in steps), f"oracle record, load steps {steps[0]['step']}..{steps[-1]['step']}"


def cpu_baseline_line(w, newton_per_step, counts_src, all_cores=True):
    """The oracle timed live on this host: one full Newton iteration (single core, then every core at
    once), scaled to a load step with the given Newton iterations per step."""
    s = oracle_sample_subprocess(w.name)
    v = oracle_step_seconds(s, newton_per_step)
    out = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"one full Newton iteration of load step 1 (Algorithm 5 on all {w.n_sub} subdomains, "
                     f"their fixing-node factorisations and the coarse matrix, Algorithm 3 to eps_PCGP = "
                     f"{w.pcg_rtol:g} ({s['pcg_iterations']} PCGP iterations) and the recovery) plus the commit, "
                     f"timed live on one core with one BLAS thread; x {newton_per_step:.2f} Newton iterations "
                     f"per load step ({counts_src})",
           "components_s": {k: s[k] for k in SAMPLE_KEYS}, "pcg_iterations_in_sample": s["pcg_iterations"]}
    if all_cores:
        sa = oracle_sample_all_cores(w.name)
        if sa is not None:
            va = oracle_step_seconds(sa, newton_per_step)
            out["all_cores"] = {"value": va / sa["cores"], "unit": UNIT, "cores": sa["cores"],
                                "per_core_step_s": va, "components_s": {k: sa[k] for k in SAMPLE_KEYS},
                                "kind": "oracle, one single-thread process per core running the same sample",
                                "note": "per-core step time with every core busy / cores = the oracle with its "
                                        "subdomain work split over all cores (a lower bound)"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = W.CUBE64
    t_start = time.perf_counter()
    try:
        newton, src = oracle_record_newton(1, args.steps)
    except (OSError, ValueError, KeyError):
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration-count record missing"}))
        return
    cb = cpu_baseline_line(w, newton, src, all_cores=not args.no_all_cores)
    cb["wall_s"] = time.perf_counter() - t_start
    v = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args.steps, args.warmup),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------------------- replicas
def max_over_ranks(values, device=None):
    """Element-wise max of per-rank timings over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def replica_value(elapsed_max, steps, world):
    """Time per load step of the whole job: every rank solves its own replica of the workload
    for `steps` load steps, so the job completes steps * world load steps in elapsed_max."""
    return elapsed_max / (steps * world)


# --------------------------------------------------------------------------------------- CUDA path
ARMS = ("fp64", "mixed", "mixed_history", "mixed_learned")
EXTRA_ARMS = ("mixed_learned_deflated", "mixed_history_bf16")   # measured variants that lose (--extra-arms)
ARM_NOTES = {
    "fp64": "Algorithm 3 in FP64 (banded K^+ applies), the paper's method",
    "mixed": "FP64-refined PCGP: FP32 dual Schur blocks on the tensor cores (elastic) and FP32 banded solves "
             "(plastic), FP32 projector and preconditioner inside; FP64 residual and stopping test",
    "mixed_history": "the mixed arm with each dual solve started from the Galerkin-optimal combination of the "
                     "solver's last 8 solutions, zero-start fallback",
    "mixed_learned": "the mixed arm with the learned start: the last 7 solutions plus the per-interface MLP "
                     "prediction (trained online on the solver's own lambda histories) as Galerkin vectors",
    "mixed_learned_deflated": "the mixed_learned arm with each inner PCGP deflated by 4 vectors: the network's "
                              "prediction and the most recent stored solutions, projected, A W by the inner operator",
    "mixed_history_bf16": "the mixed_history arm with the dual Schur blocks of the inner F-apply stored in BF16 "
                          "(X split into BF16 hi/lo, FP32 accumulation) instead of TF32 x 3",
}


def resolve_arm(args):
    if args.arm:
        return args.arm
    if args.precision == "fp64":
        return "fp64"
    if args.precision == "mixed":
        return "mixed_learned" if args.learned else "mixed"
    return "mixed_learned"


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import paper_1205_1926_gb300 as T

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w = W.WORKLOADS[args.workload]
    stream = torch.cuda.Stream(device=dev)
    pre = T.PRECOND_DIRICHLET if args.precond == "dirichlet" else T.PRECOND_LUMPED
    main_arm = resolve_arm(args)

    coarse = {"auto": T.COARSE_AUTO, "dense": T.COARSE_DENSE, "planes": T.COARSE_PLANES}[args.coarse]

    def make_ctx(arm):
        c = T.Context(w, stream=stream, precond=pre, coarse=coarse)
        if args.fapply == "schur":
            c.set_fapply(True)
        if arm != "fp64":
            c.set_precision(True, args.inner_rtol)
        if arm in ("mixed_history", "mixed_history_bf16"):
            c.set_recycling(args.history)
        if arm in ("mixed_learned", "mixed_learned_deflated"):
            c.set_recycling(min(args.history, 7))
            c.set_learned(True)
        if arm == "mixed_learned_deflated":
            c.set_deflation(args.deflation)
        if arm != "fp64" and (arm.endswith("_bf16") or args.schur_format == "bf16"):
            c.set_schur_format(True)
        if arm != "fp64":
            c.set_woodbury(0 if args.no_woodbury else args.woodbury)
        if arm != "fp64" and args.schur_threshold > 0:
            c.set_schur_threshold(args.schur_threshold)
        if args.no_graphs:
            c.set_graphs(False)
        if args.fused:
            c.set_fused_inner(True)
        return c

    def reset_start(c, arm):
        # the history and the network start over (the first-yield solve must not seed them)
        if arm in ("mixed_history", "mixed_history_bf16"):
            c.set_recycling(args.history)
        if arm in ("mixed_learned", "mixed_learned_deflated"):
            c.set_recycling(min(args.history, 7))
            c.set_learned(True)
        if arm == "mixed_learned_deflated":
            c.set_deflation(args.deflation)

    fp64_peak = T.measure_fp64_fma(stream)           # roofline denominator of the FP64 kernels
    ctx = make_ctx(main_arm)
    n = ctx.sizes["n_dof"]
    t_y = ctx.first_yield_traction(w.traction_dir, rtol=1e-10)
    reset_start(ctx, main_arm)
    fr = w.load_fractions(args.steps)               # timed: load steps 1..K of the schedule
    peak_level = max(abs(a) for a in w.load_fractions())
    dfs, prev = [], 0.0
    with torch.cuda.stream(stream):
        for a in fr:
            d = torch.zeros(n, dtype=torch.float64, device=dev)
            ctx.traction_load(tuple((a - prev) * t_y * c for c in w.traction_dir), d)
            dfs.append(d)
            prev = a
        # warm-up increment: W equal steps from 0 to the schedule's largest load level
        df_warm = torch.zeros(n, dtype=torch.float64, device=dev)
        ctx.traction_load(tuple(peak_level / max(args.warmup, 1) * t_y * c for c in w.traction_dir), df_warm)
        zero_u = torch.zeros(n, dtype=torch.float64, device=dev)
        zero_s = torch.zeros(6 * ctx.sizes["n_gp"], dtype=torch.float64, device=dev)
        zero_k = torch.zeros(ctx.sizes["n_gp"], dtype=torch.float64, device=dev)
    stream.synchronize()

    def warm_up(c, arm, on_host=None):
        """W load steps of the coarse warm-up ramp, then back to the zero state with the start
        history and the network restarted: the timed steps see warm pools, tuned F-apply and loaded
        code but nothing of the warm-up's solutions."""
        for _ in range(args.warmup):
            if on_host is not None:
                c.time_step(on_host.data_ptr(), w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit,
                            df_on_host=True)
            else:
                c.time_step(df_warm, w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit)
        c.set_state(u=zero_u, sigma=zero_s, kappa=zero_k)
        reset_start(c, arm)
        torch.cuda.synchronize()

    def timed_run(c, arm, headline=False):
        """Warm-up, then load steps 1..K timed (inputs resident in HBM, CUDA events on the context
        stream, max over ranks); u after every step is kept for the comparisons made afterwards."""
        warm_up(c, arm)
        snaps = torch.zeros((args.steps, n), dtype=torch.float64, device=dev)
        infos = []
        sampler = ClockSampler(local_rank) if headline else None
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        c.timing_reset(headline)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            infos.append(c.time_step(dfs[k], w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit))
            c.get_state(u=snaps[k])
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        elapsed = max_over_ranks([e0.elapsed_time(e1) / 1e3], dev)[0]
        return {"elapsed": elapsed, "infos": infos, "snaps": snaps, "tm": c.timing(), "clocks": clocks,
                "tuning": c.tuning() if hasattr(c, "tuning") else None,
                "deflation": c.deflation_stats() if arm == "mixed_learned_deflated" else None,
                "woodbury": c.woodbury_stats() if arm != "fp64" else None}

    main = timed_run(ctx, main_arm, headline=True)
    ctx.close()

    # ---- end-to-end pass of the headline arm through the C ABI with host (pinned) buffers, on a fresh
    # context (the learned start's history and network must start over with the states)
    e2e = None
    if not args.no_e2e:
        ce = make_ctx(main_arm)
        dfs_h = [d.cpu().pin_memory() for d in dfs]
        warm_up(ce, main_arm, on_host=df_warm.cpu().pin_memory())
        u_host = torch.zeros(n, dtype=torch.float64).pin_memory()
        u_dev = torch.zeros(n, dtype=torch.float64, device=dev)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            ce.time_step(dfs_h[k].data_ptr(), w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit, df_on_host=True)
            ce.get_state(u=u_dev)
            with torch.cuda.stream(stream):
                u_host.copy_(u_dev, non_blocking=True)
            stream.synchronize()
        torch.cuda.synchronize()
        barrier()
        elapsed_e2e = max_over_ranks([time.perf_counter() - t0], dev)[0]
        ce.close()
        e2e = {"value": replica_value(elapsed_e2e, args.steps, world), "unit": UNIT,
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
               "matches_device_pass": bool(torch.equal(u_host.to(dev), main["snaps"][-1]))}

    # ---- the other arms of the metric on the same load history
    runs = {main_arm: main}
    if not args.no_mixed:
        for arm in ARMS + (EXTRA_ARMS if args.extra_arms else ()):
            if arm == main_arm:
                continue
            c = make_ctx(arm)
            runs[arm] = timed_run(c, arm)
            c.close()
    ref = runs.get("fp64")

    def rel_u_diffs(r):
        if ref is None or r is ref:
            return None
        # compared after the timed regions: no torch kernel runs inside them
        return (torch.linalg.vector_norm(r["snaps"] - ref["snaps"], dim=1) /
                torch.linalg.vector_norm(ref["snaps"], dim=1)).tolist()

    value = replica_value(main["elapsed"], args.steps, world)
    units = args.steps * world
    pk, pk_kind = peaks()
    tm = main["tm"]
    # F-apply kernels: the banded K^+ solves (k_sub_solve: every F-apply of the FP64 arm, the residual
    # solves of the mixed arms) and, with --fapply schur, the FP64 dual-Schur DGEMM.  The roofline object
    # describes the one with the larger share of the headline arm's device time; the other sits beside it.
    # Both are FP64-FMA-bound on this GPU (0.25 flop/B against a ridge of fp64 / hbm ~ 0.18 flop/B), so the
    # peak is the FP64 FMA rate measured in this run.
    algo = algorithmic_fapply(w)
    avg_f_ms = tm["f_apply_ms_total"] / max(tm["f_apply_launches"], 1)
    achieved_tf = algo["flops"] / (avg_f_ms * 1e-3) / 1e12 if avg_f_ms > 0 else None
    traffic = measured_traffic("k_sub_solve", w.name)
    dram_gbs = traffic / (avg_f_ms * 1e-3) / 1e9 if (traffic and avg_f_ms > 0) else None
    peak_kind = (f"FP64 FMA rate measured in this run (tfeti_measure_fp64_fma); nominal {FP64_NOMINAL_TFLOPS}")
    banded = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
              "frac": achieved_tf / fp64_peak if achieved_tf else None,
              "traffic": traffic,
              "kernel": "k_sub_solve (banded forward/backward substitution with the factor records, FP64)",
              "peak_kind": peak_kind,
              "algorithmic": algo | {"note": "per launch: every subdomain's banded factor n (bw + 1) entries, "
                                             "2 flops per entry and right-hand side, forward and backward sweep"},
              "total_ms": tm["f_apply_ms_total"], "launches": tm["f_apply_launches"], "avg_launch_ms": avg_f_ms,
              "executed_flops_per_launch": tm["f_apply_flops"],
              "hbm": {"dram_gbs": dram_gbs, "peak_gbs": pk["hbm_gbs"],
                      "frac": dram_gbs / pk["hbm_gbs"] if dram_gbs else None,
                      "of": f"{pk_kind} hbm_gbs; DRAM bytes per launch from the ncu capture (traffic): the "
                            "shared elastic factor record stays in L2, so HBM does not bound this kernel"}}
    schur = None
    if tm["schur_launches"] > 0 and tm["schur_ms_total"] > 0:
        s_tf = tm["schur_flops_total"] / (tm["schur_ms_total"] * 1e-3) / 1e12
        schur = {"bound": "alu", "achieved": s_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                 "frac": s_tf / fp64_peak, "traffic": None,
                 "kernel": "k_schur_dgemm (+ gather): Y = X S with the shape's FP64 dual Schur block",
                 "peak_kind": peak_kind,
                 "total_ms": tm["schur_ms_total"], "launches": tm["schur_launches"],
                 "flops_per_launch": tm["schur_flops_total"] / tm["schur_launches"],
                 "avg_launch_ms": tm["schur_ms_total"] / tm["schur_launches"]}
    if schur is not None and schur["total_ms"] >= banded["total_ms"]:
        roof, other = dict(schur), banded
    else:
        roof, other = dict(banded), schur
    if other is not None:
        roof["other_kernel"] = other

    def per_step(r):
        return {"newton_per_step": [s["newton"] for s in r["infos"]],
                "pcg_per_step": [sum(s["pcg"]) for s in r["infos"]],
                "outer_per_step": [sum(s["outer"]) for s in r["infos"]],
                "history_starts_per_step": [sum(1 for h in s["history"] if h) for s in r["infos"]]}

    arms = {}
    for arm, r in runs.items():
        if arm == main_arm:
            continue
        v = replica_value(r["elapsed"], args.steps, world)
        d = rel_u_diffs(r)
        arms[arm] = {"value": v, "unit": UNIT, "headline_speedup": v / value, "note": ARM_NOTES[arm],
                     "deflation": r.get("deflation"), "woodbury": r.get("woodbury"),
                     "max_rel_u_diff_vs_fp64": max(d) if d else None, "rel_u_diff_vs_fp64_per_step": d,
                     "inner_fapply_tuning": r["tuning"] if arm != "fp64" else None} | per_step(r)
    main_d = rel_u_diffs(main)
    fp64_run = runs.get("fp64")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if main_arm == "fp64" else "f64+f32", "data": "synthetic",
            "config": workload_config(w, args.steps, args.warmup, args.precond) | {
                "parallelism": "replicas" if world > 1 else "1 GPU", "arm": main_arm,
                "arm_note": ARM_NOTES[main_arm],
                "inner_rtol": args.inner_rtol if main_arm != "fp64" else None, "fapply": args.fapply,
                "inner_pcgp_launch": "kernel by kernel" if args.no_graphs else "one CUDA graph (WHILE node) per inner solve",
                "coarse": args.coarse},
            "e2e": e2e,
            "gpu_launches": int(tm["kernel_launches"]),
            "roofline": roof,
            "clocks": main["clocks"],
            "max_rel_u_diff_vs_fp64": max(main_d) if main_d else None,
            "inner_iteration": {"ms_total": tm["inner_ms_total"], "iterations": tm["inner_iterations"],
                                "body_runs": tm["inner_body_runs"],
                                "us_per_body_run": 1e3 * tm["inner_ms_total"] / max(tm["inner_body_runs"], 1),
                                "note": "device time of the inner FP32 PCGP graph launches (CUDA events) per body "
                                        "run (one PCGP iteration)"},
            "solver": {"t_y": t_y, "plastic_gp_final": main["infos"][-1]["plastic_committed"],
                       "woodbury": main.get("woodbury"),
                       "refactored_per_step": [s["refactored"] for s in main["infos"]],
                       "factor_ms_total": tm["factor_ms_total"], "f_apply_ms_total": tm["f_apply_ms_total"],
                       "inner_fapply_tuning": main["tuning"] if main_arm != "fp64" else None,
                       "rel_u_diff_vs_fp64_per_step": main_d, "timed_s": main["elapsed"]} | per_step(main),
            "arms": arms}
    if fp64_run is not None:
        line["fp64_value"] = replica_value(fp64_run["elapsed"], args.steps, world)
        line["speedup_vs_fp64"] = line["fp64_value"] / value
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "cube64_8x8x8":
        counts = fp64_run if fp64_run is not None else main
        newton = statistics.mean(x["newton"] for x in counts["infos"])
        line["cpu_baseline"] = cpu_baseline_line(w, newton, "the FP64 arm's Newton iterations per step: the "
                                                            "oracle runs the same Algorithm 4",
                                                 all_cores=not args.no_all_cores)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_cases(args, rank, world, local_rank):
    """Several load cases of one mesh at once (--cases N): N case contexts sharing one base's read-only
    set-up, each on its own stream; every load step of all cases is one ssn_time_step_cases call (one host
    thread per case, the GPU overlapping the cases' kernels).  The same cases are then reset and stepped
    one after another on the same contexts (warm pools and tuning: favours the sequential run), and both
    are timed with CUDA events spanning all case streams."""
    import torch
    import paper_1205_1926_gb300 as T

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = W.WORKLOADS[args.workload]
    cases = W.direction_cases(args.cases) if args.case_set == "directions" else W.irregular_cases(0, args.cases)
    arm = resolve_arm(args)
    n_total = args.warmup + args.steps
    pre = T.PRECOND_DIRICHLET if args.precond == "dirichlet" else T.PRECOND_LUMPED
    main_stream = torch.cuda.Stream(device=dev)
    base = T.Context(w, stream=main_stream, precond=pre,
                     coarse={"auto": T.COARSE_AUTO, "dense": T.COARSE_DENSE, "planes": T.COARSE_PLANES}[args.coarse])
    streams = [torch.cuda.Stream(device=dev) for _ in cases]
    ctxs = [T.Context.case_of(base, c["sigma_y"], c["hardening"], stream=st) for c, st in zip(cases, streams)]

    def start(c):
        if arm != "fp64":
            c.set_precision(True, args.inner_rtol)
            if arm.endswith("_bf16") or args.schur_format == "bf16":
                c.set_schur_format(True)
        if arm in ("mixed_history", "mixed_history_bf16"):
            c.set_recycling(args.history)
        if arm in ("mixed_learned", "mixed_learned_deflated"):
            c.set_recycling(min(args.history, 7))
            c.set_learned(True)
        if arm == "mixed_learned_deflated":
            c.set_deflation(args.deflation)

    for c in ctxs:
        start(c)
    n = base.sizes["n_dof"]
    t_ys = [c.first_yield_traction(cs["traction_dir"], rtol=1e-10) for c, cs in zip(ctxs, cases)]
    for c in ctxs:
        start(c)      # the history and the network start over (the first-yield solve must not seed them)
    dfs = []
    for c, cs, t_y in zip(ctxs, cases, t_ys):
        row, prev = [], 0.0
        for a in w.load_fractions(n_total):
            d = torch.zeros(n, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            c.traction_load(tuple((a - prev) * t_y * x for x in cs["traction_dir"]), d)
            row.append(d)
            prev = a
        dfs.append(row)
    zero_u = torch.zeros(n, dtype=torch.float64, device=dev)
    zero_s = torch.zeros(6 * base.sizes["n_gp"], dtype=torch.float64, device=dev)
    zero_k = torch.zeros(base.sizes["n_gp"], dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    def reset():
        for c in ctxs:
            c.set_state(u=zero_u, sigma=zero_s, kappa=zero_k)
            start(c)
        torch.cuda.synchronize()

    def timed(concurrent, sampler=None):
        for k in range(args.warmup):
            if concurrent:
                T.time_step_cases(ctxs, [d[k] for d in dfs], w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit)
            else:
                for c, d in zip(ctxs, dfs):
                    c.time_step(d[k], w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit)
        torch.cuda.synchronize()
        for c in ctxs:
            c.timing_reset(False)
        if sampler:
            sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main_stream)
        for st in streams:
            st.wait_event(e0)
        infos = [[] for _ in cases]
        for k in range(args.warmup, n_total):
            if concurrent:
                out = T.time_step_cases(ctxs, [d[k] for d in dfs], w.newton_tol, w.pcg_rtol, w.newton_maxit,
                                        w.pcg_maxit)
            else:
                out = [c.time_step(d[k], w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit)
                       for c, d in zip(ctxs, dfs)]
            for j, o in enumerate(out):
                infos[j].append(o)
        for st in streams:
            ev = torch.cuda.Event()
            ev.record(st)
            main_stream.wait_event(ev)
        e1.record(main_stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        u = torch.zeros((len(cases), n), dtype=torch.float64, device=dev)
        launches = sum(c.timing()["kernel_launches"] for c in ctxs)
        for j, c in enumerate(ctxs):
            c.get_state(u=u[j])
        return e0.elapsed_time(e1) / 1e3, infos, u, clocks, launches

    el_c, inf_c, u_c, clocks, launches = timed(True, ClockSampler(local_rank))
    reset()
    el_s, inf_s, u_s, _, _ = timed(False)
    diff = (torch.linalg.vector_norm(u_c - u_s, dim=1) / torch.linalg.vector_norm(u_s, dim=1)).max().item()
    units = args.steps * len(cases)
    line = {"metric": f"time per load step per case @1e-8 dual res ({len(cases)} concurrent cases)",
            "value": el_c / units, "unit": "s/(load_step case)", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_c / args.steps * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if arm == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": workload_config(w, args.steps, args.warmup, args.precond) | {
                "arm": arm, "arm_note": ARM_NOTES[arm], "cases": len(cases), "case_set": args.case_set,
                "parallelism": "1 GPU, one stream and host thread per case",
                "shared": "mesh tables, G, H, shape templates, dual Schur blocks (one copy for all cases)"},
            "e2e": None, "gpu_launches": int(launches),
            "roofline": None, "clocks": clocks,
            "sequential_value": el_s / units, "concurrency_speedup": el_s / el_c,
            "max_rel_u_diff_concurrent_vs_sequential": diff,
            "cases": [{"sigma_y": cs["sigma_y"], "hardening": cs["hardening"], "traction_dir": cs["traction_dir"],
                       "t_y": t_y, "newton_per_step": [s["newton"] for s in inf],
                       "pcg_per_step": [sum(s["pcg"]) for s in inf],
                       "plastic_gp_final": inf[-1]["plastic_committed"]}
                      for cs, t_y, inf in zip(cases, t_ys, inf_c)],
            "device_bytes": {"base": base.sizes["device_bytes"],
                             "per_case_at_setup": [c.sizes["device_bytes"] for c in ctxs]}}
    if rank == 0:
        print(json.dumps(line))
    for c in ctxs:
        c.close()
    base.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", metavar="WORKLOAD", help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass (profiler runs)")
    ap.add_argument("--arm", default=None, choices=list(ARMS + EXTRA_ARMS),
                    help="the headline (timed, end-to-end) arm; default mixed_learned, the metric's method")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="shorthand: fp64 = --arm fp64, mixed = --arm mixed (or mixed_learned with --learned)")
    ap.add_argument("--inner-rtol", type=float, default=1e-4,
                    help="relative residual reduction of each inner FP32 PCGP solve of the mixed arms")
    ap.add_argument("--no-mixed", action="store_true", help="time the headline arm only (no other arms)")
    ap.add_argument("--fapply", default="banded", choices=["banded", "schur"],
                    help="FP64 F-apply of elastic subdomains: shape's dual Schur block (DGEMM) or banded solves")
    ap.add_argument("--extra-arms", action="store_true",
                    help="also time the deflated learned arm and the BF16 Schur arm (both measured slower)")
    ap.add_argument("--schur-threshold", type=int, default=0,
                    help="pin the inner F-apply's Schur threshold (0: autotuned; profilers serialise launches, "
                         "which misleads the tuner)")
    ap.add_argument("--woodbury", type=int, default=2, choices=[0, 1, 2],
                    help="mixed arms: plastic subdomains on their shape's elastic factor + a Woodbury correction "
                         "(1: inner FP32 F-apply only, 2: also the FP64 solves, no refactorisation; 0: off)")
    ap.add_argument("--no-woodbury", action="store_true", help="same as --woodbury 0")
    ap.add_argument("--deflation", type=int, default=4,
                    help="deflation vectors of the inner PCGP in the mixed_learned_deflated arm (1..8)")
    ap.add_argument("--coarse", default="auto", choices=["auto", "dense", "planes"],
                    help="coarse solve of the projector: explicit dense inverse, or block LDL^T over the z-planes "
                         "of subdomains (auto: planes above 6144 coarse unknowns)")
    ap.add_argument("--schur-format", default="tf32x3", choices=["tf32x3", "bf16"],
                    help="operand format of the inner F-apply's dual Schur blocks in every mixed arm")
    ap.add_argument("--precond", default="lumped", choices=["lumped", "dirichlet"],
                    help="PCGP preconditioner of Sec. 4.2 (every arm)")
    ap.add_argument("--learned", action="store_true",
                    help="with --precision mixed: the learned start (mixed_learned arm)")
    ap.add_argument("--history", type=int, default=8,
                    help="stored dual solutions of the history start in the mixed+learned arm (1..8)")
    ap.add_argument("--fused", action="store_true",
                    help="mixed arms: the inner PCGP iteration as one cooperative launch between F-applies "
                         "(measured slower than the separate kernels)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the mixed inner PCGP kernel by kernel instead of as one CUDA graph (for profilers)")
    ap.add_argument("--workload", default="cube64_8x8x8", choices=sorted(W.WORKLOADS),
                    help="cube64_8x8x8 is the benchmark; smaller cases exist for profiler captures")
    ap.add_argument("--no-all-cores", action="store_true",
                    help="skip timing the oracle sample on every host core at once (cpu_baseline.all_cores)")
    ap.add_argument("--cases", type=int, default=0,
                    help="N > 0: N load cases on one mesh stepped concurrently (case contexts), one JSON line")
    ap.add_argument("--case-set", default="directions", choices=["directions", "seeded"],
                    help="directions: theta_k = 2 pi k / N, the Sec. 5 material; seeded: sigma_y, H and the "
                         "direction drawn per case")
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_newton_sample(W.WORKLOADS[args.oracle_sample])))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.cases > 0:
        run_cases(args, rank, world, local_rank)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
