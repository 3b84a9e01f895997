"""Benchmark: time per load step of the semismooth-Newton TFETI solver (Algorithm 4).

Workload: unit cube of 64^3 trilinear bricks torn into 8x8x8 = 512 boxes of 8^3
elements (2187 dofs each, 308 544 multipliers), the Sec. 5 material, u = 0 on z = 0,
uniform x-traction on z = 1 ramped linearly to 1.5 x the first-yield load over 20
load steps; eps_PCGP = 1e-8 (dual relative residual), eps_Newton = 1e-6.

One bench step = one load step (ssn_time_step): every Newton iteration runs the
return mapping, the tangent assembly, the subdomain factorisations, the PCGP
dual solve with its F-applies and projections, and the recovery.  Warm-up steps
are the first W load steps of the history; the K timed steps continue it (beyond
step 20 the ramp continues at the same rate).  Inputs (factors 2.5 GB) are larger
than L2, so no flush is needed between steps.

Arms: default = the CUDA path; ``--impl reference`` = the FP64 CPU oracle on a
bounded sample of the same workload (see ``oracle_sample``).  For N > 1 (torchrun)
each rank solves an independent replica of the workload (weak scaling; the solver
itself runs on one GPU).
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
FP64_PEAK_TFLOPS = 1.207      # FP64 FMA throughput of a GB300 measured by a DFMA probe (nominal 1.25)


# DRAM traffic per launch of the banded F-apply kernel at the 64^3 benchmark size, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum; profiles/launches_cube64_bench.md gives the command).
# Valid only while the kernel source is the one measured.
MEASURED_TRAFFIC = {"k_sub_solve": {"workload": "cube64_8x8x8", "bytes": 34.32e6,
                                    "src": "paper_1205_1926_gb300/csrc/kernels_band.cu",
                                    "sha256": "01eefbee3c6566592055bea6187a029d8672e1baf076a248e4ff1e348cfe3f00"}}


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
            "load_steps_timed": f"{warmup + 1}..{warmup + steps}",
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
def oracle_sample(w, n_sub_sample=32, n_pcg_sample=2):
    """Time the FP64 oracle on a bounded sample of the workload (single BLAS thread).

    Sample: Algorithm 5 and the fixing-node factorisation for ``n_sub_sample`` of the
    subdomains (scaled to all of them), and ``n_pcg_sample`` full PCGP iterations over all
    subdomains (F-apply, two projections, lumped preconditioner).  Returns per-component
    seconds; the model set-up (mesh, B, R, N N^T) is excluded like the GPU's set-up.
    """
    import numpy as np
    from oracle.decomp import FixingNodeInverse
    from oracle.ssn import ElastoplasticModel
    model = ElastoplasticModel(w)
    n_sub = model.dec.n_sub
    subset = list(range(0, n_sub, max(1, n_sub // n_sub_sample)))[:n_sub_sample]
    f1 = model.traction_load(w.traction_dir)
    du = np.zeros(model.dec.n_dof)
    t0 = time.perf_counter()
    Kb_sub, _, _ = model.assemble(du, f1, subdomains=set(subset))
    t_asm = (time.perf_counter() - t0) * n_sub / len(subset)
    t0 = time.perf_counter()
    for K, p in zip(Kb_sub, subset):
        FixingNodeInverse(K, model.fixing[p])
    t_fac = (time.perf_counter() - t0) * n_sub / len(subset)
    # a full operator for the PCGP sample: the elastic factor of one box shape repeated
    kd0 = FixingNodeInverse(Kb_sub[0], model.fixing[subset[0]])
    solver = model.tfeti([Kb_sub[0]] * n_sub, kdag=[kd0] * n_sub)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(model.dec.m)
    t0 = time.perf_counter()
    for _ in range(n_pcg_sample):
        wv = solver.project(r)
        z = solver.apply_precond(wv)
        y = solver.project(z)
        solver.apply_F(y)
    t_pcg = (time.perf_counter() - t0) / n_pcg_sample
    t0 = time.perf_counter()
    solver.apply_F(r)
    t_fapply = time.perf_counter() - t0
    return {"assembly_s": t_asm, "factor_s": t_fac, "pcg_iter_s": t_pcg, "f_apply_s": t_fapply, "cores": 1,
            "sample": f"Algorithm 5 + fixing-node Cholesky on {len(subset)} of {n_sub} subdomains (scaled), "
                      f"{n_pcg_sample} PCGP iterations over all {n_sub} subdomains; 1 BLAS thread"}


THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
              "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def oracle_sample_subprocess(workload_name):
    """Run oracle_sample in a fresh interpreter whose BLAS/OpenMP pools are limited to one thread."""
    env = dict(os.environ)
    for k in THREAD_ENV:
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", workload_name],
                       env=env, capture_output=True, text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample_all_cores(workload_name, n_proc=None):
    """The same sample run as n_proc concurrent single-thread oracle processes (one per host core):
    their mean per-process result is the oracle's speed per core with every core busy (shared memory
    bandwidth and caches included).  Dividing a step's time by n_proc estimates the oracle with its
    subdomain-local work split over all cores, the parallelism of Sec. 4.3 (the coarse problem and the
    reductions would not split that well, so this is a lower bound on its time)."""
    n_proc = n_proc or os.cpu_count() or 1
    env = dict(os.environ)
    for k in THREAD_ENV:
        env[k] = "1"
    procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-sample", workload_name],
                              env=env, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
             for _ in range(n_proc)]
    outs = []
    for pr in procs:
        out, _ = pr.communicate()
        if pr.returncode == 0:
            outs.append(json.loads(out.strip().splitlines()[-1]))
    if not outs:
        return None
    keys = ("assembly_s", "factor_s", "pcg_iter_s", "f_apply_s")
    mean = {k: statistics.mean(o[k] for o in outs) for k in keys}
    return mean | {"cores": len(outs)}


def oracle_step_estimate(s, newton_per_step, pcg_per_step):
    """Seconds per load step: per Newton iteration assembly + factorisation + 3 set-up/recovery
    F-applies, plus the PCGP iterations, with the given iteration counts."""
    return newton_per_step * (s["assembly_s"] + s["factor_s"] + 3 * s["f_apply_s"]) + pcg_per_step * s["pcg_iter_s"]


def oracle_record_counts(first, last):
    path = os.path.join(ROOT, "tests", "golden", "cube64_oracle_record.json")
    with open(path) as fh:
        rec = json.load(fh)
    steps = [s for s in rec["steps"] if first <= s["step"] <= last] or rec["steps"]
    newton = statistics.mean(s["newton"] for s in steps)
    pcg = statistics.mean(sum(s["pcg"]) for s in steps)
    return newton, pcg, f"oracle record, load steps {steps[0]['step']}..{steps[-1]['step']}"


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = W.CUBE64
    t_start = time.perf_counter()
    try:
        newton, pcg, src = oracle_record_counts(args.warmup + 1, args.warmup + args.steps)
    except (OSError, ValueError, KeyError):
        newton, pcg, src = None, None, None
    s = oracle_sample_subprocess(w.name)
    if newton is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration-count record missing"}))
        return
    v = oracle_step_estimate(s, newton, pcg)
    sa = oracle_sample_all_cores(w.name) if args.oracle_all_cores else None
    elapsed = time.perf_counter() - t_start
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args.steps, args.warmup),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                             "sample": s["sample"] + f"; iteration counts per step from the {src} "
                                                     f"(Newton {newton:.2f}, PCGP {pcg:.1f})",
                             "components_s": {k: s[k] for k in ("assembly_s", "factor_s", "pcg_iter_s", "f_apply_s")},
                             "wall_s": elapsed},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if sa is not None:
        va = oracle_step_estimate(sa, newton, pcg)
        line["cpu_baseline"]["all_cores"] = {"value": va / sa["cores"], "unit": UNIT, "cores": sa["cores"],
                                             "per_core_step_s": va,
                                             "kind": "oracle, one single-thread process per core"}
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
ARM_NOTES = {
    "fp64": "Algorithm 3 in FP64 (banded K^+ applies), the paper's method",
    "mixed": "FP64-refined PCGP: FP32 dual Schur blocks on the tensor cores (elastic) and FP32 banded solves "
             "(plastic), FP32 projector and preconditioner inside; FP64 residual and stopping test",
    "mixed_history": "the mixed arm with each dual solve started from the Galerkin-optimal combination of the "
                     "solver's last 8 solutions, zero-start fallback",
    "mixed_learned": "the mixed arm with the learned start: the last 7 solutions plus the per-interface MLP "
                     "prediction (trained online on the solver's own lambda histories) as Galerkin vectors",
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
    n_total = args.warmup + args.steps
    stream = torch.cuda.Stream(device=dev)
    pre = T.PRECOND_DIRICHLET if args.precond == "dirichlet" else T.PRECOND_LUMPED
    main_arm = resolve_arm(args)

    def make_ctx(arm):
        c = T.Context(w, stream=stream, precond=pre)
        if args.fapply == "schur":
            c.set_fapply(True)
        if arm != "fp64":
            c.set_precision(True, args.inner_rtol)
        if arm == "mixed_history":
            c.set_recycling(args.history)
        if arm == "mixed_learned":
            c.set_recycling(min(args.history, 7))
            c.set_learned(True)
        if args.no_graphs:
            c.set_graphs(False)
        return c

    def reset_start(c, arm):
        # the history and the network start over (the first-yield solve must not seed them)
        if arm == "mixed_history":
            c.set_recycling(args.history)
        if arm == "mixed_learned":
            c.set_recycling(min(args.history, 7))
            c.set_learned(True)

    ctx = make_ctx(main_arm)
    n = ctx.sizes["n_dof"]
    t_y = ctx.first_yield_traction(w.traction_dir, rtol=1e-10)
    reset_start(ctx, main_arm)
    fr = w.load_fractions(n_total)
    dfs, prev = [], 0.0
    with torch.cuda.stream(stream):
        for a in fr:
            d = torch.zeros(n, dtype=torch.float64, device=dev)
            ctx.traction_load(tuple((a - prev) * t_y * c for c in w.traction_dir), d)
            dfs.append(d)
            prev = a
    stream.synchronize()

    def timed_run(c, headline=False):
        """Warm-up steps, then the K timed steps (inputs resident in HBM, CUDA events on the context
        stream, max over ranks); u after every step is kept for the comparisons made afterwards."""
        for k in range(args.warmup):
            c.time_step(dfs[k], w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit)
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
        for k in range(args.warmup, n_total):
            infos.append(c.time_step(dfs[k], w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit))
            c.get_state(u=snaps[k - args.warmup])
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        elapsed = max_over_ranks([e0.elapsed_time(e1) / 1e3], dev)[0]
        return {"elapsed": elapsed, "infos": infos, "snaps": snaps, "tm": c.timing(), "clocks": clocks,
                "tuning": c.tuning() if hasattr(c, "tuning") else None}

    main = timed_run(ctx, headline=True)
    ctx.close()

    # ---- end-to-end pass of the headline arm through the C ABI with host (pinned) buffers, on a fresh
    # context (the learned start's history and network must start over with the states)
    e2e = None
    if not args.no_e2e:
        ce = make_ctx(main_arm)
        for k in range(args.warmup):
            ce.time_step(dfs[k], w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit)
        dfs_h = [d.cpu().pin_memory() for d in dfs]
        u_host = torch.zeros(n, dtype=torch.float64).pin_memory()
        u_dev = torch.zeros(n, dtype=torch.float64, device=dev)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.warmup, n_total):
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
        for arm in ARMS:
            if arm == main_arm:
                continue
            c = make_ctx(arm)
            runs[arm] = timed_run(c)
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
    avg_f_ms = tm["f_apply_ms_total"] / max(tm["f_apply_launches"], 1)
    flops = tm["f_apply_flops"]
    byts = tm["f_apply_bytes"]
    achieved_tf = flops / (avg_f_ms * 1e-3) / 1e12 if avg_f_ms > 0 else None
    achieved_gbs = byts / (avg_f_ms * 1e-3) / 1e9 if avg_f_ms > 0 else None
    banded = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
              "frac": achieved_tf / FP64_PEAK_TFLOPS if achieved_tf else None,
              "traffic": measured_traffic("k_sub_solve", w.name),
              "kernel": "k_sub_solve (banded forward/backward substitution with the factor records, FP64)",
              "peak_kind": "measured FP64 FMA throughput (DFMA probe); nominal 1.25",
              "total_ms": tm["f_apply_ms_total"], "launches": tm["f_apply_launches"],
              "hbm": {"achieved_gbs": achieved_gbs, "peak_gbs": pk["hbm_gbs"],
                      "frac": achieved_gbs / pk["hbm_gbs"] if achieved_gbs else None,
                      "bytes_per_launch": byts, "flops_per_launch": flops, "avg_launch_ms": avg_f_ms,
                      "of": f"{pk_kind} hbm_gbs"}}
    schur = None
    if tm["schur_launches"] > 0 and tm["schur_ms_total"] > 0:
        s_tf = tm["schur_flops_total"] / (tm["schur_ms_total"] * 1e-3) / 1e12
        s_gbs = tm["schur_bytes_total"] / (tm["schur_ms_total"] * 1e-3) / 1e9
        schur = {"bound": "alu", "achieved": s_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                 "frac": s_tf / FP64_PEAK_TFLOPS, "traffic": None,
                 "kernel": "k_schur_dgemm (+ gather): Y = X S with the shape's FP64 dual Schur block",
                 "peak_kind": "measured FP64 FMA throughput (DFMA probe); nominal 1.25",
                 "total_ms": tm["schur_ms_total"], "launches": tm["schur_launches"],
                 "hbm": {"achieved_gbs": s_gbs, "peak_gbs": pk["hbm_gbs"], "frac": s_gbs / pk["hbm_gbs"],
                         "bytes_per_launch": tm["schur_bytes_total"] / tm["schur_launches"],
                         "flops_per_launch": tm["schur_flops_total"] / tm["schur_launches"],
                         "avg_launch_ms": tm["schur_ms_total"] / tm["schur_launches"],
                         "of": f"{pk_kind} hbm_gbs; bytes: the shared S (L2-resident) and X, Y"}}
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
                "inner_pcgp_launch": "kernel by kernel" if args.no_graphs else "one CUDA graph (WHILE node) per inner solve"},
            "e2e": e2e,
            "gpu_launches": int(tm["kernel_launches"]),
            "roofline": roof,
            "clocks": main["clocks"],
            "max_rel_u_diff_vs_fp64": max(main_d) if main_d else None,
            "solver": {"t_y": t_y, "plastic_gp_final": main["infos"][-1]["plastic_committed"],
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
        s = oracle_sample_subprocess(w.name)
        v = oracle_step_estimate(s, statistics.mean(x["newton"] for x in counts["infos"]),
                                 statistics.mean(sum(x["pcg"]) for x in counts["infos"]))
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                                "sample": s["sample"] + "; scaled with the FP64 arm's Newton/PCGP counts per step "
                                                        "(the oracle runs Algorithm 3 as printed)",
                                "components_s": {k: s[k] for k in ("assembly_s", "factor_s", "pcg_iter_s",
                                                                   "f_apply_s")}}
        if args.oracle_all_cores:
            sa = oracle_sample_all_cores(w.name)
            if sa is not None:
                va = oracle_step_estimate(sa, statistics.mean(x["newton"] for x in counts["infos"]),
                                          statistics.mean(sum(x["pcg"]) for x in counts["infos"]))
                line["cpu_baseline"]["all_cores"] = {
                    "value": va / sa["cores"], "unit": UNIT, "cores": sa["cores"], "per_core_step_s": va,
                    "kind": "oracle, one single-thread process per core",
                    "note": "the same sample run concurrently on every core; per-core step time / cores = the "
                            "oracle with its subdomain work split over all cores (lower bound)"}
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
    base = T.Context(w, stream=main_stream, precond=pre)
    streams = [torch.cuda.Stream(device=dev) for _ in cases]
    ctxs = [T.Context.case_of(base, c["sigma_y"], c["hardening"], stream=st) for c, st in zip(cases, streams)]

    def start(c):
        if arm != "fp64":
            c.set_precision(True, args.inner_rtol)
        if arm == "mixed_history":
            c.set_recycling(args.history)
        if arm == "mixed_learned":
            c.set_recycling(min(args.history, 7))
            c.set_learned(True)

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
    ap.add_argument("--steps", type=int, default=17)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", metavar="WORKLOAD", help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass (profiler runs)")
    ap.add_argument("--arm", default=None, choices=list(ARMS),
                    help="the headline (timed, end-to-end) arm; default mixed_learned, the metric's method")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="shorthand: fp64 = --arm fp64, mixed = --arm mixed (or mixed_learned with --learned)")
    ap.add_argument("--inner-rtol", type=float, default=1e-4,
                    help="relative residual reduction of each inner FP32 PCGP solve of the mixed arms")
    ap.add_argument("--no-mixed", action="store_true", help="time the headline arm only (no other arms)")
    ap.add_argument("--fapply", default="banded", choices=["banded", "schur"],
                    help="FP64 F-apply of elastic subdomains: shape's dual Schur block (DGEMM) or banded solves")
    ap.add_argument("--precond", default="lumped", choices=["lumped", "dirichlet"],
                    help="PCGP preconditioner of Sec. 4.2 (every arm)")
    ap.add_argument("--learned", action="store_true",
                    help="with --precision mixed: the learned start (mixed_learned arm)")
    ap.add_argument("--history", type=int, default=8,
                    help="stored dual solutions of the history start in the mixed+learned arm (1..8)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the mixed inner PCGP kernel by kernel instead of as one CUDA graph (for profilers)")
    ap.add_argument("--workload", default="cube64_8x8x8", choices=sorted(W.WORKLOADS),
                    help="cube64_8x8x8 is the benchmark; smaller cases exist for profiler captures")
    ap.add_argument("--oracle-all-cores", action="store_true",
                    help="also time the oracle sample on every host core at once (cpu_baseline.all_cores)")
    ap.add_argument("--cases", type=int, default=0,
                    help="N > 0: N load cases on one mesh stepped concurrently (case contexts), one JSON line")
    ap.add_argument("--case-set", default="directions", choices=["directions", "seeded"],
                    help="directions: theta_k = 2 pi k / N, the Sec. 5 material; seeded: sigma_y, H and the "
                         "direction drawn per case")
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(W.WORKLOADS[args.oracle_sample])))
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
