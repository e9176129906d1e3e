"""Benchmark of the H-LU setup with accumulated updates on GB300.

One step = one H-LU factorisation (the whole hot path: accumulated products,
truncations, flushes, leaf LU/TRSM) of the workload's matrix, starting from a
fresh device copy of the unfactored H-matrix.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, serial FP64) on a bounded
sample of the workload instead.  Under torchrun every rank factors its own
replica (the path does not shard); rank 0 prints the line.
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

import hmat_synth as hs  # noqa: E402

METRIC = "H-LU setup truncations/s (accumulated updates) vs plain FP64 at equal ||I-(LU)^-1 A||"
UNIT = "truncations/s"
TASK_NAMES = ["NOP", "LU", "TRSM", "HMV", "DENSIFY", "GEMM", "ADD", "RKADD", "ROWMERGE", "COPY", "ZERO", "RANKSET",
              "INV", "CHOL"]
FP64_PEAK_TFLOPS = 1.25     # GB300 nominal FP64 (vector and tensor) rate, 152 SMs at up to 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 CUDA-core FMA rate: 152 SMs x 128 lanes x 2 x 2070 MHz
WORKLOADS = {"laplace3d_32": hs.laplace3d_32, "laplace3d_64": hs.laplace3d_64, "laplace2d_64": hs.laplace2d_64,
             "diffusion2d_batch64": hs.diffusion2d_batch,
             # small case of the 3D recipe for profiling captures
             "laplace3d_16": lambda: hs.small_laplace(16, 3, 64, 1e-4),
             # the stress case: 80^3 variable-coefficient diffusion, two tolerances, PCG check
             "diffusion3d_80": lambda: hs.diffusion3d_80(1e-3),
             "diffusion3d_80_eps1e-5": lambda: hs.diffusion3d_80(1e-5)}
PCG_WORKLOADS = ("diffusion3d_80", "diffusion3d_80_eps1e-5")
# bounded oracle sample: the same operator family, tolerance and leaf size at 16^3
SAMPLE = {"laplace3d_32": lambda: hs.small_laplace(16, 3, 64, 1e-4),
          "laplace3d_16": lambda: hs.small_laplace(16, 3, 64, 1e-4),
          "laplace3d_64": lambda: hs.small_laplace(16, 3, 64, 1e-4),
          "laplace2d_64": hs.laplace2d_64,
          "diffusion2d_batch64": lambda: hs.diffusion2d_batch()[0],
          "diffusion3d_80": lambda: hs.Problem("diffusion3d_16", 16, 3, 64, 2.0, 1e-3, kind="diffusion", lc=0.05,
                                               seed=4),
          "diffusion3d_80_eps1e-5": lambda: hs.Problem("diffusion3d_16", 16, 3, 64, 2.0, 1e-5, kind="diffusion",
                                                       lc=0.05, seed=4)}


T_START = time.time()
FALLBACK_HBM_GBS = 6800.0  # an earlier GB300 measurement, used only without the measured peaks file
# plain FP64 factorisation time over the mixed one, for the time guard of the
# comparator (measured at 64^3; a guess errs towards skipping)
FP64_OVER_MIXED = 12.0
STANDARD_OVER_ACC = 3.0  # the same for the standard form (the paper: factor 2 to 3)
TRAFFIC_NOTE = ("DRAM read + write bytes of one launch from an ncu capture of this source tree (profiles/), "
                "scaled by the truncations where the capture is of a smaller case; null when the kernel source "
                "changed since")


def oracle_values(workload: str):
    """The oracle's stored values for the workload (tests/golden/, written by
    a script that calls only the oracle), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{workload}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    return {k: d[k] for k in ("precond_error", "truncations", "mean_rank", "blocktree_sha256", "oracle_lu_seconds",
                              "oracle_cores") if k in d} | {"source": os.path.relpath(path, ROOT)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_sample(workload: str, min_seconds: float = 10.0) -> dict:
    """The oracle as it stands, serial, on the bounded sample, repeated until
    at least min_seconds of CPU work."""
    import oracle
    oracle.build()
    p = SAMPLE[workload]()
    trunc = 0
    el = 0.0
    runs = 0
    while el < min_seconds or runs == 0:
        ct, bt, csr, H = oracle.setup(p)
        oracle.stats_reset()
        t0 = time.perf_counter()
        H.lu(p.eps, True)
        el += time.perf_counter() - t0
        trunc += oracle.stats()["truncations"]
        runs += 1
    return {"value": trunc / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{runs} x serial FP64 oracle H-LU (accumulated) of {p.name} (n={p.n}, leaf {p.leaf}, "
                      f"eps {p.eps:g}), {el:.1f} s, {trunc} truncations"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6), ("sw_thermal_slowdown", 7),
                              ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows)}


def instance_cost(n: int) -> float:
    """Work model of one instance's H-LU for the partition: n log2(n)^2."""
    return n * math.log2(max(n, 2)) ** 2


def lpt_partition(costs, world: int):
    """Greedy longest-processing-time assignment: instances in decreasing
    cost, each to the rank with the least load so far (ties: lowest rank).
    Returns the instance indices of every rank (ascending)."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def rank_problems(workload: str, rank: int, world: int = 1):
    """This rank's problems.  A single H-LU does not shard, so every rank
    factors a replica of it.  The batch workload's 64 independent instances
    are split over the ranks by LPT on n log2(n)^2, with no exchange."""
    if workload == "diffusion2d_batch64":
        probs = hs.diffusion2d_batch(64, seed=2)
        part = lpt_partition([instance_cost(p.n) for p in probs], world)[rank]
        return [probs[i] for i in part]
    w = WORKLOADS[workload]()
    return w if isinstance(w, list) else [w]


def job_throughput(units: float, seconds: float, world: int, device=None):
    """(units of all ranks / the slowest rank's time, that time)."""
    if world > 1:
        import torch
        u = torch.tensor([float(units)], dtype=torch.float64, device=device)
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(u, op=torch.distributed.ReduceOp.SUM)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        units, seconds = float(u.item()), float(t.item())
    return units / seconds, seconds


# DRAM bytes (read + write) of one exec_tasks launch, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the source tree whose
# csrc hash is given; see profiles/launches_laplace3d_32.md.
# The 64^3 figure scales the 32^3 capture by the truncations per launch
# (621 514 / 34 684): ncu's device-memory save and restore of a 52 GB launch
# is beyond a capture that ends by itself.
TRAFFIC = {"laplace3d_32": {"csrc": "a7e1365b93d004b9", "bytes": 5842257920 + 15209673472},
           "laplace3d_64": {"csrc": "a7e1365b93d004b9", "bytes": round((5842257920 + 15209673472) * 621514 / 34684)}}


def csrc_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1703_09085_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def traffic_per_launch(workload: str):
    rec = TRAFFIC.get(workload)
    return rec["bytes"] if rec and rec["csrc"] == csrc_hash() else None


def train_predictor(g, ctx):
    """The rank predictor trained as the 64^3 configuration asks: (features,
    rank) pairs of the exact truncations of plain FP64 H-LUs of the smaller
    configurations (the 64^2 Laplacian, the 32^3 Laplacian, the first four
    instances of the diffusion batch), then Adam on the GPU."""
    t0 = time.perf_counter()
    Xs, ys = [], []
    for p in [hs.laplace2d_64(), hs.laplace3d_32()] + list(hs.diffusion2d_batch()[:4]):
        ct = g.ClusterTree(ctx, p.coords(), p.leaf)
        bt = g.BlockTree(ctx, ct, ct, p.eta)
        H = g.HMatrix(ctx, bt, p.matrix())
        H.lu(p.eps, record_training=True)
        X, y = H.training_data()
        Xs.append(X)
        ys.append(y)
    X, y = np.concatenate(Xs), np.concatenate(ys)
    P = g.RankPredictor(ctx, seed=7)
    loss0, _ = P.grad(X, y)
    loss = P.train(X, y, epochs=60, batch=256, lr=3e-3, seed=3)
    return P, {"pairs": int(len(y)), "sources": "FP64 H-LUs of laplace2d_64, laplace3d_32, diffusion batch 0-3",
               "loss_before": float(loss0), "loss_after": float(loss), "seconds": time.perf_counter() - t0}


def workload_config(args, probs, world: int) -> dict:
    """The config object of both arms' JSON lines."""
    par = (f"instances sharded: 64 instances over {world} rank(s) by LPT on n log2(n)^2"
           if args.workload == "diffusion2d_batch64" else f"replicas{world}")
    return {"workload": args.workload, "instances": len(probs), "n": sum(p.n for p in probs), "leaf": probs[0].leaf,
            "eta": probs[0].eta, "eps": probs[0].eps, "precision": args.precision,
            "max_rank": args.max_rank or 64, "l2": "flushed between steps (256 MiB write)",
            "parallelism": par, "rank_predictor": "on" if getattr(args, "predictor", False) else "off"}


def run_reference_hmul(args) -> None:
    """The oracle's accumulated H-mult Z <- A - X X on a 16^3 sample, as the
    reference arm of the H-mult workload."""
    import oracle
    oracle.build()
    q = hs.small_laplace(16, 3, 64, 1e-4)
    times, truncs = [], []
    for i in range(args.warmup + args.steps):
        oct_, obt, ocsr, OX = oracle.setup(q)
        OX.lu(q.eps, True)
        OZ = oracle.HMatrix.from_csr(obt, ocsr)
        oracle.stats_reset()
        t0 = time.perf_counter()
        oracle.hmul(-1.0, OX, OX, OZ, q.eps, accumulated=True)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(el)
            truncs.append(oracle.stats()["truncations"])
    value = sum(truncs) / sum(times)
    p = hs.laplace3d_32()
    line = {"impl": "reference", "metric": HMUL_METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": p.n, "leaf": p.leaf, "eta": p.eta, "eps": p.eps,
                       "operand": "X = H-LU factors (eps 1e-4) of the 32^3 Laplacian, Z = A",
                       "precision": args.precision, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "replicas1"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step one serial FP64 oracle H-mult (accumulated) of {q.name} "
                                       f"(n={q.n}), the same recipe at a size the oracle finishes in seconds"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    if args.workload == "hmul_3d32":
        run_reference_hmul(args)
        return
    p = SAMPLE[args.workload]()
    # the sample's own configuration: the oracle runs a smaller case of the
    # same recipe, so this line is not the GPU line's problem size
    cfg = {"workload": p.name, "n": p.n, "leaf": p.leaf, "eta": p.eta, "eps": p.eps, "sample_of": args.workload,
           "precision": "fp64", "parallelism": "1 host core"}
    import oracle
    oracle.build()
    times, truncs = [], []
    for i in range(args.warmup + args.steps):
        ct, bt, csr, H = oracle.setup(p)
        oracle.stats_reset()
        t0 = time.perf_counter()
        H.lu(p.eps, True)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(el)
            truncs.append(oracle.stats()["truncations"])
    value = sum(truncs) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step one serial FP64 oracle H-LU (accumulated) of {p.name} "
                                       f"(n={p.n}, leaf {p.leaf}, eps {p.eps:g}), the same recipe at a size "
                                       f"the oracle finishes in seconds"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank: int, world: int, local_rank: int) -> None:
    import torch
    import paper_1703_09085_gb300 as g
    from paper_1703_09085_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    probs = rank_problems(args.workload, rank, world)
    eps = probs[0].eps
    assert all(p.eps == eps for p in probs)
    csrs = [p.matrix() for p in probs]
    ctx = g.Context(local_rank, stream)
    t0 = time.perf_counter()
    cts = [g.ClusterTree(ctx, p.coords(), p.leaf) for p in probs]
    bts = [g.BlockTree(ctx, ct, ct, p.eta) for ct, p in zip(cts, probs)]
    tree_s = time.perf_counter() - t0
    pristine = [g.HMatrix(ctx, bt, c) for bt, c in zip(bts, csrs)]
    work = [g.HMatrix(ctx, bt, c) for bt, c in zip(bts, csrs)]
    flush = torch.empty(int(256 * 2**20) // 4, dtype=torch.float32, device=dev)
    prec = g.HMAT_MIXED if args.precision == "mixed" else g.HMAT_FP64
    predictor, pred_info = train_predictor(g, ctx) if args.predictor else (None, None)

    def step(precision=prec, mode=g.HMAT_ACCUMULATED):
        for wk, pr in zip(work, pristine):
            wk.copy_values_from(pr)
        if args.op == "lu":
            g.lu_batched(ctx, work, eps, max_rank=args.max_rank, precision=precision, reuse_schedule=True, mode=mode,
                         predictor=predictor if precision == prec else None)
        else:  # H-Cholesky or H-inversion: the schedule is built in every call, inside the step
            for wk in work:
                getattr(wk, args.op)(eps, max_rank=args.max_rank, precision=precision)

    sched_first = None
    for i in range(args.warmup):
        step()
        if i == 0:
            # the LU's timed steps reuse this schedule, so its pass is added to
            # every step; the other operations build theirs inside the step
            sched_first = work[0].stats()["schedule_seconds"] if args.op == "lu" else 0.0
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms, flops, flops32, truncs, tasks, sched, nbytes = [], [], [], [], [], [], [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        st = work[0].stats()  # batch totals
        kern_ms.append(1e3 * st["factor_seconds"])
        flops.append(st["flops"])
        flops32.append(st["flops32"])
        nbytes.append(st["bytes"])
        truncs.append(st["truncations"])
        tasks.append(st["tasks"])
        sched.append(st["schedule_seconds"])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    # the symbolic pass (host) of the first call counted in every step, so that
    # the headline is the whole setup; the kept schedule saves it in practice
    # when the same sparsity pattern is factored again
    value, total_s = job_throughput(sum(truncs), sum(step_ms) / 1e3 + args.steps * sched_first, world, dev)
    value_numeric, _ = job_throughput(sum(truncs), sum(step_ms) / 1e3, world, dev)
    st = work[0].stats()

    # end to end through the public API with host buffers: CSR -> device,
    # factorisation, ranks back to the host, every step
    h2d = sum(8 * (c.rowptr.size + c.colidx.size + c.val.size) + 16 * c.n for c in csrs)
    d2h = sum(8 * g.lib().hmat_blocktree_size(bt.h) for bt in bts)
    e2e_times = []
    e2e_steps = 0 if args.no_e2e else min(args.steps, 2)
    for i in range(1 + e2e_steps if e2e_steps else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Hs = [g.HMatrix(ctx, bt, c) for bt, c in zip(bts, csrs)]
        if args.op == "lu":
            g.lu_batched(ctx, Hs, eps, max_rank=args.max_rank, precision=prec, predictor=predictor)
        else:
            for H in Hs:
                getattr(H, args.op)(eps, max_rank=args.max_rank, precision=prec)
        for H in Hs:
            H.ranks()
        torch.cuda.synchronize()
        if i >= 1:
            e2e_times.append(time.perf_counter() - t0)
        del Hs
    e2e_value, e2e_s = (job_throughput(statistics.mean(truncs) * e2e_steps, sum(e2e_times), world, dev)
                        if e2e_steps else (None, None))

    if rank != 0:
        return
    # preconditioner quality of the last factorisation (power iteration with the
    # GPU solves); batches report their first instances
    nq = min(len(probs), 4)
    # (the LU solve measures the LU factors; the other operations' quality is
    # checked against the oracle by the tests)
    perr = [precond_error(g, work[i], cts[i], csrs[i], probs[i]) for i in range(nq)] if args.op == "lu" else [None]
    types = {name: {"count": st["type_count"][i], "cta_s": st["type_seconds"][i]}
             for i, name in enumerate(TASK_NAMES) if st["type_count"][i]}
    pcg = None
    if args.workload in PCG_WORKLOADS and args.op == "lu":
        # 8 seeded N(0, 1) right-hand sides (seed 4), FP64 CG to 1e-10
        p0 = probs[0]
        B = np.stack([hs.normal(4 + c, p0.n) for c in range(8)])  # (8, n), original ordering
        Bt = torch.from_numpy(B).to(dev)
        Xt = torch.zeros_like(Bt)
        t0 = time.perf_counter()
        its, res = work[0].pcg(csrs[0], Bt, Xt, rtol=1e-10, maxit=1000)
        pcg = {"rhs": 8, "rtol": 1e-10, "iterations": [int(x) for x in its], "rel_residual": [float(x) for x in res],
               "seconds": time.perf_counter() - t0}
    # the plain FP64 accumulated form on the same GPU, same matrices: the comparator
    fp64 = None
    est = FP64_OVER_MIXED * statistics.mean(step_ms) / 1e3
    if args.op != "lu":
        fp64 = None
    elif args.precision == "mixed" and not args.no_fp64 and time.time() - T_START + est > args.time_budget:
        fp64 = {"skipped": f"the plain FP64 factorisation (about {est:.0f} s) would end past the bench's time "
                           f"budget of {args.time_budget:.0f} s"}
    elif args.precision == "mixed" and not args.no_fp64:
        ev0.record(stream)
        step(g.HMAT_FP64)
        ev1.record(stream)
        ev1.synchronize()
        s64 = work[0].stats()
        fp64 = {"setup_s": ev0.elapsed_time(ev1) / 1e3, "truncations": s64["truncations"],
                "value": s64["truncations"] / (ev0.elapsed_time(ev1) / 1e3),
                "precond_error": [precond_error(g, work[i], cts[i], csrs[i], probs[i]) for i in range(nq)],
                "kernel_s": s64["factor_seconds"], "flops": s64["flops"]}
        fp64["schedule_s"] = s64["schedule_seconds"]
        fp64["note"] = "setup_s includes this first FP64 call's symbolic pass (inside the events)"
        fp64["speedup_of_chosen_form"] = fp64["setup_s"] / (statistics.mean(step_ms) / 1e3 + sched_first)
    # the standard form (every product applied at once, Section 4) in the
    # chosen precision: the paper's comparison, time and truncations
    standard = None
    est = STANDARD_OVER_ACC * statistics.mean(step_ms) / 1e3
    if args.op != "lu":
        standard = None
    elif not args.no_standard and time.time() - T_START + est > args.time_budget:
        standard = {"skipped": f"the standard-form factorisation (about {est:.0f} s) would end past the bench's "
                               f"time budget of {args.time_budget:.0f} s"}
    elif not args.no_standard:
        ev0.record(stream)
        step(prec, g.HMAT_STANDARD)
        ev1.record(stream)
        ev1.synchronize()
        sstd = work[0].stats()
        t_std = ev0.elapsed_time(ev1) / 1e3
        # (its first call builds its schedule inside the events)
        standard = {"setup_s": t_std, "numeric_s": t_std - sstd["schedule_seconds"],
                    "schedule_s": sstd["schedule_seconds"], "truncations": sstd["truncations"],
                    "precond_error": [precond_error(g, work[i], cts[i], csrs[i], probs[i]) for i in range(nq)],
                    "time_ratio_standard_over_accumulated": t_std / (statistics.mean(step_ms) / 1e3 + sched_first),
                    "truncation_ratio_standard_over_accumulated": sstd["truncations"] / statistics.mean(truncs)}
    peaks = measured_peaks()
    avg_kern_s = statistics.mean(kern_ms) / 1e3
    achieved = statistics.mean(flops) / avg_kern_s / 1e12
    achieved32 = statistics.mean(flops32) / avg_kern_s / 1e12
    hbm_peak = peaks.get("hbm_gbs") or FALLBACK_HBM_GBS
    achieved_gbs = statistics.mean(nbytes) / avg_kern_s / 1e9
    ref = oracle_values(args.workload)
    line = {
        "metric": OP_METRIC[args.op], "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms) + 1e3 * sched_first, "higher_is_better": True,
        "scaling": "strong" if args.workload == "diffusion2d_batch64" else "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": workload_config(args, probs, world),
        "setup_s": statistics.mean(step_ms) / 1e3 + sched_first,
        "numeric_s": statistics.mean(step_ms) / 1e3,
        "value_numeric_only": value_numeric,
        "truncations_per_step": int(statistics.mean(truncs)),
        "tasks_per_step": int(statistics.mean(tasks)),
        "schedule_s": statistics.mean(sched),
        "schedule_s_first_call": sched_first,
        "schedule_note": ("setup_s and value include the first call's symbolic pass in every step (the timed "
                          "numeric steps reuse its schedule); e2e builds it every step") if args.op == "lu" else
                         "the operation builds its schedule in every call, inside the timed step",
        "tree_build_s": tree_s,
        "precond_error": perr if len(probs) > 1 else perr[0],
        "oracle": ref if args.op == "lu" else None,
        "pcg": pcg,
        "randomised_truncations": st["rand_truncations"], "randomised_fallbacks": st["rand_fallbacks"],
        "sketch_attempts": st["sketch_attempts"], "sketch_columns": st["sketch_columns"],
        "rank_predictor": pred_info,
        "plain_fp64": fp64,
        "standard_form": standard,
        "task_types": types,
        "critical_path_tasks": st["levels"],
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved_gbs / hbm_peak, "traffic": traffic_per_launch(args.workload),
                     "kernel": "exec_tasks", "kernel_ms": statistics.mean(kern_ms),
                     "bytes_per_launch": statistics.mean(nbytes),
                     "peak_note": ("measured" if peaks.get("hbm_gbs") else "fallback") + " HBM copy bandwidth; "
                                  "achieved = algorithmic bytes per launch (counted on the device per task: "
                                  "8 [(m + n) l + (m + n) k] per truncation, leaves and thin blocks read and "
                                  "written once) / the launch's CUDA-event time",
                     "fp64": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": achieved / FP64_PEAK_TFLOPS, "flops_per_launch": statistics.mean(flops)},
                     "fp32": {"bound": "alu", "achieved": achieved32, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": achieved32 / FP32_PEAK_TFLOPS, "flops_per_launch": statistics.mean(flops32)},
                     "alu_peak_note": "nominal FP64 (1.25 TFLOP/s) and FP32 (152 SMs x 128 lanes x 2 x 2070 MHz) "
                                      "rates: the measured peaks file has no FP64 or FP32 vector figure",
                     "traffic_note": TRAFFIC_NOTE},
        "e2e": ({"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                 "ms_per_step": 1e3 * e2e_s / e2e_steps, "steps": e2e_steps} if e2e_steps else
                {"skipped": "--no-e2e: a second factorisation beside the kept schedule does not fit in device "
                            "memory at this size"}),
        "clocks": clk,
        "device_bytes": st["device_bytes"],
        "bench_wall_s": time.time() - T_START,
        "peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")},
    }
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_sample(args.workload)
    print(json.dumps(line), flush=True)


OP_METRIC = {"lu": METRIC, "cholesky": "H-Cholesky setup truncations/s (accumulated updates)",
             "invert": "H-inversion truncations/s (accumulated updates, Fig. invert)"}


HMUL_METRIC = "H-matrix multiplication Z <- blocktrunc(Z - X Y) truncations/s (accumulated updates) vs plain FP64"


def run_hmul(args, rank: int, world: int, local_rank: int) -> None:
    """H x H multiplication (hmat_addmul) on the factors of a 3D H-LU:
    Z <- blocktrunc(A - X X), X = the H-LU of the 32^3 Laplacian (L and U in
    one H-matrix), Z starting from A.  Each step restores Z and multiplies;
    the symbolic pass runs in every step (hmat_addmul keeps no schedule)."""
    import torch
    import paper_1703_09085_gb300 as g
    from paper_1703_09085_gb300 import build
    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    p = hs.laplace3d_32()
    csr = p.matrix()
    ctx = g.Context(local_rank, stream)
    ct = g.ClusterTree(ctx, p.coords(), p.leaf)
    bt = g.BlockTree(ctx, ct, ct, p.eta)
    prec = g.HMAT_MIXED if args.precision == "mixed" else g.HMAT_FP64
    X = g.HMatrix(ctx, bt, csr)
    X.lu(p.eps, precision=g.HMAT_MIXED)  # the operand: the H-LU factors (setup, untimed)
    Z0 = g.HMatrix(ctx, bt, csr)
    Z = g.HMatrix(ctx, bt, csr)
    flush = torch.empty(int(256 * 2**20) // 4, dtype=torch.float32, device=dev)

    def step(precision=prec, mode=g.HMAT_ACCUMULATED):
        Z.copy_values_from(Z0)
        g.addmul(ctx, -1.0, X, X, Z, p.eps, max_rank=args.max_rank, precision=precision, mode=mode)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms, flops, flops32, truncs, sched = [], [], [], [], [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        st = Z.stats()
        kern_ms.append(1e3 * st["factor_seconds"])
        flops.append(st["flops"])
        flops32.append(st["flops32"])
        truncs.append(st["truncations"])
        sched.append(st["schedule_seconds"])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    value, _ = job_throughput(sum(truncs), sum(step_ms) / 1e3, world, dev)
    st = Z.stats()
    # end to end: Z from the host CSR arrays, the product, ranks back
    h2d = 8 * (csr.rowptr.size + csr.colidx.size + csr.val.size) + 16 * csr.n
    d2h = 8 * g.lib().hmat_blocktree_size(bt.h)
    e2e_times = []
    for i in range(1 + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ze = g.HMatrix(ctx, bt, csr)
        g.addmul(ctx, -1.0, X, X, Ze, p.eps, max_rank=args.max_rank, precision=prec)
        Ze.ranks()
        torch.cuda.synchronize()
        if i >= 1:
            e2e_times.append(time.perf_counter() - t0)
        del Ze
    e2e_value, e2e_s = job_throughput(sum(truncs), sum(e2e_times), world, dev)
    if rank != 0:
        return

    def rel_error(Zm):
        # ||(Z - (A - X X)) v|| / ||(A - X X) v|| for 4 seeded vectors (cluster order)
        perm = ct.perm()
        V = np.stack([hs.start_vector(p.n, 10 + j) for j in range(4)])  # (4, n), original order
        Vp = V[:, perm]
        tv = torch.from_numpy(np.ascontiguousarray(Vp)).cuda()
        xv = torch.zeros_like(tv)
        X.addeval(1.0, tv, xv)
        xxv = torch.zeros_like(tv)
        X.addeval(1.0, xv, xxv)
        zv = torch.zeros_like(tv)
        Zm.addeval(1.0, tv, zv)
        av = np.stack([csr.matvec(V[j])[perm] for j in range(4)])
        ref = av - xxv.cpu().numpy()
        return float(np.linalg.norm(zv.cpu().numpy() - ref) / np.linalg.norm(ref))

    err = rel_error(Z)
    fp64 = None
    est = FP64_OVER_MIXED * statistics.mean(step_ms) / 1e3
    if args.op != "lu":
        fp64 = None
    elif args.precision == "mixed" and not args.no_fp64 and time.time() - T_START + est > args.time_budget:
        fp64 = {"skipped": f"the plain FP64 factorisation (about {est:.0f} s) would end past the bench's time "
                           f"budget of {args.time_budget:.0f} s"}
    elif args.precision == "mixed" and not args.no_fp64:
        ev0.record(stream)
        step(g.HMAT_FP64)
        ev1.record(stream)
        ev1.synchronize()
        s64 = Z.stats()
        fp64 = {"ms": ev0.elapsed_time(ev1), "truncations": s64["truncations"],
                "value": s64["truncations"] / (ev0.elapsed_time(ev1) / 1e3), "rel_error": rel_error(Z)}
        fp64["speedup_of_chosen_form"] = fp64["ms"] / statistics.mean(step_ms)
    # the standard multiplication (every product applied at once) in the
    # chosen precision: the paper's Exp. 1 comparison
    standard = None
    if not args.no_standard:
        ev0.record(stream)
        step(prec, g.HMAT_STANDARD)
        ev1.record(stream)
        ev1.synchronize()
        sst = Z.stats()
        standard = {"ms": ev0.elapsed_time(ev1), "truncations": sst["truncations"], "rel_error": rel_error(Z),
                    "time_ratio_standard_over_accumulated": ev0.elapsed_time(ev1) / statistics.mean(step_ms),
                    "truncation_ratio_standard_over_accumulated": sst["truncations"] / statistics.mean(truncs)}
    avg_kern_s = statistics.mean(kern_ms) / 1e3
    achieved = statistics.mean(flops) / avg_kern_s / 1e12
    achieved32 = statistics.mean(flops32) / avg_kern_s / 1e12
    line = {
        "metric": HMUL_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": args.workload, "n": p.n, "leaf": p.leaf, "eta": p.eta, "eps": p.eps,
                   "operand": "X = H-LU factors (eps 1e-4) of the 32^3 Laplacian, Z = A",
                   "precision": args.precision, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas{world}"},
        "truncations_per_step": int(statistics.mean(truncs)), "schedule_s": statistics.mean(sched),
        "rel_error": err, "plain_fp64": fp64, "standard_form": standard, "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "exec_tasks",
                     "fp32": {"achieved": achieved32, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": achieved32 / FP32_PEAK_TFLOPS}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": 1e3 * e2e_s / args.steps},
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        q = hs.small_laplace(16, 3, 64, 1e-4)
        t_all, n_tr, runs = 0.0, 0, 0
        while t_all < 10.0 and runs < 20:
            oct_, obt, ocsr, OX = oracle.setup(q)
            OX.lu(q.eps, True)
            OZ = oracle.HMatrix.from_csr(obt, ocsr)
            oracle.stats_reset()
            t0 = time.perf_counter()
            oracle.hmul(-1.0, OX, OX, OZ, q.eps, accumulated=True)
            t_all += time.perf_counter() - t0
            n_tr += oracle.stats()["truncations"]
            runs += 1
        line["cpu_baseline"] = {"value": n_tr / t_all, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{runs} x serial FP64 oracle H-mult (accumulated) Z <- A - X X of "
                                          f"{q.name} (n={q.n}), {t_all:.1f} s, {n_tr} truncations"}
    print(json.dumps(line), flush=True)


def precond_error(g, H, ct, csr, p, maxit=50, rtol=1e-3) -> float:
    import torch
    perm = ct.perm()
    v = hs.start_vector(p.n, 0)[perm]
    v = v / np.linalg.norm(v)

    def Ap(x):
        y = np.zeros(p.n)
        y[perm] = x
        return csr.matvec(y)[perm]

    def solve(b, trans):
        t = torch.from_numpy(b.copy()).cuda()
        H.solve(t, trans=trans)
        return t.cpu().numpy()

    est = 0.0
    for it in range(maxit):
        w = v - solve(Ap(v), False)
        new = float(np.linalg.norm(w))
        z = w - Ap(solve(w, True))
        done = it > 0 and abs(new - est) <= rtol * new
        est = new
        nz = np.linalg.norm(z)
        if nz == 0 or done:
            break
        v = z / nz
    return est


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="laplace3d_64", choices=sorted(WORKLOADS) + ["hmul_3d32"])
    ap.add_argument("--max-rank", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparator")
    ap.add_argument("--no-standard", action="store_true", help="skip the standard-form comparator")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end steps (largest workloads)")
    ap.add_argument("--predictor", action="store_true",
                    help="train the rank predictor on the smaller configurations' pairs and use it in the timed steps")
    ap.add_argument("--op", default="lu", choices=["lu", "cholesky", "invert"],
                    help="the operation timed on an LU workload: H-LU (default), H-Cholesky or H-inversion")
    ap.add_argument("--time-budget", type=float, default=1650.0,
                    help="seconds after which the optional comparators are skipped")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "hmul_3d32":
            run_hmul(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
