"""Benchmark of one CPRA training step on GB300 (edge*shot*steps/s).

Workload (default): MIS on a seeded random 5-regular graph with N = 10^6
nodes (nnz = 2|E| = 5*10^6), S = 256 penalty shots with lambda_s log-spaced
0.5..10, a two-layer GCN of width 128 with BF16 dense layers (FP32 loss,
Adam and rounding).  A step is the whole hot path: forward, fused SpMM +
loss, adjoint, Adam, rounding and exact integer evaluation of all shots.
Inputs are larger than L2 (P alone is N*S*4 = 1.0 GB), so no L2 flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

prints one JSON line.  The reference arm times the FP64 CPU oracle.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

if "reference" in sys.argv:
    # the CPU reference arm runs single-threaded so its core count is exact
    # (set before numpy loads its BLAS)
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2402_02190_gb300 import inputs as I  # noqa: E402

METRIC = "edge·shot·steps/s"

WORKLOADS = {
    # name: (graph, N, degree, seed, problem, S, H, lambda, nu, precision, diversity
    # form, recompute); the N = 10^6 and the max-cut shapes recompute the
    # layer-1 ReLU mask in the backward instead of keeping the activations.
    "mis_rrg5_n1e6_s256_h128_bf16": dict(graph="rrg", N=10**6, d=5, seed=5, problem=0, S=256,
                                         H=128, lam=("geom", 0.5, 10.0), nu=0.0, precision=1,
                                         div=0, recompute=1),
    "mis_rrg5_n1e6_s256_h128_fp32": dict(graph="rrg", N=10**6, d=5, seed=5, problem=0, S=256,
                                         H=128, lam=("geom", 0.5, 10.0), nu=0.0, precision=0,
                                         div=0, recompute=1),
    # same shape at N/5 (P = 205 MB, still larger than L2): the small case
    # for full ncu captures
    "mis_rrg5_n2e5_s256_h128_bf16": dict(graph="rrg", N=2 * 10**5, d=5, seed=5, problem=0, S=256,
                                         H=128, lam=("geom", 0.5, 10.0), nu=0.0, precision=1,
                                         div=0, recompute=1),
    "mis_rrg5_n2e5_s256_h128_fp32": dict(graph="rrg", N=2 * 10**5, d=5, seed=5, problem=0, S=256,
                                         H=128, lam=("geom", 0.5, 10.0), nu=0.0, precision=0,
                                         div=0, recompute=1),
    "mis_rrg20_n1e4_s100_h256_bf16": dict(graph="rrg", N=10**4, d=20, seed=2, problem=0, S=100,
                                          H=256, lam=("geom", 0.5, 10.0), nu=0.0, precision=1,
                                          div=0, recompute=0),
    "maxcut_er10_n1e5_s64_h128_bf16": dict(graph="er", N=10**5, d=10, seed=3, problem=1, S=64,
                                           H=128, lam=None, nu=0.1, precision=1, div=1,
                                           recompute=1),
    "mis_rrg3_n100_s8_h16_fp32": dict(graph="rrg", N=100, d=3, seed=1, problem=0, S=8, H=16,
                                      lam=("lin", 1.0, 8.0), nu=0.0, precision=0, div=0,
                                      recompute=0),
}
DEFAULT_WORKLOAD = "mis_rrg5_n1e6_s256_h128_bf16"
# Bounded CPU sample for the oracle: the same degree, width and shots on a
# graph of 2,500 nodes (about 0.25 s per single-threaded FP64 step).
CPU_SAMPLE_N = 2500


def make_graph(w):
    if w["graph"] == "rrg":
        return I.random_regular_graph(w["N"], w["d"], w["seed"])
    return I.erdos_renyi_graph(w["N"], w["d"] / (w["N"] - 1), w["seed"])


def make_lambda(w):
    if w["lam"] is None:
        return None
    kind, lo, hi = w["lam"]
    return I.lambda_geomspace(lo, hi, w["S"]) if kind == "geom" else I.lambda_linspace(lo, hi, w["S"])


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` at `workload` from its committed ncu
    summary, if that was taken on the current kernel source; else None.
    Returns (bytes, basis): the summary's DRAM capture is taken on a smaller
    case of the same kernel and scaled by the units (node rows) processed."""
    p = os.path.join(ROOT, "profiles", f"{kernel}__{workload}.md")
    if not os.path.exists(p):
        return None, None
    fields = {}
    for line in open(p):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    src = os.path.join(ROOT, "paper_2402_02190_gb300", "csrc", fields.get("source", "k_loss.cu"))
    if not os.path.exists(src):
        return None, None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if fields.get("source_sha256_16") != sha:
        return None, None
    try:
        return float(fields["dram_bytes_per_launch"]), fields.get("traffic_basis")
    except (KeyError, ValueError):
        return None, None


def max_over_ranks(x: float, dist_mod=None, device="cuda") -> float:
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if dist_mod is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job rate of `world` independent replicas that each processed
    units_per_rank units, timed by the slowest rank."""
    return world * units_per_rank / seconds


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def loss_kernel_bytes(N, nnz, S, g_bytes):
    """Algorithmic bytes of one fused SpMM + loss launch: neighbour-row
    gathers nnz*S*4, own P row N*S*4, G write N*S*g_bytes, CSR 4(N+1)+4nnz,
    rounded bits N*ceil(S/32)*4."""
    return nnz * S * 4 + N * S * 4 + N * S * g_bytes + 4 * (N + 1) + 4 * nnz + N * ((S + 31) // 32) * 4


def loss_compulsory_bytes(N, nnz, S, g_bytes):
    """The same launch's compulsory bytes: every input read once (P, CSR) and
    every output written once (G, bits), as if every neighbour row were
    served from on-chip memory."""
    return N * S * 4 + N * S * g_bytes + 4 * (N + 1) + 4 * nnz + N * ((S + 31) // 32) * 4


# ---------------------------------------------------------------- CPU oracle
def oracle_steps(w, n_nodes, steps, seed=0):
    """Runs `steps` FP64 oracle steps on the bounded sample; returns
    (seconds, nnz, S)."""
    from oracle import cpra_oracle as O
    ws = dict(w, N=n_nodes)
    rp, col = make_graph(ws)
    g = O.Graph(rp, col)
    S, H = w["S"], w["H"]
    lam = make_lambda(w)
    theta, X0 = I.seeded_params(n_nodes, H, H, S, seed=seed + 1)
    cfg = dict(H0=H, H1=H, S=S, problem=w["problem"], alpha=2,
               lam=(np.zeros(S) if lam is None else lam.astype(np.float64)), gamma=-1.0,
               nu=w["nu"], div_kind=w["div"], lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0,
               train_embedding=True)
    state = None
    th, x0 = theta.astype(np.float64), X0.astype(np.float64)
    t0 = time.perf_counter()
    for t in range(steps):
        out = O.step(g, th, x0, cfg, t=t + 1, adam_state=state)
        th, x0, state = out["theta_next"], out["X0_next"], out["adam_next"]
    return time.perf_counter() - t0, int(rp[-1]), S


def cpu_baseline_child(argv):
    """Child process (single-threaded BLAS): times the oracle on the bounded
    sample for about `budget` seconds and prints one JSON line."""
    wname, budget = argv[0], float(argv[1])
    w = WORKLOADS[wname]
    n = min(CPU_SAMPLE_N, w["N"])
    dt, nnz, S = oracle_steps(w, n, 1)
    steps = max(1, int(budget / max(dt, 1e-3)))
    dt2, nnz, S = oracle_steps(w, n, steps)
    print(json.dumps({"value": nnz * S * steps / dt2, "steps": steps, "seconds": dt2,
                      "nnz": nnz, "N": n}))


def run_cpu_baseline(wname, budget=15.0, threads=1):
    """The oracle on the host cores in a child process whose BLAS uses
    `threads` threads (the oracle's dense products; its sparse scatter-adds
    stay on one thread)."""
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-child", wname,
                        str(budget)], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": METRIC, "cores": threads, "kind": "oracle",
                "sample": "failed: " + r.stderr.strip()[-200:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    w = WORKLOADS[wname]
    how = "single-threaded numpy" if threads == 1 else f"numpy with {threads} BLAS threads"
    return {"value": d["value"], "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": (f"{d['steps']} FP64 oracle step(s) on a {w['graph']} graph N={d['N']} "
                       f"(degree {w['d']}, nnz={d['nnz']}), S={w['S']}, H={w['H']}, same problem; "
                       f"{d['seconds']:.1f} s {how}")}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch

    from paper_2402_02190_gb300 import cpra

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = WORKLOADS[args.workload]
    recompute = w["recompute"] if args.recompute is None else args.recompute
    rp, col = make_graph(w)
    N, nnz, S, H = w["N"], int(rp[-1]), w["S"], w["H"]
    lam = make_lambda(w)
    kw = dict(problem=w["problem"], S=S, H0=H, H1=H, precision=w["precision"], nu=w["nu"],
              diversity_kind=w["div"], gamma0=-2.0, gamma1=0.1,
              schedule_steps=args.warmup + args.steps, seed=1 + rank, recompute=recompute)

    solver = cpra.Solver(rp, col, lam=lam, **kw)
    stream = solver.stream          # the stream every library kernel is launched on
    if args.graph:
        solver.steps(0, args.warmup)   # captures the step graph before timing
    else:
        for t in range(args.warmup):
            solver.step(t)
    torch.cuda.synchronize()
    cpra.cpra_profile_enable(solver.ctx, True)
    cpra.cpra_profile_read(solver.ctx)          # reset counters
    launches0 = solver.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        if args.graph:    # one call: a captured step replayed (cpra_steps)
            solver.steps(args.warmup, args.steps)
        else:
            for t in range(args.warmup, args.warmup + args.steps):
                solver.step(t)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = e0.elapsed_time(e1)
    prof = cpra.cpra_profile_read(solver.ctx)
    launches = solver.launches - launches0
    ms = max_over_ranks(ms, dist)
    graph_ms = None
    if not args.graph:
        # the same steps once more through cpra_steps (one captured step
        # replayed as a CUDA graph), timed the same way, as a second figure
        cpra.cpra_profile_enable(solver.ctx, False)
        t_next = args.warmup + args.steps
        solver.steps(t_next, args.warmup)            # capture + warm replays
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0.record(stream)
        solver.steps(t_next + args.warmup, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        graph_ms = max_over_ranks(e0.elapsed_time(e1), dist)
    solver.close()
    del solver
    torch.cuda.synchronize()

    # end to end through the public API with host buffers: init from the host
    # CSR, every step returns its loss terms to the host, final evaluation
    # copied back.
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s2 = cpra.Solver(rp, col, lam=lam, **kw)
    for t in range(args.steps):
        s2.step(t, want_terms=True)
    rec, ham, _ = s2.round_eval()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    s2.close()
    if dist:
        dist.barrier()
    e2e_s = max_over_ranks(e2e_s, dist)
    h2d = (8 * (N + 1) + 4 * nnz + (4 * S if lam is not None else 0)) / args.steps
    d2h = (3 * S + 1) * 4 + (S * 24 + 8) / args.steps

    # the plain FP32 form (every dense layer in FP32) on the same graph and
    # shots, timed the same way: the comparator of the BF16 form, with each
    # of its two engines
    def time_fp32(engine):
        s3 = cpra.Solver(rp, col, lam=lam, **dict(kw, precision=0, fp32_engine=engine))
        for t in range(args.warmup):
            s3.step(t)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0.record(s3.stream)
        for t in range(args.warmup, args.warmup + args.steps):
            s3.step(t)
        e1.record(s3.stream)
        torch.cuda.synchronize()
        ms32 = max_over_ranks(e0.elapsed_time(e1), dist)
        s3.close()
        return {"ms_per_step": ms32 / args.steps,
                "value": replica_throughput(world, nnz * S * args.steps, ms32 / 1e3),
                "unit": METRIC, "steps": args.steps, "warmup": args.warmup}

    fp32_form = None
    if w["precision"] == 1 and not args.no_fp32_form:
        fp32_form = time_fp32(cpra.FP32_TENSOR)
        fp32_form["how"] = ("the same workload with precision fp32: dense layers and input "
                            "gradients as split-TF32 tensor-core GEMMs (FP32-accurate), weight "
                            "gradients on CUDA cores; per-step launches, CUDA events on the "
                            "library stream")
        fp32_form["cuda_cores"] = time_fp32(cpra.FP32_CUDA_CORES)
        fp32_form["cuda_cores"]["how"] = "the same with every dense product on CUDA cores"

    value = replica_throughput(world, nnz * S * args.steps, ms / 1e3)
    peak, peak_src = read_peaks()
    loss_ms, loss_n = prof.get("loss_fused", (0.0, 0))
    g_bytes = 2 if w["precision"] == 1 else 4
    alg = loss_kernel_bytes(N, nnz, S, g_bytes)
    comp = loss_compulsory_bytes(N, nnz, S, g_bytes)
    achieved = alg / (loss_ms / loss_n / 1e3) / 1e9 if loss_n else None
    traffic, traffic_basis = ncu_traffic("loss_fused", args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if w["precision"] == 1 else "f32",
        "dtype_detail": ("dense layers bf16 operands / fp32 accumulation; loss, Adam, rounding fp32; "
                         "objective reduction int64/fp64") if w["precision"] == 1 else "all fp32",
        "data": "synthetic (seeded random graph, random-init GCN)",
        "config": {"workload": args.workload, "graph": f"{w['graph']} degree {w['d']}", "N": N,
                   "nnz": nnz, "S": S, "H0": H, "H1": H,
                   "problem": ["MIS", "MaxCut"][w["problem"]], "nu": w["nu"],
                   "precision": ["fp32", "bf16"][w["precision"]], "parallelism": f"replicas{world}",
                   "recompute": recompute,
                   "launch": "one captured step replayed (CUDA graph)" if args.graph else "per-step launches",
                   "l2": f"inputs larger than L2 (P = {N * S * 4 / 1e9:.2f} GB), no flush"},
        "roofline": {"kernel": "loss_fused", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_basis": traffic_basis,
                     "alg_bytes_per_launch": alg, "avg_ms": loss_ms / loss_n if loss_n else None,
                     # a second line: the bound if no neighbour row were re-read
                     # (the gathers' amplification over it is alg / compulsory)
                     "compulsory": {"bytes_per_launch": comp,
                                    "achieved": comp / (loss_ms / loss_n / 1e3) / 1e9 if loss_n else None,
                                    "frac": (comp / (loss_ms / loss_n / 1e3) / 1e9 / peak) if loss_n else None,
                                    "gather_amplification": alg / comp},
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"},
        "e2e": {"value": replica_throughput(world, nnz * S * args.steps, e2e_s), "unit": METRIC,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "seconds": e2e_s},
        "gpu_launches": launches,
        "fp32_form": fp32_form,
        "graph": None if graph_ms is None else {
            "ms_per_step": graph_ms / args.steps,
            "value": replica_throughput(world, nnz * S * args.steps, graph_ms / 1e3),
            "how": "the same steps through cpra_steps: one captured step replayed as a CUDA graph"},
        "clocks": clk.summary(),
        "kernels_ms_per_step": {k: v[0] / max(v[1], 1) * (v[1] / args.steps)
                                for k, v in prof.items() if v[1]},
        "best_eval": {"max_objective_feasible": int(max(
            [r["objective"] for r in rec if r["violations"] == 0] or [-1]))},
    }
    if world == 1 and w["precision"] == 1 and not args.no_quality:
        # the time-to-quality half of the metric, in compact form
        line["quality_compact"] = run_quality_compact(args)
    if rank == 0:
        line["cpu_baseline"] = run_cpu_baseline(args.workload) if not args.no_cpu else None
        if not args.no_cpu and world == 1:
            # the same oracle with every host core behind its dense products
            cores = len(os.sched_getaffinity(0))
            line["cpu_baseline_all_cores"] = run_cpu_baseline(args.workload, 10.0, cores)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------ reference arm
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    n = min(CPU_SAMPLE_N, w["N"])
    for _ in range(args.warmup):
        oracle_steps(w, n, 1)
    dt, nnz, S = oracle_steps(w, n, args.steps)
    value = nnz * S * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", "0")) or len(os.sched_getaffinity(0))
    sample = (f"{args.steps} FP64 oracle steps on a {w['graph']} graph N={n} (degree {w['d']}, "
              f"nnz={nnz}), S={S}, H={w['H']}: the workload's degree, shots and width on {n} nodes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "sample_N": n},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------ quality mode
def _reach(trace, target):
    from paper_2402_02190_gb300 import warm as WM
    r = WM.time_to_reach(trace, target)
    return {"seconds_to_99pct": r[0] if r else None, "steps_to_99pct": r[1] if r else None,
            "best": trace[-1][2], "total_seconds": trace[-1][0]}


def run_quality(args):
    """The metric's second half: wall time for the BF16 + warm-start form to
    come within 1% of the best MIS the plain FP32 form finds on the same graph
    (the workload's graph, shots and widths).

    Arms on that graph, all from the same seeds: plain FP32 and plain BF16
    with the full schedule (gamma -2 -> 0.1), plain BF16 and BF16 + warm start
    with the warm arm's shorter convex phase (gamma from q_warm_gamma0), and
    BF16 + warm start with the full schedule.  The warm start's own effect is
    the warm arm against the plain arm with the same schedule.  Also: the
    warm-start network's training cost (target solves + fit) and how many
    solves it takes to pay for it, and a held-out check where every graph's
    warm and schedule-matched plain runs are measured against a longer plain
    run (q_ref_steps, full schedule) whose final binarisation is reported."""
    import torch
    from paper_2402_02190_gb300 import cpra
    from paper_2402_02190_gb300 import warm as WM
    w = WORKLOADS[args.workload]
    S, H = w["S"], w["H"]
    lam = make_lambda(w)
    q = args.q_steps
    g0 = args.q_warm_gamma0
    out = {"metric": "wall time to within 1% of the FP32 form's best MIS (BF16 + warm start)",
           "unit": "s", "higher_is_better": False, "mode": "quality",
           "data": "synthetic (seeded random regular graphs)",
           "config": {"workload": args.workload, "steps": q, "eval_every": args.q_eval,
                      "warm_gamma0": g0, "warm_graphs": args.q_train,
                      "warm_heldout": args.q_heldout, "graph_nodes": [args.q_nmin, args.q_nmax],
                      "target_steps": args.q_target_steps, "heldout_ref_steps": args.q_ref_steps,
                      "target_union_nodes": args.q_union_nodes}}
    # 1. targets from plain CPRA (BF16, full schedule) on seeded training graphs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    graphs = WM.training_graphs(args.q_train + args.q_heldout, seed=77, n_min=args.q_nmin,
                                n_max=args.q_nmax)
    t_gen = time.perf_counter() - t0
    train, held = graphs[:args.q_train], graphs[args.q_train:]
    t0 = time.perf_counter()
    dataset = []
    if args.q_union_nodes > 0:  # multi-instance solves of disjoint unions
        tbits = WM.cpra_targets_union([(g[0], g[1]) for g in train], S, lam, args.q_target_steps,
                                      cpra.BF16, H=64, seed=1, max_nodes=args.q_union_nodes)
        dataset = [(g[0], g[1], b, 1000 + k) for k, (g, b) in enumerate(zip(train, tbits))]
    else:
        for k, (rp, col, d) in enumerate(train):
            bits, _ = WM.cpra_targets(rp, col, S, lam, args.q_target_steps, cpra.BF16, H=64,
                                      seed=k + 1)
            dataset.append((rp, col, bits, 1000 + k))
    torch.cuda.synchronize()
    t_targets = time.perf_counter() - t0
    # 2. fit the warm-start network
    max_n = max(len(g[0]) - 1 for g in train) * args.q_batch
    max_e = max(int(g[0][-1]) for g in train) * args.q_batch
    net = cpra.WarmStartNet(max_n, max_e, F=16, H=64, S=S, precision=cpra.BF16, lr=3e-3)
    t0 = time.perf_counter()
    losses = WM.train_network(net, dataset, args.q_epochs, args.q_batch)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    theta = net.params(0)
    net.close()
    out["warm_training"] = {"graphs": len(dataset), "target_steps": args.q_target_steps,
                            "graph_generation_seconds": t_gen,
                            "target_seconds": t_targets, "fit_seconds": t_fit,
                            "cost_seconds": t_targets + t_fit,
                            "epochs": args.q_epochs, "loss_first": losses[0], "loss_last": losses[-1]}
    # 3. held-out graphs: warm and schedule-matched plain runs against a long
    #    plain run of the full schedule
    per_graph = []
    for k, (rp, col, d) in enumerate(held):
        N = len(rp) - 1
        big = cpra.WarmStartNet(N, int(rp[-1]), F=16, H=64, S=S, precision=cpra.BF16)
        big.set_params(theta)
        L0 = WM.predict_logits(big, rp, col, 5000 + k)
        big.close()
        fin = []
        ref = WM.run_trace(rp, col, S, lam, args.q_ref_steps, args.q_eval, cpra.BF16, H=64, seed=7,
                           final_terms=fin)
        best = ref[-1][2]
        arms = {
            "plain_full": WM.run_trace(rp, col, S, lam, args.q_target_steps, args.q_eval,
                                       cpra.BF16, H=64, seed=7),
            "plain_matched": WM.run_trace(rp, col, S, lam, args.q_target_steps, args.q_eval,
                                          cpra.BF16, H=64, seed=7, gamma0=g0),
            "warm": WM.run_trace(rp, col, S, lam, args.q_target_steps, args.q_eval, cpra.BF16,
                                 H=64, seed=7, init_logits=L0, gamma0=g0),
        }
        row = {"N": N, "d": d, "ref_best": best,
               "ref_binarised": WM.binarised_fraction(fin[0], N, S),
               "ref_steps_to_99pct": (WM.time_to_reach(ref, 0.99 * best) or (None, None))[1]}
        for name, tr in arms.items():
            r = WM.time_to_reach(tr, 0.99 * best)
            row[name] = {"best": tr[-1][2], "gap": (best - tr[-1][2]) / max(best, 1),
                         "steps_to_99pct": r[1] if r else None}
        per_graph.append(row)
    def _mean(xs):
        xs = [x for x in xs if x is not None]
        return float(np.mean(xs)) if xs else None
    out["heldout"] = {
        "graphs": len(per_graph),
        "ref_binarised_min": min(r["ref_binarised"] for r in per_graph),
        "ref_binarised_mean": _mean([r["ref_binarised"] for r in per_graph]),
        "warm_gap_mean": _mean([r["warm"]["gap"] for r in per_graph]),
        "plain_matched_gap_mean": _mean([r["plain_matched"]["gap"] for r in per_graph]),
        "plain_full_gap_mean": _mean([r["plain_full"]["gap"] for r in per_graph]),
        "warm_better_than_plain_full": sum(r["warm"]["best"] > r["plain_full"]["best"]
                                           for r in per_graph),
        "warm_worse_than_plain_full": sum(r["warm"]["best"] < r["plain_full"]["best"]
                                          for r in per_graph),
        "plain_full_reached_99pct": sum(r["plain_full"]["steps_to_99pct"] is not None
                                        for r in per_graph),
        "warm_better_than_plain_matched": sum(r["warm"]["best"] > r["plain_matched"]["best"]
                                              for r in per_graph),
        "warm_worse_than_plain_matched": sum(r["warm"]["best"] < r["plain_matched"]["best"]
                                             for r in per_graph),
        "warm_reached_99pct": sum(r["warm"]["steps_to_99pct"] is not None for r in per_graph),
        "plain_matched_reached_99pct": sum(r["plain_matched"]["steps_to_99pct"] is not None
                                           for r in per_graph),
        "warm_steps_to_99pct_mean": _mean([r["warm"]["steps_to_99pct"] for r in per_graph]),
        "plain_matched_steps_to_99pct_mean": _mean([r["plain_matched"]["steps_to_99pct"]
                                                    for r in per_graph]),
        "per_graph": per_graph,
    }
    # 4. the workload graph: every arm, wall clock from context creation
    rp, col = make_graph(w)
    fp32 = WM.run_trace(rp, col, S, lam, q, args.q_eval, cpra.FP32, H=H, seed=1)
    best = fp32[-1][2]
    target = 0.99 * best
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    big = cpra.WarmStartNet(len(rp) - 1, int(rp[-1]), F=16, H=64, S=S, precision=cpra.BF16)
    big.set_params(theta)
    L0 = WM.predict_logits(big, rp, col, 99)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    warm = WM.run_trace(rp, col, S, lam, q, args.q_eval, cpra.BF16, H=H, seed=1, init_logits=L0,
                        gamma0=g0, t0=t0)
    big.close()
    plain16 = WM.run_trace(rp, col, S, lam, q, args.q_eval, cpra.BF16, H=H, seed=1)
    plain16_m = WM.run_trace(rp, col, S, lam, q, args.q_eval, cpra.BF16, H=H, seed=1, gamma0=g0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    big = cpra.WarmStartNet(len(rp) - 1, int(rp[-1]), F=16, H=64, S=S, precision=cpra.BF16)
    big.set_params(theta)
    L0 = WM.predict_logits(big, rp, col, 99)
    warm_full = WM.run_trace(rp, col, S, lam, q, args.q_eval, cpra.BF16, H=H, seed=1,
                             init_logits=L0, gamma0=-2.0, t0=t0)
    big.close()
    arms = {"fp32": fp32, "bf16_plain": plain16, "bf16_plain_matched_schedule": plain16_m,
            "bf16_warm": warm, "bf16_warm_full_schedule": warm_full}
    out["race"] = {"target": target, "fp32_best": best,
                   "warm_inference_seconds": t_inf,
                   "arms": {k: _reach(x, target) for k, x in arms.items()},
                   "traces": {k: [(round(a, 4), b, c) for a, b, c in x[::max(1, len(x) // 10)]]
                              for k, x in arms.items()}}
    a = out["race"]["arms"]
    rw, rm = a["bf16_warm"]["seconds_to_99pct"], a["bf16_plain_matched_schedule"]["seconds_to_99pct"]
    saved = (rm - rw) if (rw is not None and rm is not None) else None
    rf = a["bf16_plain"]["seconds_to_99pct"]
    saved_f = (rf - rw) if (rw is not None and rf is not None) else None
    out["warm_effect"] = {
        "vs": "bf16_plain_matched_schedule (same precision, same gamma schedule, same seed)",
        "seconds_saved_per_solve": saved,
        "matched_reached_target": rm is not None,
        "vs_fastest_plain": "bf16_plain (full schedule, the fastest plain BF16 arm)",
        "seconds_saved_per_solve_vs_fastest_plain": saved_f,
        "training_cost_seconds": t_targets + t_fit,
        "solves_to_amortise": ((t_targets + t_fit) / saved) if saved and saved > 0 else None,
        "solves_to_amortise_vs_fastest_plain": ((t_targets + t_fit) / saved_f)
        if saved_f and saved_f > 0 else None}
    out["value"] = rw
    out["vs_fp32_seconds"] = a["fp32"]["seconds_to_99pct"]
    print(json.dumps(out))


def run_quality_compact(args):
    """A compact form of the time-to-quality race for the default line: MIS on
    a seeded 5-regular graph of 2*10^5 nodes (S = 256, H = 128, the default
    workload's shots and widths), 2000-step schedules, evaluation every 50
    steps; the warm-start network trained on 512 small graphs (N 1,000-5,000,
    1000-step targets) whose targets come from multi-instance solves: the
    graphs are packed into disjoint unions of up to 2*10^5 nodes and each
    union is solved by one CPRA run.  Arms as in --quality: FP32 (split-TF32
    engine), BF16 plain, BF16 plain with the warm arm's schedule, BF16 + warm
    start.  The first 8 training graphs are also solved one by one, to report
    how the union-solved targets compare."""
    import torch
    from paper_2402_02190_gb300 import cpra
    from paper_2402_02190_gb300 import warm as WM
    S, H, steps, ev = 256, 128, 2000, 50
    n_train, target_steps, union_nodes, n_check = 512, 1000, 200_000, 8
    lam = I.lambda_geomspace(0.5, 10.0, S)
    g0 = args.q_warm_gamma0
    graphs = WM.training_graphs(n_train, seed=78, n_min=1000, n_max=5000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tbits = WM.cpra_targets_union([(g[0], g[1]) for g in graphs], S, lam, target_steps,
                                  cpra.BF16, H=64, seed=1, max_nodes=union_nodes)
    torch.cuda.synchronize()
    t_targets = time.perf_counter() - t0
    dataset = [(g[0], g[1], b, 2000 + k) for k, (g, b) in enumerate(zip(graphs, tbits))]
    net = cpra.WarmStartNet(max(len(g[0]) - 1 for g in graphs) * 8,
                            max(int(g[0][-1]) for g in graphs) * 8, F=16, H=64, S=S,
                            precision=cpra.BF16, lr=3e-3)
    t0 = time.perf_counter()
    WM.train_network(net, dataset, 40, 8)
    theta = net.params(0)
    net.close()
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    # union-solved targets against separate solves of the same graphs
    check = []
    for k in range(n_check):
        rp_k, col_k, _ = graphs[k]
        sep, _ = WM.cpra_targets(rp_k, col_k, S, lam, target_steps, cpra.BF16, H=64, seed=1)
        check.append((WM.mis_best_from_bits(rp_k, col_k, tbits[k], S),
                      WM.mis_best_from_bits(rp_k, col_k, sep, S)))
    rp, col = I.random_regular_graph(2 * 10**5, 5, seed=55)
    fp32 = WM.run_trace(rp, col, S, lam, steps, ev, cpra.FP32, H=H, seed=1)
    target = 0.99 * fp32[-1][2]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    big = cpra.WarmStartNet(len(rp) - 1, int(rp[-1]), F=16, H=64, S=S, precision=cpra.BF16)
    big.set_params(theta)
    L0 = WM.predict_logits(big, rp, col, 99)
    warm = WM.run_trace(rp, col, S, lam, steps, ev, cpra.BF16, H=H, seed=1, init_logits=L0,
                        gamma0=g0, t0=t0)
    big.close()
    plain = WM.run_trace(rp, col, S, lam, steps, ev, cpra.BF16, H=H, seed=1)
    matched = WM.run_trace(rp, col, S, lam, steps, ev, cpra.BF16, H=H, seed=1, gamma0=g0)

    def arm(tr):
        r = WM.time_to_reach(tr, target)
        return {"seconds_to_99pct": r[0] if r else None, "steps_to_99pct": r[1] if r else None,
                "best": tr[-1][2]}
    return {"metric": "wall seconds to within 1% of the FP32 form's best MIS", "unit": "s",
            "graph": "rrg degree 5, N=200000, seed 55", "S": S, "H": H, "steps": steps,
            "eval_every": ev, "warm_gamma0": g0,
            "warm_training": {"graphs": n_train, "target_steps": target_steps,
                              "targets": "multi-instance: disjoint unions of up to %d nodes, "
                                         "one CPRA run each" % union_nodes,
                              "target_seconds": t_targets, "fit_seconds": t_fit,
                              "seconds": t_targets + t_fit,
                              "union_vs_separate_best_mis": [list(c) for c in check]},
            "fp32": arm(fp32), "bf16_plain": arm(plain), "bf16_plain_matched_schedule": arm(matched),
            "bf16_warm": arm(warm),
            "how": "compact form of bench.py --quality; wall clock from context creation "
                   "(the warm arm includes its network inference)"}


# ------------------------------------------------------------ two-stage mode
def run_two_stage_bench(args):
    """The two-stage experiment's shape (App. two-stage): weighted-MIS tasks on
    one seeded 1000-node 5-regular graph, S' warm-up heads then a fresh S-way
    head on the frozen encoder, against one S-head network from scratch."""
    from paper_2402_02190_gb300 import cpra
    from paper_2402_02190_gb300 import two_stage as TS
    rp, col = I.random_regular_graph(1000, 5, seed=2024)
    S, Sp = args.ts_tasks, args.ts_warm
    W = np.random.default_rng(7).uniform(0.0, 1.0, size=(1000, S)).astype(np.float32)
    lam = np.full(S, 2.0, np.float32)
    ts = TS.run_two_stage(rp, col, W, lam, Sp, args.ts_pre_steps, args.ts_ft_steps, H=64,
                          precision=cpra.BF16, eval_every=100)
    sc = TS.run_scratch(rp, col, W, lam, args.ts_pre_steps + args.ts_ft_steps, H=64,
                        precision=cpra.BF16, eval_every=100)
    out = {"metric": "weighted-MIS average best weight and wall time, two-stage vs scratch",
           "mode": "two-stage", "data": "synthetic (seeded 5-regular graph, U(0,1) weights)",
           "config": {"N": 1000, "d": 5, "tasks": S, "warm_tasks": Sp, "H": 64, "precision": "bf16",
                      "pre_steps": args.ts_pre_steps, "ft_steps": args.ts_ft_steps,
                      "lambda": 2.0, "stop": "annealing term < 1e-4"},
           "two_stage": {k: ts[k] for k in ("pre_seconds", "ft_seconds", "total_seconds", "pre_stop",
                                             "ft_stop", "avg_weight", "feasible_tasks",
                                             "encoder_unchanged")},
           "scratch": {k: sc[k] for k in ("total_seconds", "stop", "avg_weight", "feasible_tasks")}}
    print(json.dumps(out))


# ------------------------------------------------------------ DBM mode
def run_dbm_bench(args):
    """Diverse bipartite matching at the paper's sizes (App. problem
    specification: 50 + 50 nodes, 2500 pair variables; network width 2500,
    here 2512): the 11 x 11 penalty grid on one instance and multi-instance
    CPRA over 27 instances, with the paper's optimiser, schedule and early
    stopping.  Seeded synthetic instances stand in for the CORA-derived ones;
    ApR is measured against scipy's exact MILP optimum."""
    import torch
    from paper_2402_02190_gb300 import cpra
    from paper_2402_02190_gb300 import dbm
    N1 = N2 = 50
    rp, col = I.dbm_graph(N1, N2)
    pq = args.dbm_pq
    H = args.dbm_h
    modes = ("grid", "multi") if args.dbm_mode == "both" else (args.dbm_mode,)
    for mode in modes:
        if mode == "grid":
            C, M, p, q = I.dbm_instance(N1, N2, seed=11, p=pq, q=pq)
            shots = dbm.penalty_grid_shots(N1, N2, C, M, p, q)
            opt = np.full(shots[2].shape[0], dbm.best_diverse_matching(C, M, N1, N2, p, q)[0])
            paper = {"0.25": 1961, "0.05": 2154}.get(str(pq))
        else:
            insts = [I.dbm_instance(N1, N2, seed=1000 + k, p=pq, q=pq) for k in range(27)]
            shots = dbm.multi_instance_shots(N1, N2, [(c, m) for c, m, _, _ in insts], pq=(pq, pq))
            opt = np.array([dbm.best_diverse_matching(c, m, N1, N2, pq, pq)[0] for c, m, _, _ in insts])
            paper = {"0.25": 5617, "0.05": 2907}.get(str(pq))
        S = shots[2].shape[0]
        # step time: graph-replayed steps of a separate context, CUDA events on its stream
        t = cpra.Solver(rp, col, problem=cpra.DBM, S=S, H0=H, H1=H, precision=cpra.BF16, seed=2,
                        **cpra.paper_preset(cpra.DBM, args.dbm_steps))
        t.set_dbm(N1, *shots)
        t.steps(0, args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(t.stream)
        t.steps(args.warmup, args.steps)
        e1.record(t.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        t.close()
        r = dbm.run(rp, col, N1, N2, shots, H, args.dbm_steps, args.dbm_eval)
        a = dbm.apr(r["best"], opt)
        ok = np.isfinite(a)
        print(json.dumps({
            "metric": "DBM: wall seconds of a full CPRA run and ApR of its best feasible matchings",
            "mode": f"dbm-{mode}", "data": "synthetic (seeded 50 x 50 instances, U^3 rewards, 7 fields)",
            "config": {"N1": N1, "N2": N2, "S": S, "H0": H, "H1": H, "precision": "bf16",
                       "p": pq, "q": pq, "max_steps": args.dbm_steps, "eval_every": args.dbm_eval,
                       "optimiser": "AdamW lr 1e-4 wd 1e-2", "gamma": "-20 + 1e-3 t",
                       "early_stopping": "tol 1e-5, patience 1000",
                       "lambda": "(a, a, b, b), a, b in 2^0..2^10" if mode == "grid" else "(2, 2, 12, 12)"},
            "ms_per_step": ms, "step_timing": f"{args.steps} graph-replayed steps after {args.warmup}",
            "seconds": r["seconds"], "steps_applied": r["steps_applied"], "stop_step": r["stop"],
            "apr": {"max": float(np.nanmax(a)) if ok.any() else None,
                    "mean_feasible": float(np.nanmean(a)) if ok.any() else None,
                    "min_feasible": float(np.nanmin(a)) if ok.any() else None,
                    "feasible_shots": int(ok.sum()), "shots": int(S),
                    "shots_at_optimum": int((a[ok] >= 1 - 1e-6).sum())},
            "optimum": float(opt[0]) if mode == "grid" else [float(v) for v in opt],
            "paper_seconds_v100": paper}))


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--cpu-baseline-child":
        cpu_baseline_child(sys.argv[2:])
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp32-form", action="store_true",
                    help="skip timing the FP32 form of a BF16 workload")
    ap.add_argument("--no-quality", action="store_true",
                    help="skip the compact time-to-quality race of the default line")
    ap.add_argument("--recompute", type=int, choices=[0, 1], default=None,
                    help="override the workload's activation-recompute setting")
    ap.add_argument("--graph", action="store_true",
                    help="time the steps through cpra_steps (one captured step replayed as a CUDA "
                         "graph); per-kernel times are then not available")
    ap.add_argument("--quality", action="store_true",
                    help="time-to-quality run: FP32 plain vs BF16 + warm start on the workload graph")
    ap.add_argument("--q-steps", type=int, default=2000)
    ap.add_argument("--q-eval", type=int, default=50)
    ap.add_argument("--q-train", type=int, default=4096)
    ap.add_argument("--q-heldout", type=int, default=256)
    ap.add_argument("--q-nmin", type=int, default=1000)
    ap.add_argument("--q-nmax", type=int, default=10000)
    ap.add_argument("--q-ref-steps", type=int, default=3000)
    ap.add_argument("--q-target-steps", type=int, default=1000)
    ap.add_argument("--q-union-nodes", type=int, default=0,
                    help="solve the training targets as disjoint unions of up to this many "
                         "nodes (multi-instance CPRA); 0: one solve per graph")
    ap.add_argument("--q-epochs", type=int, default=40)
    ap.add_argument("--q-batch", type=int, default=8)
    ap.add_argument("--q-warm-gamma0", type=float, default=-0.5)
    ap.add_argument("--two-stage", action="store_true",
                    help="two-stage (S' -> S) weighted-MIS run against training all heads from scratch")
    ap.add_argument("--ts-tasks", type=int, default=500)
    ap.add_argument("--ts-warm", type=int, default=200)
    ap.add_argument("--ts-pre-steps", type=int, default=8000)
    ap.add_argument("--ts-ft-steps", type=int, default=2000)
    ap.add_argument("--dbm", action="store_true",
                    help="diverse bipartite matching runs (penalty grid, multi-instance) with ApR")
    ap.add_argument("--dbm-mode", default="both", choices=["both", "grid", "multi"])
    ap.add_argument("--dbm-pq", type=float, default=0.25, help="p = q (Matching-1 0.25, -2 0.05)")
    ap.add_argument("--dbm-h", type=int, default=2512)
    ap.add_argument("--dbm-steps", type=int, default=50_000)
    ap.add_argument("--dbm-eval", type=int, default=500)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)   # at least three untimed warm-up steps
    if args.dbm:
        run_dbm_bench(args)
        return
    if args.two_stage:
        run_two_stage_bench(args)
        return
    if args.quality:
        run_quality(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
