"""Benchmark of the LEM hot path on GB300: 2D periodic advection-diffusion, 2048^2 nodes,
32^2 owner tiles + 8-node buffers (48^2 = 2304-node windows), one shared 1024 x 2304 phi_1
propagator applied to all 4096 tiles every step (Sec. 3, Eq. lem).

One bench step = one lem_step call advancing the state by --inner LEM time steps (the
residual, the halo gather inside TMA, the propagator apply and the owner scatter for all
4096 tiles, every LEM step). Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split|split_fast|fp64]
                  [--impl reference] [--workload advdiff2d|batch512|serve|heat1d|vardiff2d|
                  vardiff1d|schrodinger1d] [--trunc TOL]

--workload picks another configuration: batch512 (512 uneven problems under one CUDA graph),
serve (a Poisson stream of requests through the server), heat1d (1D heat, persistent GEMV),
vardiff2d (per-tile propagators with the u - u^3 reaction, batched GEMV; --scheme rb3 for the
third-order scheme), vardiff1d (2^20-node 1D variable-coefficient diffusion, a propagator per
tile; --trunc TOL applies truncated propagators) and schrodinger1d (the complex Schroedinger
test; --sn sets the mesh).

Metric: LEM dof-steps/s = owner nodes x LEM steps / device time. L2 is flushed (256 MiB
write) between timed calls; each call is bracketed by CUDA events on the context stream.
Multi-GPU (torchrun): every rank advances its own independent problem (weak scaling, no
collective on the data path); rank 0 reports the aggregate over ranks with the max time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LEM dof-steps/s"
WORKLOAD = "advdiff2d_2048x2048_periodic_tile32_H8_phi"
BATCH_WORKLOAD = "batch512_uneven_advdiff2d_periodic_side64-512_tile8-32_H4-8"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--inner", type=int, default=10, help="LEM time steps per bench step")
    ap.add_argument("--prec", default="split", choices=["split", "split_fast", "fp64"],
                    help="split: three FP16 pieces per operand (six tensor-core products); split_fast: two "
                         "pieces (four products); fp64: the plain FP64 GPU path")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=2048)
    ap.add_argument("--workload", default="advdiff2d",
                    choices=["advdiff2d", "batch512", "serve", "heat1d", "vardiff2d", "vardiff1d", "schrodinger1d"],
                    help="advdiff2d: one 2048^2 problem (default); batch512: 512 uneven problems under one "
                         "CUDA graph; serve: a Poisson stream of advance requests through the server")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: mean arrivals per second")
    ap.add_argument("--duration", type=float, default=1.0, help="serve: seconds of arrivals")
    ap.add_argument("--drain", type=float, default=120.0, help="serve: seconds to wait for completions")
    ap.add_argument("--nprob", type=int, default=512, help="batch512: number of problems")
    ap.add_argument("--vside", type=int, default=1024, help="vardiff2d: mesh side")
    ap.add_argument("--vn", type=int, default=1 << 20, help="vardiff1d: mesh nodes")
    ap.add_argument("--trunc", type=float, default=None,
                    help="heat1d / vardiff1d / vardiff2d: truncated propagators with this tolerance")
    ap.add_argument("--sn", type=int, default=400, help="schrodinger1d: mesh points (the paper's test: 400)")
    ap.add_argument("--scheme", default="euler", choices=["euler", "rb3"],
                    help="vardiff2d: exponential Euler-Rosenbrock (phi_1) or the third-order exprb32 (phi_1 + phi_3)")
    ap.add_argument("--lanes", type=int, default=16, help="batch512: concurrent lanes in the graph")
    ap.add_argument("--tile", type=int, nargs=2, default=[32, 32], metavar=("TY", "TX"),
                    help="advdiff2d: tile shape (rows, columns)")
    ap.add_argument("--overlap", type=int, nargs=2, default=[8, 8], metavar=("HY", "HX"),
                    help="advdiff2d: overlap per side (rows, columns)")
    ap.add_argument("--vel", type=float, nargs=2, default=[1.0, 0.5], metavar=("AX", "AY"),
                    help="advdiff2d: velocity (h = 1, dt = 4: Courant numbers 4 a)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    return ap.parse_args()


def max_over_ranks(local_ms: float) -> float:
    """The slowest rank's time (every rank gets it): an all-reduce MAX when a process group
    is up (a CUDA tensor for NCCL, a CPU tensor for gloo), else the local time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(local_ms)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("bf16_tflops", 1900.0), d.get("hbm_gbs", 6800.0), "measured"
    return 1900.0, 6800.0, "fallback"


def fp64_dgemm_tflops(dev, n=8192, reps=5):
    """The FP64 roofline denominator: cuBLAS DGEMM (torch.matmul on float64, n^3) on this GPU,
    best of `reps` after one warm-up, timed with CUDA events (2 n^3 flop each)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None or ms < best else best
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("step_split.cu", "tc_ptx.cuh", "ff_convert.h"):
        with open(os.path.join(ROOT, "paper_1505_02248_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_hash):
    """DRAM bytes per launch of the split GEMM from the committed ncu summary, if it was
    captured from the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "split_gemm_advdiff2d_2048.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_hash") != kernel_hash:
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def advdiff_workload(a, seed=1):
    """The advdiff2d workload of the command line, and its name for the JSON line."""
    from paper_1505_02248_gb300 import workloads as W
    wl = W.advdiff2d(side=a.side, tile=tuple(a.tile), overlap=tuple(a.overlap), a=tuple(a.vel), seed=seed)
    if tuple(a.tile) == (32, 32) and tuple(a.overlap) == (8, 8) and tuple(a.vel) == (1.0, 0.5) and a.side == 2048:
        return wl, WORKLOAD
    return wl, (f"advdiff2d_{a.side}x{a.side}_periodic_tile{a.tile[0]}x{a.tile[1]}_H{a.overlap[0]}x{a.overlap[1]}"
                f"_C{4 * a.vel[0]:g}x{4 * a.vel[1]:g}_phi")


def oracle_sample(a, max_seconds=20.0):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload: the shared
    propagator build once, then LEM steps restricted to a subset of tiles."""
    import oracle as O
    wl, _ = advdiff_workload(a)
    X = O.assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = O.decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    t0 = time.perf_counter()
    P = O.local_propagators(X, wins, "phi", tiles=[0])[0]
    t_build = time.perf_counter() - t0
    ntile = 64
    sample = list(range(0, len(wins), max(1, len(wins) // ntile)))[:ntile]
    props = [P if i in set(sample) else None for i in range(len(wins))]
    u = wl["u0"].copy()
    steps, t_step = 0, 0.0
    while t_step < max_seconds / 2 and steps < 50:
        t0 = time.perf_counter()
        u = O.lem_step(X, u, wins, props, "phi", tiles=sample)
        t_step += time.perf_counter() - t0
        steps += 1
    dofs = sum(len(wins[i].D) for i in sample) * steps
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {"value": dofs / t_step, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{len(sample)} of {len(wins)} tiles x {steps} LEM steps (numpy FP64 oracle); "
                      f"the one-time propagator build took {t_build:.1f} s and is excluded"}


def oracle_batch_sample(nprob, inner, max_seconds=20.0):
    """The FP64 oracle on a bounded sample of the uneven batch: whole problems (the smallest
    first, so that several fit), their propagators built once, then LEM steps."""
    import oracle as O
    from paper_1505_02248_gb300 import workloads as W
    probs = sorted(W.batch_problems(n=nprob, seed=3), key=lambda p: p["shape"][0])[:4]
    t_build = 0.0
    prepared = []
    for p in probs:
        X = O.assemble_operator(p["shape"], p["bc"], p["coef"], p["dt"])
        wins = O.decompose(p["shape"], p["bc"], p["tile"], p["overlap"])
        t0 = time.perf_counter()
        P = O.local_propagators(X, wins, "phi", tiles=[0])[0]
        t_build += time.perf_counter() - t0
        prepared.append((X, wins, [P] * len(wins), p["u0"].copy()))
    dofs, t_step, steps = 0, 0.0, 0
    while t_step < max_seconds / 2 and steps < inner:
        for k, (X, wins, props, u) in enumerate(prepared):
            t0 = time.perf_counter()
            u = O.lem_step(X, u, wins, props, "phi")
            t_step += time.perf_counter() - t0
            prepared[k] = (X, wins, props, u)
            dofs += u.size
        steps += 1
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {"value": dofs / t_step, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{len(prepared)} smallest of {nprob} problems x {steps} LEM steps (numpy FP64 oracle); "
                      f"their propagator builds took {t_build:.1f} s and are excluded"}


def oracle_serve_sample(rate, duration, max_seconds=20.0):
    """The FP64 oracle on a bounded sample of the request stream: the smallest requests (their
    propagators built once per operator and excluded), each for its own number of steps."""
    import oracle as O
    from paper_1505_02248_gb300 import workloads as W
    reqs = sorted(serve_requests(rate, duration), key=lambda r: int(np.prod(r["shape"])))
    props, dofs, t_run, done = {}, 0, 0.0, 0
    for r in reqs:
        if t_run > max_seconds / 2 or done >= 32:
            break
        X = O.assemble_operator(r["shape"], r["bc"], r["coef"], r["dt"])
        wins = O.decompose(r["shape"], r["bc"], r["tile"], r["overlap"])
        key = (len(r["shape"]), tuple(sorted(r["coef"].items())))
        if key not in props:
            props[key] = O.local_propagators(X, wins, "phi", tiles=[0])[0]
        u = (W.grf_1d(r["shape"][0], 8.0, 1) if len(r["shape"]) == 1 else W.grf_2d(r["shape"], 16.0, 1).ravel())
        t0 = time.perf_counter()
        for _ in range(r["steps"]):
            u = O.lem_step(X, u, wins, [props[key]] * len(wins), "phi")
        t_run += time.perf_counter() - t0
        dofs += u.size * r["steps"]
        done += 1
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {"value": dofs / t_run, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"the {done} smallest of {len(reqs)} requests, each for its own steps (numpy FP64 oracle); "
                      f"propagator builds excluded"}


def small_workload(a):
    """The single-problem workloads of run_small: (workload dict, precision, name)."""
    from paper_1505_02248_gb300 import workloads as W
    if a.workload == "heat1d":
        return W.heat1d(), "fp64", "heat1d_N1024_dirichlet_tile64_H16_fp64"
    if a.workload == "schrodinger1d":
        return W.schrodinger1d(n=a.sn), a.prec, f"schrodinger1d_{a.sn}_periodic_kappa10_mu2_tile80_H20"
    if a.workload == "vardiff1d":
        name = f"vardiff1d_{a.vn}_dirichlet_tile64_H16_mu2" + (f"_trunc{a.trunc:g}" if a.trunc is not None else "")
        return W.vardiff1d(n=a.vn), a.prec, name
    name = f"vardiff2d_{a.vside}_dirichlet_tile16_H6_reaction" + ("_rb3" if a.scheme == "rb3" else "")
    return W.vardiff2d(side=a.vside), a.prec, name


def oracle_small_sample(a, max_seconds=8.0):
    """The FP64 oracle (as it stands) on a bounded sample of a single-problem workload: the
    propagators of up to 64 sampled tiles built once (Jacobian at u0 with the reaction), then
    LEM steps restricted to those tiles."""
    import oracle as O
    wl, _, _ = small_workload(a)
    X = O.assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = O.decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    J = O.jacobian(X, wl["u0"], wl["dt"], True) if wl["reaction"] else X
    sample = list(range(0, len(wins), max(1, len(wins) // 64)))[:64]
    t0 = time.perf_counter()
    props = O.local_propagators(J, wins, "phi", tiles=sample)
    t_build = time.perf_counter() - t0
    u = wl["u0"].copy()
    steps, t_step = 0, 0.0
    while t_step < max_seconds and steps < 200:
        t0 = time.perf_counter()
        u = O.lem_step(X, u, wins, props, "phi", wl["dt"], wl["reaction"], tiles=sample)
        t_step += time.perf_counter() - t0
        steps += 1
    dofs = sum(len(wins[i].D) for i in sample) * steps
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {"value": dofs / t_step, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{len(sample)} of {len(wins)} tiles x {steps} LEM steps (numpy FP64 oracle); "
                      f"their propagators took {t_build:.1f} s and are excluded"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if a.workload in ("heat1d", "vardiff2d", "vardiff1d", "schrodinger1d"):
        _, _, name = small_workload(a)
        if a.scheme == "rb3" and a.workload == "vardiff2d":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle's third-order Rosenbrock step "
                              "runs on whole meshes only (no bounded tile sample)", "config": {"workload": name}}),
                  flush=True)
            return
        per, cb = [], None
        for _ in range(a.warmup + a.steps):
            cb = oracle_small_sample(a, max_seconds=2.0)
            per.append(cb["value"])
        v = statistics.median(per[a.warmup:]) if len(per) > a.warmup else per[-1]
        cb["value"] = v
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": name, "impl": "FP64 CPU oracle on a tile sample"},
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if a.workload == "serve":
        cb = oracle_serve_sample(a.rate, a.duration)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC, "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": SERVE_WORKLOAD, "impl": "FP64 CPU oracle on a request sample"},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if a.workload == "batch512":
        per, cb = [], None
        for _ in range(a.warmup + a.steps):
            cb = oracle_batch_sample(a.nprob, a.inner, max_seconds=4.0)
            per.append(cb["value"])
        v = statistics.median(per[a.warmup:]) if len(per) > a.warmup else per[-1]
        cb["value"] = v
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD, "impl": "FP64 CPU oracle on a problem sample"},
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    per = []
    cb = None
    for _ in range(a.warmup + a.steps):
        cb = oracle_sample(a, max_seconds=4.0)
        per.append(cb["value"])
    v = statistics.median(per[a.warmup:]) if len(per) > a.warmup else per[-1]
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": advdiff_workload(a)[1], "impl": "FP64 CPU oracle on a tile sample"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(a):
    """Uneven batch: a.nprob independent periodic advection-diffusion problems (side
    32 U{2..16}, mu U[1, 50], tile {8, 16, 32}, overlap U{4..8}) advanced by one CUDA graph
    launch per bench step (a.inner LEM steps each). Replicas per rank for N > 1."""
    import torch
    import torch.distributed as dist
    from paper_1505_02248_gb300 import lem as L
    from paper_1505_02248_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    L.load()
    stream = torch.cuda.current_stream(dev)
    probs = W.batch_problems(n=a.nprob, seed=3)
    npts = [p["u0"].size for p in probs]
    t0 = time.perf_counter()
    ctxs = [L.Lem.from_workload(p, prec=a.prec, device=local, stream=stream.cuda_stream) for p in probs]
    states = [torch.tensor(p["u0"], device=dev) for p in probs]
    for c in ctxs:
        c.build()
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = L.Batch(ctxs, states, steps_per_launch=a.inner, lanes=a.lanes, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    schedule_s = time.perf_counter() - t0
    est, lane = batch.schedule()
    loads = np.bincount(lane, weights=est)
    sched = batch.info()
    paths = sorted({L.APPLY_PATHS[c.info()["apply_path"]] for c in ctxs})

    batch.run(a.warmup)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(a.steps):
            starts[k].record(stream)
            batch.run(1)
            stops[k].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, stops))
    dev_ms_max = max_over_ranks(dev_ms)
    total = sum(npts)

    # end to end: every problem's state from pinned host memory, one graph launch, back to host
    host = [torch.tensor(p["u0"]).pin_memory() for p in probs]
    e2e_ms = []
    for _ in range(max(3, min(a.steps, 5))):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for s, h in zip(states, host):
            s.copy_(h, non_blocking=True)
        batch.run(1)
        for s, h in zip(states, host):
            h.copy_(s, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    e2e_ms_med = statistics.median(e2e_ms)

    # dominant kernel (the split GEMM), algorithmic FLOPs = products x 2 x owner rows x window
    # nodes x windows. Fused schedule: the multi-problem GEMM launches of a.inner steps timed
    # with events outside the graph; lanes: each problem's launches timed on a copy of its state.
    gemm_ms, gemm_n, flops, prof, exec_flops = 0.0, 0, 0.0, None, None
    cands = batch.candidates()
    if sched["fused"]:
        prof = batch.profile(a.inner)
        gemm_ms, gemm_n, flops = prof["gemm_ms"], a.inner, prof["gemm_flops"]
        exec_flops = batch.gemm_work()[1] * a.inner
    else:
        nprod = {"split": 6, "split_fast": 4}.get(a.prec, 1)
        for p, c, s in zip(probs, ctxs, states):
            v = s.clone()
            c.set_timing(True)
            c.get_timing()
            c.step(v, 1)
            ms, n = c.get_timing()
            c.set_timing(False)
            gemm_ms += ms
            gemm_n += n
            (ty, tx), (hy, hx) = p["tile"], p["overlap"]
            ntiles = (p["shape"][0] // ty) * (p["shape"][1] // tx)
            flops += nprod * 2.0 * ty * tx * (ty + 2 * hy) * (tx + 2 * hx) * ntiles
    batch.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    tflops_peak, _, peak_src = peaks()
    value = job_rate(total * a.inner * a.steps, world, dev_ms_max)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": dev_ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"split": "f16x3-split/f32-acc", "split_fast": "f16x2-split/f32-acc"}.get(a.prec, "f64"),
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "problems": a.nprob, "nodes": total,
                   "lem_steps_per_step": a.inner, "lanes": int(len(loads)), "prec": a.prec, "apply_paths": paths,
                   "l2": "working set (states, residual pieces, propagator pieces) several GB > L2",
                   "parallelism": f"replicas x{world}", "build_s": round(build_s, 1),
                   "schedule_s": round(schedule_s, 1),
                   "schedule": "fused" if sched["fused"] else "lanes",
                   "candidate_ms_per_launch": {"lanes": sched["lanes_ms"], "fused": sched["fused_ms"]},
                   "autotuner": [{"schedule": "fused" if c["fused"] else "lanes",
                                  ("block_cap" if c["fused"] else "lanes"): c["n_cap"] if c["fused"] else c["lanes"],
                                  "ms": round(c["ms"], 4), "chosen": bool(c["chosen"])} for c in cands],
                   "lane_load_ms": {"max": float(loads.max()), "mean": float(loads.mean())}},
        # per problem and launch (lanes): max|r| pass (with the FP64 -> float-float conversion),
        # (residual + GEMM) per LEM step, float-float -> FP64 (split); residual, gather, GEMM,
        # scatter per step (FP64). Fused: conversion, max|r| pass, (residual + GEMM) per LEM
        # step, conversion back
        "gpu_launches": a.steps * (3 + 2 * a.inner) if sched["fused"] else
        a.steps * sum((2 + 2 * a.inner) if L.APPLY_PATHS[c.info()["apply_path"]] == "tc_split"
                      else 4 * a.inner for c in ctxs),
    }
    if gemm_n:
        ach = flops / (gemm_ms * 1e-3) / 1e12
        line["roofline"] = {"kernel": "split_gemm_kernel (tcgen05 kind::f16), " +
                            ("one multi-problem launch per step" if sched["fused"] else "per problem"),
                            "bound": "tensor",
                            "achieved": ach, "peak": tflops_peak, "unit": "TFLOP/s", "frac": ach / tflops_peak,
                            "traffic": None, "avg_launch_us": gemm_ms / gemm_n * 1e3, "launches": gemm_n,
                            "peak_source": f"{peak_src} bf16 dense (fp16 same rate)"}
        if exec_flops:
            line["roofline"]["executed_over_algorithmic"] = exec_flops / flops
            line["roofline"]["executed_frac"] = exec_flops / (gemm_ms * 1e-3) / 1e12 / tflops_peak
    line["e2e"] = {"value": total * a.inner / (e2e_ms_med * 1e-3), "unit": METRIC,
                   "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 8 * total, "ms_per_step": e2e_ms_med}
    line["clocks"] = clk.summary()
    if prof is not None:
        line["step_breakdown_ms"] = {"gemm": prof["gemm_ms"], "residual": prof["residual_ms"],
                                     "conversions": prof["other_ms"], "lem_steps": a.inner}
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = oracle_batch_sample(a.nprob, a.inner)
    print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    if world > 1:
        dist.destroy_process_group()


SERVE_WORKLOAD = "serve_poisson_1d2d_advdiff_periodic_tiers_1e-6_1e-10"


def serve_requests(rate, duration, seed=4, variants=8):
    """Poisson arrivals (mean `rate` per second for `duration` s), seed 4. Half 1D (N log-uniform
    in [256, 65536], rounded to 64, tile 64 + H 16), half 2D (side log-uniform in [128, 2048],
    rounded to 32, tile 32 + H 8); periodic upwind advection-diffusion, h = dt = 1, drawn from
    `variants` operators per dimension (mu ~ U[1, 20], C ~ U[0, 4], C_y = C / 2); steps U{1..50};
    tolerance tier 1e-6 (70 %) or 1e-10 (30 %)."""
    from paper_1505_02248_gb300 import workloads as W
    g = W.rng(seed)
    ops = {1: [], 2: []}
    for dim in (1, 2):
        for _ in range(variants):
            mu, c = float(g.uniform(1.0, 20.0)), float(g.uniform(0.0, 4.0))
            ops[dim].append(W.stencil_advdiff_1d(mu, c, 1.0, upwind=True) if dim == 1
                            else W.stencil_advdiff_2d(mu, c, c / 2, 1.0))
    t, out = 0.0, []
    while True:
        t += float(g.exponential(1.0 / rate))
        if t >= duration:
            break
        dim = 1 if g.random() < 0.5 else 2
        if dim == 1:
            n = int(round(np.exp(g.uniform(np.log(256), np.log(65536))) / 64)) * 64
            shape, tile, H = (n,), (64,), (16,)
        else:
            side = int(round(np.exp(g.uniform(np.log(128), np.log(2048))) / 32)) * 32
            shape, tile, H = (side, side), (32, 32), (8, 8)
        out.append(dict(t=t, shape=shape, bc=("periodic",) * dim, coef=ops[dim][int(g.integers(variants))],
                        dt=1.0, tile=tile, overlap=H, steps=int(g.integers(1, 51)),
                        tol=1e-6 if g.random() < 0.7 else 1e-10))
    return out


def run_serve(a):
    """Stream of requests through lem_server (continuous batching, 80 GB budget): submitted on
    their Poisson arrival times, latency arrival -> result back in host memory."""
    import torch
    from paper_1505_02248_gb300 import lem as L
    from paper_1505_02248_gb300 import workloads as W

    L.load()
    reqs = serve_requests(a.rate, a.duration)
    base = {}
    for r in reqs:  # one initial field per mesh size (a fresh copy per request)
        if r["shape"] not in base:
            base[r["shape"]] = (W.grf_1d(r["shape"][0], 8.0, 1) if len(r["shape"]) == 1
                                else W.grf_2d(r["shape"], 16.0, 1).ravel())
    states = [base[r["shape"]].copy() for r in reqs]
    srv = L.Server(80 * 10 ** 9)
    # warm-up: one small request per (operator, tier) builds every propagator of the catalogue
    # (the server keeps them and lends them to every mesh size), then the counters restart
    seen, warm = set(), []
    for r in reqs:
        key = (len(r["shape"]), tuple(sorted(r["coef"].items())), r["tol"])
        if key in seen:
            continue
        seen.add(key)
        shape = (256,) if len(r["shape"]) == 1 else (128, 128)
        h = (W.grf_1d(256, 8.0, 2) if len(shape) == 1 else W.grf_2d(shape, 16.0, 2).ravel())
        warm.append((srv.submit(shape, r["bc"], r["coef"], r["dt"], r["tile"], r["overlap"], h, 1, r["tol"]), h))
    t_w = time.perf_counter()
    for t, _ in warm:
        srv.wait(t, 300.0)
    warm_s = time.perf_counter() - t_w
    srv.reset_stats()
    tickets = []
    t0 = time.perf_counter()
    with ClockSampler(0) as clk:
        i = 0
        while i < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i]["t"] <= now:
                r = reqs[i]
                tickets.append(srv.submit(r["shape"], r["bc"], r["coef"], r["dt"], r["tile"], r["overlap"], states[i],
                                          r["steps"], r["tol"]))
                i += 1
            time.sleep(0.0002)
        t_sub = time.perf_counter() - t0
        while time.perf_counter() - t0 < a.duration + a.drain:
            st = srv.stats()
            if st["completed"] + st["failed"] >= len(reqs):
                break
            time.sleep(0.01)
    st = srv.stats()
    srv.close()
    dofs = sum(int(np.prod(r["shape"])) * r["steps"] for r in reqs)
    span = st["first_admit_to_last_done_s"]
    line = {
        "metric": METRIC, "value": st["dof_steps"] / span if span > 0 else None, "unit": METRIC, "n_gpus": 1,
        "steps": len(reqs), "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "mixed: f16x3-split (tier 1e-6, 2D) / f64", "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "rate_per_s": a.rate, "arrival_s": a.duration,
                   "submit_span_s": round(t_sub, 3), "requests": len(reqs), "offered_dof_steps": dofs,
                   "budget_bytes": 80 * 10 ** 9, "operator_variants_per_dim": 8,
                   "warmup": f"{len(warm)} one-step requests (one per operator and tier) in {warm_s:.1f} s, "
                             "then the counters restart"},
        "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"]},
        "tiers": {name: {"completed": st["tier_completed"][k], "dof_steps": st["tier_dof_steps"][k],
                         "p50_ms": st["tier_p50_ms"][k], "p99_ms": st["tier_p99_ms"][k],
                         "dof_steps_per_s": st["tier_dof_steps"][k] / span if span > 0 else None}
                  for k, name in enumerate(("1e-6 (split where eligible)", "1e-10 (FP64)"))},
        "requests": {k: st[k] for k in ("submitted", "admitted", "completed", "failed", "queued", "active")},
        "contexts": {"hits": st["ctx_hits"], "misses": st["ctx_misses"], "adopted_propagators": st["ctx_adopted"]},
        "worker_s": {"admit": st["worker_admit_s"], "issue": st["worker_issue_s"], "build": st["worker_build_s"],
                     "contexts_built": st["ctx_built"], "adopt_failed": st["adopt_failed"]},
        "gpu_launches": None,
        "e2e": {"value": st["dof_steps"] / span if span > 0 else None, "unit": METRIC,
                "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "every request's state goes host -> device -> host inside its latency"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_small(a):
    """Config-style single problems on their own paths: heat1d (1D Dirichlet heat, N = 1024,
    FP64, three propagator classes) and vardiff2d (1024^2 variable-coefficient diffusion with
    the reaction, per-tile propagators applied by the batched GEMV; the Jacobian is frozen at
    u0 for the timed steps and one propagator build is timed separately)."""
    import torch
    from paper_1505_02248_gb300 import lem as L
    from paper_1505_02248_gb300 import workloads as W

    L.load()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    # schrodinger1d: the Sec. 4.1 equation at the paper's size (400 points, 5 subdomains,
    # buffer 20) or on a finer mesh over the same interval (same mu: smaller dt)
    wl, prec, name = small_workload(a)
    npts = wl["u0"].size
    ctx = L.Lem.from_workload(wl, prec=prec, stream=stream.cuda_stream,
                              scheme=a.scheme if a.workload == "vardiff2d" else "euler")
    if a.trunc is not None:
        ctx.set_truncation(a.trunc)
    u = torch.tensor(wl["u0"], device=dev)
    t0 = time.perf_counter()
    ctx.build(u)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    band_values = None
    if a.trunc is not None:
        band_values = ctx.band_total()  # values of all packed boxes (extents from this build)
    info = ctx.info()
    path = L.APPLY_PATHS[info["apply_path"]]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(a.warmup):
        ctx.step(u, a.inner)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ctx.set_timing(True)
    ctx.get_timing()
    with ClockSampler(0) as clk:
        for k in range(a.steps):
            flush.zero_()
            starts[k].record(stream)
            ctx.step(u, a.inner)
            stops[k].record(stream)
        torch.cuda.synchronize()
    k_ms, k_n = ctx.get_timing()
    ctx.set_timing(False)
    # small linear problems run all of a call's steps in one persistent launch
    persistent = bool(k_n) and k_n == a.steps and a.inner > 1
    dev_ms = sum(x.elapsed_time(y) for x, y in zip(starts, stops))
    h = wl["u0"].copy()
    ctx.step_host(h, 1)
    e2e = []
    for _ in range(3):
        t1 = time.perf_counter()
        ctx.step_host(h, a.inner)
        e2e.append((time.perf_counter() - t1) * 1e3)
    _, hbm_peak, peak_src = peaks()
    line = {"metric": METRIC, "value": npts * a.inner * a.steps / (dev_ms * 1e-3), "unit": METRIC, "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dev_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("c128 (real-embedded f64)" if ctx.complex else "f64") if path.startswith("fp64") else
                     ("c64 (real-embedded f32)/ff-acc" if ctx.complex else "f32-gemv/ff-acc"),
            "data": "synthetic",
            "config": {"workload": name, "nodes": npts, "lem_steps_per_step": a.inner, "apply_path": path,
                       "scheme": a.scheme if a.workload == "vardiff2d" else "euler",
                       "propagator_classes": info["nclasses"], "n_loc": info["n_loc"], "n_int": info["n_int"],
                       "build_s": round(build_s, 2), "l2": "256 MiB write between timed steps"},
            "gpu_launches": a.steps if persistent else
                            a.steps * a.inner * ((2 if ("gemv" in path or "band" in path) else 4) +
                                                 (3 if a.scheme == "rb3" else 0)),
            "e2e": {"value": npts * a.inner / (statistics.median(e2e) * 1e-3), "unit": METRIC,
                    "h2d_bytes_per_step": (16 if ctx.complex else 8) * npts,
                    "d2h_bytes_per_step": (16 if ctx.complex else 8) * npts},
            "clocks": clk.summary()}
    if band_values is not None:
        dense_values = info["nclasses"] * info["n_int"] * info["n_loc"]
        line["config"]["truncation"] = {"tol": a.trunc, "kept_values": band_values, "dense_values": dense_values,
                                        "kept_frac": band_values / dense_values}
    if k_n and "band" in path:
        pbytes = (4 if path == "f32_band" else 8) * band_values
        ach = pbytes / (k_ms / k_n * 1e-3) / 1e9
        line["roofline"] = {"kernel": f"gemv_band_kernel ({path})", "bound": "hbm", "achieved": ach,
                            "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak, "traffic": None,
                            "avg_launch_us": k_ms / k_n * 1e3, "launches": k_n,
                            "algorithmic_bytes": "truncated propagator boxes streamed once per step (the packed "
                                                 "values of every tile's owner rows)",
                            "peak_source": f"{peak_src} HBM copy"}
    elif k_n and "gemv" in path:
        pbytes = (4 if path == "f32_gemv" else 8) * info["nclasses"] * info["n_int"] * info["n_loc"]
        if ctx.complex:
            pbytes //= 2  # the Re and Im rows of each owner, left halves of the stored embedding
        if a.scheme == "rb3":
            pbytes *= 2  # phi_1 and phi_3 propagators, one GEMV each per step (timed together)
        steps_per_launch = a.inner if persistent else 1
        ach = pbytes * steps_per_launch / (k_ms / k_n * 1e-3) / 1e9
        kname = "gemv_persistent_kernel (all steps of a call in one cooperative launch)" if persistent else \
            f"gemv_tiles_kernel ({path})"
        line["roofline"] = {"kernel": kname, "bound": "hbm", "achieved": ach, "steps_per_launch": steps_per_launch,
                            "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak, "traffic": None,
                            "avg_launch_us": k_ms / k_n * 1e3, "launches": k_n,
                            "algorithmic_bytes": "propagators streamed once per step (n_int x n_loc per tile; complex: its Re and "
                                 "Im planes, n_int x n_loc / 2 of the stored real embedding)",
                            "peak_source": f"{peak_src} HBM copy"}
    elif k_n:
        line["roofline"] = {"kernel": "dgemm_kernel (FP64 apply)", "bound": "alu", "avg_launch_us": k_ms / k_n * 1e3,
                            "launches": k_n, "note": "latency-bound at this size (16 windows)"}
    if not a.no_cpu_baseline and not (a.workload == "vardiff2d" and a.scheme == "rb3"):
        line["cpu_baseline"] = oracle_small_sample(a)
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.workload in ("heat1d", "vardiff2d", "vardiff1d", "schrodinger1d") and a.impl == "ours":
        run_small(a)
        return
    if a.workload == "serve" and a.impl == "ours":
        run_serve(a)
        return
    if a.impl == "reference":
        run_reference(a)
        return
    if a.workload == "batch512":
        run_batch(a)
        return
    import torch
    import torch.distributed as dist
    from paper_1505_02248_gb300 import lem as L
    from paper_1505_02248_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    L.load()

    wl, workload_name = advdiff_workload(a, seed=1 + rank)
    npts = wl["u0"].size
    stream = torch.cuda.current_stream(dev)
    ctx = L.Lem.from_workload(wl, prec=a.prec, device=local, stream=stream.cuda_stream)
    u = torch.tensor(wl["u0"], device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    t0 = time.perf_counter()
    ctx.build()
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3

    for _ in range(a.warmup):
        ctx.step(u, a.inner)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # the split GEMM of the first LEM step of every call is bracketed by events (an event
    # between two launches keeps the later one from starting its set-up early, so timing every
    # launch would slow the steps it measures)
    split_path = L.APPLY_PATHS[ctx.info()["apply_path"]] == "tc_split"
    ctx.set_timing(True, period=a.inner if split_path else 1)
    ctx.get_timing()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        for k in range(a.steps):
            flush.zero_()
            starts[k].record(stream)
            ctx.step(u, a.inner)
            stops[k].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    gemm_ms, gemm_launches = ctx.get_timing()
    ctx.set_timing(False)
    if world > 1:
        dist.barrier()
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, stops))
    dev_ms_max = max_over_ranks(dev_ms)
    total_lem_steps = a.warmup * a.inner + a.steps * a.inner

    # end to end through the public host API: pinned host state, H2D + steps + D2H per call
    h = torch.tensor(wl["u0"]).pin_memory()
    hn = h.numpy()
    ctx.step_host(hn, 1)
    e2e_ms = []
    for k in range(max(3, min(a.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.step_host(hn, a.inner)
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    e2e_ms_med = statistics.median(e2e_ms)

    # numerical check of the timed run against the plain FP64 GPU LEM (same start, same steps)
    err = None
    fp64_rate = None
    if a.prec != "fp64" and not a.no_fp64_compare and total_lem_steps <= 400:
        ref = L.Lem.from_workload(wl, prec="fp64", device=local, stream=stream.cuda_stream)
        v = torch.tensor(wl["u0"], device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ref.build()
        e0.record(stream)
        ref.step(v, total_lem_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_rate = npts * total_lem_steps / (e0.elapsed_time(e1) * 1e-3)
        err = float(torch.linalg.vector_norm(u - v) / torch.linalg.vector_norm(v))
        ref.close()

    # the two-piece tier on the same workload, same start (reported beside the main line)
    alt = None
    if a.prec == "split" and not a.no_fp64_compare and err is not None:
        fast = L.Lem.from_workload(wl, prec="split_fast", device=local, stream=stream.cuda_stream)
        w = torch.tensor(wl["u0"], device=dev)
        fast.build()
        fast.step(w, total_lem_steps - a.steps * a.inner)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        fast.set_timing(True, period=a.inner)
        fast.get_timing()
        e0.record(stream)
        fast.step(w, a.steps * a.inner)
        e1.record(stream)
        torch.cuda.synchronize()
        fms, fn = fast.get_timing()
        inf = fast.info()
        flops4 = 4 * 2.0 * inf["n_int"] * inf["n_loc"] * (npts // inf["n_int"])
        alt = {"split_fast": {"value": npts * a.steps * a.inner / (e0.elapsed_time(e1) * 1e-3),
                              "unit": METRIC, "rel_l2_vs_fp64_gpu": float(torch.linalg.vector_norm(w - v) /
                                                                          torch.linalg.vector_norm(v)),
                              "gemm_us": fms / fn * 1e3, "gemm_tflops": flops4 / (fms / fn * 1e-3) / 1e12,
                              "note": "two FP16 pieces (four products); no L2 flush between its steps"}}
        fast.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    tflops_peak, hbm_peak, peak_src = peaks()
    khash = kernel_source_hash()
    value = job_rate(npts * a.inner * a.steps, world, dev_ms_max)
    info = ctx.info()
    ntiles = npts // info["n_int"]
    # algorithmic flop of one FP16 product over all windows: 2 n_int n_loc per window
    flops1 = 2.0 * info["n_int"] * info["n_loc"] * ntiles
    path = L.APPLY_PATHS[info["apply_path"]]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": METRIC,
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": dev_ms_max / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"split": "f16x3-split/f32-acc", "split_fast": "f16x2-split/f32-acc"}.get(a.prec, "f64"),
        "data": "synthetic",
        "config": {"workload": workload_name, "nodes": npts, "tiles": ntiles,
                   "propagator": f"{info['n_int']}x{info['n_loc']} phi_1 (shared)", "lem_steps_per_step": a.inner,
                   "prec": a.prec, "apply_path": path, "l2": "256 MiB write between timed steps",
                   "parallelism": f"replicas x{world}", "build_ms": round(build_ms, 1)},
        # split: max|r| pass (which also converts FP64 -> float-float), (residual + GEMM) per LEM
        # step, float-float -> FP64; FP64: residual, gather, GEMM, scatter per LEM step
        "gpu_launches": a.steps * ((2 + 2 * a.inner) if path == "tc_split" else
                                   a.inner * (2 if "gemv" in path else 4)),
    }
    if gemm_launches:
        avg_ms = gemm_ms / gemm_launches
        if path == "tc_split":
            nprod = 6 if a.prec == "split" else 4  # FP16 products per split GEMM
            flops = nprod * flops1
            line["roofline"] = {"kernel": "split_gemm_kernel (tcgen05 kind::f16)", "bound": "tensor",
                                "achieved": flops / (avg_ms * 1e-3) / 1e12, "peak": tflops_peak,
                                "unit": "TFLOP/s", "frac": flops / (avg_ms * 1e-3) / 1e12 / tflops_peak,
                                "traffic": ncu_traffic(khash) if workload_name == WORKLOAD else None,
                                "avg_launch_us": avg_ms * 1e3,
                                "launches": gemm_launches, "peak_source": f"{peak_src} bf16 dense (fp16 same rate)",
                                "kernel_hash": khash}
        else:
            flops = flops1
            fp64_peak = fp64_dgemm_tflops(dev)
            line["roofline"] = {"kernel": "dgemm_kernel (FP64 apply)", "bound": "alu",
                                "achieved": flops / (avg_ms * 1e-3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                                "frac": flops / (avg_ms * 1e-3) / 1e12 / fp64_peak, "traffic": None,
                                "avg_launch_us": avg_ms * 1e3, "launches": gemm_launches,
                                "peak_source": "cuBLAS FP64 GEMM (torch.matmul, 8192^3, best of 5) measured in this run"}
    line["e2e"] = {"value": npts * a.inner / (e2e_ms_med * 1e-3), "unit": METRIC,
                   "h2d_bytes_per_step": 8 * npts, "d2h_bytes_per_step": 8 * npts,
                   "ms_per_step": e2e_ms_med}
    line["clocks"] = clk.summary()
    if err is not None:
        line["rel_l2_vs_fp64_gpu"] = err
        line["fp64_gpu_lem"] = {"value": fp64_rate, "unit": METRIC, "lem_steps": total_lem_steps}
    if alt is not None:
        for k, d in alt.items():
            d["gemm_frac_of_peak"] = d["gemm_tflops"] / tflops_peak
        line["alt_tiers"] = alt
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(a)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
