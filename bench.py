"""Benchmark of the CGP time step on one GB300 (or N independent replicas under torchrun).

Workload: the backward-facing-step channel [0,30]x[0,2] minus [0,1]^2, jittered random-diagonal
coarse mesh with h = 1/33 (65,308 coarse / 259,117 fine nodes, one 1:4 refinement), Re = 400,
dt = 0.005, rtol = 1e-8 for every solve (the paper's Sect. 2.3 tolerance). A "step" is one whole
cgp_step (Eqs. 19-23). The state is warmed up for W steps from rest, then K steps are timed one
by one with CUDA events on the launching stream; between timed steps L2 is flushed (outside the
timed region) by writing a 512 MB buffer and then reading a 256 MB one, so it holds clean lines.
A second measurement times the Krylov SpMV on a matrix larger than L2 (the HBM roofline).

Prints one JSON line: steps/s (value), coarse Poisson solves/s, the roofline of the dominant
kernel (the persistent coarse CG), the end-to-end rate through cgp_step_host with host buffers,
and the oracle timed on the host cores (cpu_baseline). ``--impl reference`` times the CPU oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import cgp_inputs as ci  # noqa: E402

WORKLOAD = "bfs33"       # the headline workload; --workload cylinder / cavity33 time the other meshes
DESCR = {"bfs33": "backward-facing step",
         "cylinder": "flow past a cylinder, graded Poisson-disk Delaunay mesh, slip walls",
         "cavity33": "lid-driven cavity"}
METRIC = "time steps/sec & coarse Poisson solves/sec at 1e-8 rel. residual; SpMV HBM GB/s vs peak"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class L2Flush:
    """Evicts L2 between timed regions: writes a 512 MB buffer, then reads a separate 256 MB buffer,
    so L2 is left holding clean lines and no write-back of the flush overlaps the timed kernels."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.acc = torch.zeros((), dtype=torch.float32, device=dev)

    def fill_(self, v):
        import torch
        self.w.fill_(v)
        torch.sum(self.r, dim=0, out=self.acc)


def measured_traffic(kernel: str, workload: str = WORKLOAD):
    """DRAM bytes per launch of ``kernel`` from the committed ncu capture, or None when there is
    none or the kernel's source has changed since it was taken (its SHA-256 is recorded)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != rec["sha256"]:
                return None
        return rec["bytes_per_launch"] if rec.get("workload") == workload else None
    except Exception:
        return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_time_ms(ms: float, ws: int, device) -> float:
    """The job's time per step: the maximum of the ranks' times (each rank runs its own replica;
    the slowest one bounds the whole job). Identity for a single rank."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms: float, ws: int) -> float:
    """Whole-job throughput: the units all ranks processed per second at the job's step time."""
    return ws * units_per_rank * 1000.0 / ms


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(n_steps: int, n_warmup: int = 0):
    """Time the CPU oracle on the same workload: setup once, ``n_warmup`` untimed steps from rest,
    then ``n_steps`` timed steps."""
    from oracle import cgp as ocgp
    coarse, prob, _ = ci.workload(WORKLOAD)
    t0 = time.perf_counter()
    orc = ocgp.CGPOracle(coarse.xy, coarse.tri, prob.rho, prob.mu, prob.dt, prob.levels, prob.vel_bc, prob.p_bc)
    t_setup = time.perf_counter() - t0
    mask, g = orc.dirichlet(0.0)
    u = prob.u0(orc.fine.xy, mask, g)
    times = []
    for k in range(n_warmup + n_steps):
        t0 = time.perf_counter()
        r = orc.step(u, (k + 1) * prob.dt)
        if k >= n_warmup:
            times.append(time.perf_counter() - t0)
        u = r.u
    try:
        from threadpoolctl import threadpool_info
        cores = max([1] + [int(i.get("num_threads", 1)) for i in threadpool_info()])
    except Exception:
        cores = 1
    return times, t_setup, cores


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    # about 3 s per oracle step: at most 3 warm-up and 10 timed steps keep the run near a minute
    n_warm, n_steps = min(args.warmup, 3), max(1, min(args.steps, 10))
    times, t_setup, cores = oracle_sample(n_steps, n_warm)
    ms = 1000.0 * statistics.mean(times)
    v = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": n_steps, "warmup": n_warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: {DESCR[WORKLOAD]}, coarse 65,308 / fine 259,117 nodes, l=1, "
                                   f"Re=400, dt=0.005", "rtol": "direct LU (the oracle)"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{len(times)} oracle steps after {n_warm} untimed steps from rest and a "
                                       f"{t_setup:.1f}s setup (requested: {args.steps} steps, {args.warmup} warm-up)"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def spmv_hbm(L, Flow, dev, flush, stream, reps: int = 10):
    """The Krylov SpMV (two right-hand sides, FP64) on a matrix larger than L2: the backward-facing
    step at h = 1/48 refined twice (~2.2M rows, ~15M nnz, ~265 MB per product). Algorithmic bytes
    per product: 12 nnz (values, columns) + 4 (n + 1) (row pointers) + 16 n (x) + 16 n (y)."""
    import torch
    coarse = ci.bfs_mesh(48, 1001)
    prob = ci.bfs_problem(400.0, 0.005, 2)
    peak, kind = peaks()
    best = None
    for fmt, kname in ((2, "k_spmv_probe<2> (CSR, autotuned lanes)"), (1, "k_spmv_sell2 (sliced ELL, 32-row slices)")):
        f = Flow(coarse, prob, device=dev, spmv_format=fmt)
        L.cgp_autotune(f.ctx, stream)
        info = L.cgp_mesh_info(f.ctx)
        n, nnz = info.n_fine, info.nnz_fine
        x = torch.randn(n, 2, dtype=torch.float64, device=dev)
        y = torch.empty_like(x)
        L.cgp_spmv(f.ctx, x, y, stream)
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.cgp_spmv(f.ctx, x, y, stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        f.close()
        t = statistics.median(ms)
        nbytes = 12 * nnz + 4 * (n + 1) + 32 * n
        gbs = nbytes / (t * 1e-3) / 1e9
        rec = {"kernel": kname, "workload": f"bfs48 l=2 fine A0: {n} rows, {nnz} nnz, 2 RHS", "bytes": nbytes,
               "ms": t, "achieved": gbs, "unit": "GB/s", "peak": peak, "frac": gbs / peak, "peak_kind": kind,
               "lanes": info.spmv_lanes, "l2": "flushed before each product (512 MB write, then 256 MB read)"}
        if best is None or gbs > best["achieved"]:
            if best is not None:
                rec["other"] = {"kernel": best["kernel"], "achieved": best["achieved"]}
            best = rec
        else:
            best["other"] = {"kernel": rec["kernel"], "achieved": rec["achieved"]}
    return best


def run_gpu(args):
    import torch
    from paper_1610_06993_gb300 import cgp as L
    from paper_1610_06993_gb300.flow import Flow

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if not os.path.exists(L.LIB_PATH):
        raise RuntimeError("libcgp.so is not built; run python -c 'import __graft_entry__ as g; g.build()'")
    wname = args.workload
    coarse, prob, _ = ci.workload(wname)
    prec = L.CGP_MIXED if args.precision == "mixed" else L.CGP_FP64
    f = Flow(coarse, prob, precision=prec, rtol=args.rtol, device=f"cuda:{local}",
             block_threads=args.threads, spmv_lanes=args.lanes, coarse_solver=args.coarse_solver,
             precond_degree=args.precond_degree, precond_ratio=args.precond_ratio,
             **({"warm_start": args.warm_start} if args.warm_start >= 0 else {}),
             **({"inner_rtol": args.inner_rtol} if args.inner_rtol > 0 else {}),
             **({"mass_degree": args.mass_degree} if args.mass_degree > 0 else {}))
    stream = torch.cuda.current_stream()
    flush = L2Flush(f"cuda:{local}")
    bc = torch.empty_like(f.pc)
    ut = torch.empty_like(f.u)

    def step_parts(ev):
        """One cgp_step through its stage entry points, with events around the Poisson solve."""
        L.cgp_assemble(f.ctx, f.u, stream)
        L.cgp_momentum_solve(f.ctx, f.u, ut, stream)
        L.cgp_restrict(f.ctx, ut, bc, stream)
        if f.params.warm_start >= 1:
            L.cgp_predict_pressure(f.ctx, f.pc, stream)
        ev[0].record(stream)
        L.cgp_poisson_solve(f.ctx, bc, f.pc, stream)
        ev[1].record(stream)
        L.cgp_prolong_correct(f.ctx, f.pc, ut, f.u, None, None, stream)

    for _ in range(args.warmup):
        L.cgp_step(f.ctx, f.u, f.pc, stream)
    L.cgp_get_stats(f.ctx, stream, check=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    step_ms, poi_ms, poi_iters, poi_outer, mom_iters, mass_iters = [], [], [], [], [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[2].record(stream)
            step_parts(e)
            e[3].record(stream)
            st = L.cgp_get_stats(f.ctx, stream, check=True)
            step_ms.append(e[2].elapsed_time(e[3]))
            poi_ms.append(e[0].elapsed_time(e[1]))
            poi_iters.append(st.poisson_iters)
            poi_outer.append(st.poisson_outer)
            mom_iters.append(st.momentum_iters)
            mass_iters.append(st.mass_iters)
    torch.cuda.synchronize()
    ms = job_time_ms(statistics.mean(step_ms), ws, f"cuda:{local}")

    # end to end through the host-buffer entry point (copies inside the timed region)
    uh = torch.empty(f.u.shape, dtype=torch.float64, pin_memory=True)
    ph = torch.empty(f.pc.shape, dtype=torch.float64, pin_memory=True)
    uh.copy_(f.u)
    ph.copy_(f.pc)
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        L.cgp_step_host(f.ctx, uh, ph, stream)
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    L.cgp_get_stats(f.ctx, stream, check=True)
    h2d = (2 * f.info.n_fine + f.info.n_coarse) * 8

    # roofline of the dominant kernel: the persistent coarse CG, algorithmic bytes per launch
    nnz, n = f.info.nnz_coarse, f.info.n_coarse
    it = statistics.mean(poi_iters)
    outer = statistics.mean(poi_outer)
    if prec == L.CGP_FP64:
        per_iter = 12 * nnz + 60 * n
    else:
        per_iter = 8 * nnz + 32 * n
    if f.info.coarse_kernel in (3, 4):
        # Schwarz preconditioner: degree - 1 Chebyshev products with the subdomain matrices
        # (FP32 values + columns, read and write of the iterate) per application
        deg = args.precond_degree if args.precond_degree > 0 else 6
        per_iter += (deg - 1) * (8 * nnz + 8 * n)
    per_pass = 12 * nnz + 20 * n + 8 * n       # FP64 true residual (+ x update) per refinement pass
    alg_bytes = it * per_iter + (outer + 1) * per_pass
    pms = statistics.mean(poi_ms)
    achieved = alg_bytes / (pms * 1e-3) / 1e9
    peak, peak_kind = peaks()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and wname == WORKLOAD:
        times, t_setup, cores = oracle_sample(args.cpu_steps)
        cpu = {"value": 1.0 / statistics.mean(times), "unit": "steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(times)} oracle steps of the same workload from rest (setup {t_setup:.1f}s excluded)"}

    launches_per_step = 9 + f.info.levels + (4 if f.params.warm_start >= 1 else 0)
    tname = "double" if prec == L.CGP_FP64 else "float"
    kname = {0: f"k_cg<{tname}, 1>", 1: f"k_pcg_onchip<{tname}>", 2: f"k_pcg_pipe<{tname}>",
             3: "k_pcg_schwarz<double, float>", 4: f"k_pcg_schwarz<{tname}, {tname}>"}[f.info.coarse_kernel]
    line = {
        "metric": METRIC, "value": job_rate(1.0, ms, ws), "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == L.CGP_FP64 else "f32+f64-ir", "data": "synthetic",
        "config": {"workload": f"{wname}: {DESCR[wname]}, coarse {f.info.n_coarse:,} / fine {f.info.n_fine:,} nodes, "
                               f"l={f.info.levels}, Re={prob.mu and round(1.0 / prob.mu * (2.0 if wname == 'bfs33' else 1.0))}, "
                               f"dt={prob.dt}", "rtol": args.rtol, "precision": args.precision,
                   "l2": "flushed between timed steps (512 MB write, then 256 MB read)", "parallelism": "replicas" if ws > 1 else "1gpu",
                   "block_threads": f.info.block_threads, "grid_blocks": f.info.grid_blocks,
                   "spmv_lanes": f.info.spmv_lanes, "coarse_kernel": kname,
                   "precond_degree": args.precond_degree,
                   "coarse_initial_guess": {0: "p^n", 1: "2 p^n - p^(n-1)",
                                            2: "3 p^n - 3 p^(n-1) + p^(n-2)",
                                            3: "4 p^n - 6 p^(n-1) + 4 p^(n-2) - p^(n-3)"}[f.params.warm_start]},
        "coarse_solves_per_s": 1000.0 / pms,
        "poisson_ms": pms, "poisson_iters": it, "poisson_outer": outer,
        "momentum_iters": statistics.mean(mom_iters), "mass_iters": statistics.mean(mass_iters),
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": measured_traffic(kname, wname),
                     "alg_bytes_per_launch": alg_bytes,
                     "note": "coarse matrix + vectors live in shared memory, registers and L2 (ncu: 0.1 % DRAM "
                             "throughput); the kernel is bound by barrier latency, so achieved is an effective rate: "
                             "the bytes a memory-streaming CG would move per iteration x iterations / time",
                     "latency": {"us_per_iter": 1000.0 * pms / max(it, 1.0), "grid_barriers_per_iter": 2}},
        "e2e": {"value": 1000.0 / statistics.mean(e2e_ms), "unit": "steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": h2d},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    f.close()
    if not args.no_spmv:
        line["spmv_hbm"] = spmv_hbm(L, Flow, f"cuda:{local}", flush, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """64 independent cavities (coarse sizes log-uniform in [2k, 50k], Re in [100, 1000], dt =
    0.005, one refinement), advanced together by the batched step replayed as a CUDA graph.

    value = aggregate instance-steps/s. Coarse-solve throughput is compared in the same run:
    the plain path (FP64, zero initial guess, one instance after another through
    cgp_poisson_solve) against the batched path (this run's precision, previous-step pressure as
    the initial guess, one launch for all instances), on the same right-hand sides at rtol."""
    import torch
    from paper_1610_06993_gb300 import cgp as L
    from paper_1610_06993_gb300.flow import Batch, Flow

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    cases = ci.batch_cavities()
    prec = L.CGP_MIXED if args.precision == "mixed" else L.CGP_FP64
    flows = [Flow(m, p, precision=prec, rtol=args.rtol, device=dev) for m, p in cases]
    for f in flows:
        L.cgp_autotune(f.ctx)                        # per-instance SpMV lanes (project autotuner)
    b = Batch(flows)
    stream = torch.cuda.current_stream()
    flush = L2Flush(dev)
    b.run(args.warmup, stream)
    b.stats(check=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(1, stream)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    st = b.stats(check=True)
    ms = job_time_ms(statistics.mean(step_ms), ws, dev)
    n_inst = len(flows)

    # coarse solves: batched, warm-started from the previous step's pressure
    prev = [f.pc.clone() for f in flows]
    prev_u = [f.u.clone() for f in flows]
    b.run(1, stream)
    for f, p in zip(flows, prev):
        f.pc.copy_(p)
    flush.fill_(1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.cgp_batch_poisson_solve(b.handle, stream)
    e1.record(stream)
    e1.synchronize()
    t_batch = e0.elapsed_time(e1)
    it_batch = [s.poisson_iters for s in b.stats(check=True)]
    # plain: FP64 contexts on the same right-hand sides, zero initial guess, one after another;
    # coarse_solver 5 is the paper's Jacobi-preconditioned CG, 0 this library's default (two-level
    # Schwarz preconditioned CG)
    plain = {}
    for solver in (5, 0):
        t_plain, it_plain = 0.0, []
        for f, u0, (m, p) in zip(flows, prev_u, cases):
            g = Flow(m, p, precision=L.CGP_FP64, rtol=args.rtol, device=dev, coarse_solver=solver)
            bc = torch.empty_like(f.pc)
            ut = torch.empty_like(f.u)
            # the right-hand side of the batched instance's latest step, rebuilt on the FP64 context
            L.cgp_assemble(g.ctx, u0, stream)
            L.cgp_momentum_solve(g.ctx, u0, ut, stream)
            L.cgp_restrict(g.ctx, ut, bc, stream)
            x = torch.zeros_like(f.pc)
            torch.cuda.synchronize()
            e0.record(stream)
            L.cgp_poisson_solve(g.ctx, bc, x, stream)
            e1.record(stream)
            e1.synchronize()
            t_plain += e0.elapsed_time(e1)
            it_plain.append(g.stats(check=True).poisson_iters)
            g.close()
        plain[solver] = (t_plain, it_plain)

    line = {
        "metric": METRIC, "value": job_rate(n_inst, ms, ws), "unit": "instance-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == L.CGP_FP64 else "f32+f64-ir", "data": "synthetic",
        "config": {"workload": "batch64: 64 lid-driven cavities, coarse nodes log-uniform in [2k, 50k] "
                               f"(total {sum(f.info.n_coarse for f in flows)} coarse / "
                               f"{sum(f.info.n_fine for f in flows)} fine), Re U[100,1000], dt=0.005, l=1",
                   "rtol": args.rtol, "precision": args.precision, "graph": "one CUDA graph per step",
                   "l2": "flushed between timed steps (512 MB write, then 256 MB read)", "blocks": b.blocks},
        "coarse_solves_per_s": {"batched_warm": n_inst * 1000.0 / t_batch,
                                "plain_fp64_jacobi_zero_sequential": n_inst * 1000.0 / plain[5][0],
                                "ratio": plain[5][0] / t_batch,
                                "plain_fp64_schwarz_zero_sequential": n_inst * 1000.0 / plain[0][0],
                                "ratio_vs_schwarz": plain[0][0] / t_batch,
                                "iters_batched_mean": statistics.mean(it_batch),
                                "iters_plain_jacobi_mean": statistics.mean(plain[5][1]),
                                "iters_plain_schwarz_mean": statistics.mean(plain[0][1])},
        "gpu_launches": None, "clocks": clk.summary(),
    }
    b.close()
    for f in flows:
        f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_warmstart(args):
    """Learned warm start on the 129x129-node cavity: (b_c, p_c) pairs logged from seeded runs
    (Re uniform in [100, 1000], dt = 0.005) by the batched solver, an 80/20 split by run, training
    by the tensor-core kernels, then a batch of 256 held-out right-hand sides solved to rtol from
    zero, previous-step and network initial guesses (network inference time included)."""
    import torch
    from paper_1610_06993_gb300 import cgp as L, warmstart
    from paper_1610_06993_gb300.flow import Flow

    ws_, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    mesh, _, _ = ci.workload("cavity129")
    res = 100.0 + 900.0 * ci.uniform01(1004, np.arange(args.runs))
    problems = [ci.cavity_problem(float(r), 0.005, 1) for r in res]
    t0 = time.perf_counter()
    B, P, Pp, run, held = warmstart.generate(mesh, problems, args.run_steps)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    test = run >= int(round(0.8 * args.runs))
    n = B.shape[1]
    w = L.cgp_ws_create(n, 512, 256)
    L.cgp_ws_set_params(w, ci.mlp_init_params(n, 512, 4))
    L.cgp_ws_set_mask(w, held)
    t0 = time.perf_counter()
    hist = warmstart.train(w, B[~test].contiguous(), P[~test].contiguous(), epochs=args.epochs, batch=256, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    idx = torch.nonzero(test).flatten()
    idx = idx[torch.randperm(idx.numel(), generator=torch.Generator().manual_seed(5)).to(idx.device)[:256]]
    f = Flow(mesh, problems[0], rtol=args.rtol)
    out = warmstart.evaluate(f, w, B[idx].contiguous(), P[idx].contiguous(), Pp[idx].contiguous())
    f.close()
    L.cgp_ws_destroy(w)
    line = {"metric": "coarse Poisson solves/s at rtol with zero / previous-step / learned warm starts",
            "value": out["network"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16 network, f64 CG", "data": "synthetic",
            "config": {"workload": f"cavity129 (16,641 coarse nodes), {args.runs} runs x {args.run_steps} steps, "
                                   f"Re U[100,1000], network 16641-512-512-16641 GELU, batch 256, {args.epochs} epochs",
                       "rtol": args.rtol},
            "pairs": int(B.shape[0]), "gen_s": t_gen, "train_s": t_train, "loss_first_last": [hist[0], hist[-1]],
            "results": out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="bfs33",
                    choices=["bfs33", "cylinder", "cavity33", "batch64", "warmstart", "spmv"])
    ap.add_argument("--runs", type=int, default=100)
    ap.add_argument("--run-steps", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--coarse-solver", type=int, default=0)
    ap.add_argument("--precond-degree", type=int, default=0)
    ap.add_argument("--precond-ratio", type=float, default=0.0)
    ap.add_argument("--warm-start", type=int, default=-1)
    ap.add_argument("--inner-rtol", type=float, default=0.0)   # 0: the library default (1e-4)
    ap.add_argument("--mass-degree", type=int, default=0)      # 0: the library default (4)   # -1: the library default (1, extrapolation)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-spmv", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "warmstart":
        run_warmstart(args)
    elif args.workload == "spmv":
        import torch
        from paper_1610_06993_gb300 import cgp as L
        from paper_1610_06993_gb300.flow import Flow
        torch.cuda.set_device(0)
        flush = L2Flush("cuda:0")
        print(json.dumps(spmv_hbm(L, Flow, "cuda:0", flush, torch.cuda.current_stream(), reps=args.steps)), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
