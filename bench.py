"""Benchmark of the CGP time step on one GB300 (or N independent replicas under torchrun).

Headline workload: flow past a cylinder (Sect. 3.3 geometry): 63,485 coarse nodes of a graded
Poisson-disk Delaunay mesh, two 1:4 refinements to 1,006,982 fine nodes, Re = 100, dt = 0.002,
FP32 inner Krylov iterations inside FP64 refinement, rtol = 1e-8 for every solve (the paper's
Sect. 2.3 tolerance). A "step" is one whole CGP step (Eqs. 19-23) through the stage entry points.
The state is developed by --develop steps from rest on the GPU path, then W warm-up steps, then K
timed steps: before each, L2 is flushed (a 512 MB write, then a 256 MB read); each step's device
time comes from CUDA events on the launching stream (inputs resident in HBM), and the same steps'
end-to-end time from the host clock around the host->device copy of the state, the step and the
device->host copy of the new state (e2e).

Prints one JSON line: steps/s (value), coarse Poisson solves/s, the per-stage times and
iterations, the other precision's rate from the same state, the roofline of the dominant kernel
(the momentum BiCGStab), the relative L2 errors of both precisions against the CPU oracle after
one step from the developed state, the oracle timed on a host core (cpu_baseline), a secondary
workload (the backward-facing step) and the stand-alone SpMV on a matrix larger than L2.
``--impl reference`` times the CPU oracle alone.
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

WORKLOAD = "cylinder"    # the headline workload; --workload bfs33 / cavity33 time the other meshes
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


def measured_traffic(kernel: str, workload: str):
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


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_threads() -> int:
    """Threads the oracle's numerical libraries may use (its sparse LU, SuperLU, is sequential)."""
    try:
        from threadpoolctl import threadpool_info
        return max([1] + [int(i.get("num_threads", 1)) for i in threadpool_info()])
    except Exception:
        return 1


def _oracle_worker(wname: str, conn) -> None:
    """Child process (spawned): the CPU oracle on the workload. Sets up, reports, then runs one
    step from each state it receives and sends back the step time and the result."""
    from oracle import cgp as ocgp
    coarse, prob, _ = ci.workload(wname)
    t0 = time.perf_counter()
    orc = ocgp.CGPOracle(coarse.xy, coarse.tri, prob.rho, prob.mu, prob.dt, prob.levels, prob.vel_bc, prob.p_bc)
    conn.send(("ready", time.perf_counter() - t0))
    while True:
        msg = conn.recv()
        if msg[0] != "step":
            break
        u, t_next = msg[1], msg[2]
        t0 = time.perf_counter()
        r = orc.step(u, t_next)
        conn.send(("done", time.perf_counter() - t0, r.u, r.gp, oracle_threads()))
    conn.close()


class OracleJob:
    """The oracle in a spawned child process, so that its set-up and its step overlap the GPU
    work of the bench (one host core; the GPU arm uses another)."""

    def __init__(self, wname: str):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_oracle_worker, args=(wname, child), daemon=True)
        self.proc.start()
        self.t_setup = None

    def step(self, u: np.ndarray, t_next: float):
        if self.t_setup is None:
            tag, self.t_setup = self.conn.recv()
        self.conn.send(("step", u, t_next))
        tag, dt, u1, gp, threads = self.conn.recv()
        return dt, u1, gp, threads

    def close(self):
        try:
            self.conn.send(("stop",))
        except Exception:
            pass
        self.proc.join(timeout=30)


def oracle_sample(wname: str, n_steps: int, n_warmup: int = 0):
    """Time the CPU oracle in this process: setup once, ``n_warmup`` untimed steps from rest,
    then ``n_steps`` timed steps."""
    from oracle import cgp as ocgp
    coarse, prob, _ = ci.workload(wname)
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
    return times, t_setup, oracle_threads(), orc.n_fine


def workload_config(wname: str, n_coarse: int, n_fine: int, levels: int, prob) -> str:
    re_ = round((2.0 if wname.startswith("bfs") else 1.0) / prob.mu)
    return (f"{wname}: {DESCR.get(wname, wname)}, coarse {n_coarse:,} / fine {n_fine:,} nodes, l={levels}, "
            f"Re={re_}, dt={prob.dt}")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wname = args.workload
    # one oracle step of the cylinder takes minutes (sparse LU of the 1M-node momentum system,
    # per component): at most one timed step after no warm-up there; other workloads take up to
    # 3 warm-up and 10 timed steps
    big = wname == "cylinder"
    n_warm = 0 if big else min(args.warmup, 3)
    n_steps = 1 if big else max(1, min(args.steps, 10))
    times, t_setup, cores, n_fine = oracle_sample(wname, n_steps, n_warm)
    ms = 1000.0 * statistics.mean(times)
    v = 1000.0 / ms
    coarse, prob, _ = ci.workload(wname)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": n_steps, "warmup": n_warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_config(wname, coarse.n_nodes, n_fine, prob.levels, prob),
                       "rtol": "direct sparse LU (the oracle)"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "host_cores": host_cores(),
                             "kind": "oracle",
                             "sample": f"{len(times)} oracle steps after {n_warm} untimed steps from rest and a "
                                       f"{t_setup:.1f}s setup (requested: {args.steps} steps, {args.warmup} warm-up)"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def solver_spmv(L, f, flush, stream, reps: int = 10):
    """The fine solvers' FP32 product (cgp_solver_spmv: their launch shape and layout, two
    right-hand sides) on the headline's momentum matrix as assembled for its last timed step,
    L2 cleaned before each product. Algorithmic bytes: 8 nnz (FP32 values, columns) + 4 (n + 1)
    (row pointers) + 8 n (x) + 8 n (y)."""
    import torch
    info = L.cgp_mesh_info(f.ctx)
    n, nnz = info.n_fine, info.nnz_fine
    if f.params.precision != L.CGP_MIXED:
        return None
    x = torch.randn(n, 2, dtype=torch.float32, device=f.u.device)
    y = torch.empty_like(x)
    L.cgp_assemble(f.ctx, f.u, stream)
    L.cgp_solver_spmv(f.ctx, x, y, stream)
    ms = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.cgp_solver_spmv(f.ctx, x, y, stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    nbytes = 8 * nnz + 4 * (n + 1) + 16 * n
    peak, kind = peaks()
    gbs = nbytes / (t * 1e-3) / 1e9
    layout = "sliced ELL" if info.solver_format == 1 else "CSR"
    return {"kernel": f"k_solver_spmv<{'true' if info.solver_format == 1 else 'false'}> ({layout}, the fine solvers' "
                      f"FP32 product, {info.grid_blocks} blocks x {info.block_threads} threads)",
            "workload": f"the headline's momentum matrix: {n} rows, {nnz} nnz, 2 RHS, stored fine order",
            "bytes": nbytes, "ms": t, "achieved": gbs, "unit": "GB/s", "peak": peak, "frac": gbs / peak,
            "peak_kind": kind, "l2": "flushed before each product (512 MB write, then 256 MB read)"}


def spmv_hbm(L, Flow, dev, flush, stream, reps: int = 10, fine_order: int = 0):
    """The Krylov SpMV (two right-hand sides, FP64) on a matrix larger than L2: the backward-facing
    step at h = 1/48 refined twice (~2.2M rows, ~15M nnz, ~265 MB per product). Algorithmic bytes
    per product: 12 nnz (values, columns) + 4 (n + 1) (row pointers) + 16 n (x) + 16 n (y)."""
    import torch
    coarse = ci.bfs_mesh(48, 1001)
    prob = ci.bfs_problem(400.0, 0.005, 2)
    peak, kind = peaks()
    best = None
    for fmt, kname in ((2, "k_spmv_probe<2> (CSR, autotuned lanes)"), (1, "k_spmv_sell2 (sliced ELL, 32-row slices)")):
        f = Flow(coarse, prob, device=dev, spmv_format=fmt, fine_order=fine_order)
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
        order = "stored (Hilbert-curve)" if info.fine_order == 0 else "refinement"
        rec = {"kernel": kname, "workload": f"bfs48 l=2 fine A0: {n} rows, {nnz} nnz, 2 RHS, fine nodes in the "
                                             f"{order} order", "bytes": nbytes,
               "ms": t, "achieved": gbs, "unit": "GB/s", "peak": peak, "frac": gbs / peak, "peak_kind": kind,
               "lanes": info.spmv_lanes, "l2": "flushed before each product (512 MB write, then 256 MB read)"}
        if best is None or gbs > best["achieved"]:
            if best is not None:
                rec["other"] = {"kernel": best["kernel"], "achieved": best["achieved"]}
            best = rec
        else:
            best["other"] = {"kernel": rec["kernel"], "achieved": rec["achieved"]}
    return best


def momentum_alg_bytes(nnz: int, n: int, v: int, iters: float, outer: float) -> float:
    """Algorithmic bytes of one momentum solve (two right-hand sides), each operand counted once
    per use: per BiCGStab iteration two products (values and columns (v + 4) nnz, row pointers
    4 n, the input and output pairs 4 v n each) and the vector updates (90 n at v = 8, scaled by
    v / 8), which gives the ~330 bytes per row of an FP64 iteration at 7 entries per row; per FP64
    refinement pass (outer + 1 of them) the true residual b - A x: 12 nnz + 4 n + 48 n."""
    per_iter = 2.0 * ((v + 4) * nnz + 4 * n + 4 * v * n) + 90.0 * n * v / 8.0
    per_pass = 12.0 * nnz + 52.0 * n
    return iters * per_iter + (outer + 1.0) * per_pass


def timed_steps(L, f, K: int, flush, stream):
    """K steps through the stage entry points, each preceded by an L2 flush. Per step the device
    time of the step itself (CUDA events on the launching stream; inputs resident in HBM) and,
    around it on the host clock, the end-to-end time including the host->device copy of u^n and
    p^n from pinned host memory and the device->host copy of u^{n+1} and p^{n+1}."""
    import torch
    bc = torch.empty_like(f.pc)
    uh = torch.empty(f.u.shape, dtype=torch.float64, pin_memory=True)
    ph = torch.empty(f.pc.shape, dtype=torch.float64, pin_memory=True)
    uh.copy_(f.u)
    ph.copy_(f.pc)
    out = {k: [] for k in ("step", "e2e", "asm", "mom", "poi", "corr", "poi_it", "poi_out", "mom_it", "mom_out",
                           "mass_it")}
    for _ in range(K):
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f.u.copy_(uh, non_blocking=True)
        f.pc.copy_(ph, non_blocking=True)
        ev[0].record(stream)
        L.cgp_assemble(f.ctx, f.u, stream)
        ev[1].record(stream)
        L.cgp_momentum_solve(f.ctx, None, None, stream)   # u^n of the assembly; u~ stays inside
        ev[2].record(stream)
        L.cgp_restrict(f.ctx, None, bc, stream)
        if f.params.warm_start >= 1:
            L.cgp_predict_pressure(f.ctx, f.pc, stream)
        ev[3].record(stream)
        L.cgp_poisson_solve(f.ctx, bc, f.pc, stream)
        ev[4].record(stream)
        L.cgp_prolong_correct(f.ctx, f.pc, None, f.u, None, None, stream)
        ev[5].record(stream)
        uh.copy_(f.u, non_blocking=True)
        ph.copy_(f.pc, non_blocking=True)
        stream.synchronize()
        out["e2e"].append(1000.0 * (time.perf_counter() - t0))
        st = L.cgp_get_stats(f.ctx, stream, check=True)
        out["step"].append(ev[0].elapsed_time(ev[5]))
        out["asm"].append(ev[0].elapsed_time(ev[1]))
        out["mom"].append(ev[1].elapsed_time(ev[2]))
        out["poi"].append(ev[3].elapsed_time(ev[4]))
        out["corr"].append(ev[4].elapsed_time(ev[5]))
        out["poi_it"].append(st.poisson_iters)
        out["poi_out"].append(st.poisson_outer)
        out["mom_it"].append(st.momentum_iters)
        out["mom_out"].append(st.momentum_outer)
        out["mass_it"].append(st.mass_iters)
        f.t += f.problem.dt
    return {k: statistics.mean(v) for k, v in out.items()}


def one_step_with_gradient(L, f, u0, p0, stream):
    """One step from the state (u0, p0) through the stage entry points; returns u^{n+1} and
    w = M^-1 G p_f (the pressure gradient the correction applies) on the host."""
    import torch
    f.u.copy_(u0)
    f.pc.copy_(p0)
    ut = torch.empty_like(f.u)
    bc = torch.empty_like(f.pc)
    gp = torch.empty_like(f.u)
    L.cgp_assemble(f.ctx, f.u, stream)
    L.cgp_momentum_solve(f.ctx, f.u, ut, stream)
    L.cgp_restrict(f.ctx, ut, bc, stream)
    L.cgp_poisson_solve(f.ctx, bc, f.pc, stream)
    L.cgp_prolong_correct(f.ctx, f.pc, ut, f.u, None, gp, stream)
    L.cgp_get_stats(f.ctx, stream, check=True)
    return f.u.cpu().numpy(), gp.cpu().numpy()


def rel(a, b) -> float:
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_gpu(args):
    import torch

    ws, rank, local = dist_env()
    wname = args.workload
    # the oracle (CPU baseline and reference for the errors) starts first, in a spawned process,
    # so its set-up overlaps the GPU arm's work; rank 0 of a single-rank run only
    job = OracleJob(wname) if (rank == 0 and ws == 1 and not args.no_cpu_baseline) else None

    from paper_1610_06993_gb300 import cgp as L
    from paper_1610_06993_gb300.flow import Flow
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if not os.path.exists(L.LIB_PATH):
        raise RuntimeError("libcgp.so is not built; run python -c 'import __graft_entry__ as g; g.build()'")
    dev = f"cuda:{local}"
    coarse, prob, _ = ci.workload(wname)
    prec = L.CGP_MIXED if args.precision == "mixed" else L.CGP_FP64

    def make(precision, coarse_solver=None):
        return Flow(coarse, prob, precision=precision, rtol=args.rtol, device=dev,
                    block_threads=args.threads, spmv_lanes=args.lanes,
                    coarse_solver=args.coarse_solver if coarse_solver is None else coarse_solver,
                    precond_degree=args.precond_degree, precond_ratio=args.precond_ratio,
                    **({"warm_start": args.warm_start} if args.warm_start >= 0 else {}),
                    **({"inner_rtol": args.inner_rtol} if args.inner_rtol > 0 else {}),
                    **({"mass_degree": args.mass_degree} if args.mass_degree > 0 else {}),
                    **({"momentum_degree": args.momentum_degree} if args.momentum_degree > 0 else {}),
                    solver_format=args.solver_format, fine_order=args.fine_order,
                    momentum_rtol=args.momentum_rtol)

    stream = torch.cuda.current_stream()
    flush = L2Flush(dev)
    f = make(prec)
    if args.autotune:
        L.cgp_autotune(f.ctx, stream)      # lanes, fine-solver layout and threads per block
        f.info = L.cgp_mesh_info(f.ctx)
    # developed state: args.develop steps from rest on the GPU path, outside the timed region; the
    # coarse right-hand sides and pressures of its second half are logged for the coarse-solve
    # throughput comparison
    n_log = args.develop - args.develop // 2
    B_log = torch.empty(max(n_log, 1), f.info.n_coarse, dtype=torch.float64, device=dev)
    P_log = torch.empty_like(B_log)
    for k in range(args.develop):
        f.step(1, stream)
        j = k - args.develop // 2
        if j >= 0:
            L.cgp_copy_coarse_rhs(f.ctx, B_log[j], stream)
            P_log[j].copy_(f.pc)
    L.cgp_get_stats(f.ctx, stream, check=True)
    for _ in range(args.warmup):
        f.step(1, stream)
    L.cgp_get_stats(f.ctx, stream, check=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        r = timed_steps(L, f, args.steps, flush, stream)
    torch.cuda.synchronize()
    ms = job_time_ms(r["step"], ws, dev)
    e2e_ms = job_time_ms(r["e2e"], ws, dev)
    state_u, state_p, state_t = f.u.cpu().numpy().copy(), f.pc.cpu().numpy().copy(), f.t

    other = None
    if args.other_precision and ws == 1:
        # the other precision from the same developed state (its own history built by the warm-up)
        g = make(L.CGP_FP64 if prec == L.CGP_MIXED else L.CGP_MIXED)
        if args.autotune:
            L.cgp_autotune(g.ctx, stream)
        g.u.copy_(f.u)
        g.pc.copy_(f.pc)
        g.t = f.t
        # its own solver histories need some tens of steps to reach their steady behaviour (a
        # fresh history gives cheaper momentum solves for the first ~25 steps)
        for _ in range(max(args.warmup, 60)):
            g.step(1, stream)
        L.cgp_get_stats(g.ctx, stream, check=True)
        ro = timed_steps(L, g, args.steps, flush, stream)
        other = (g, ro)

    coarse_tp = None
    if args.coarse_throughput and ws == 1 and n_log >= 8:
        coarse_tp = coarse_throughput(L, Flow, make, f, other, B_log, P_log, stream, args)

    # errors against the oracle: one step of each path from the same developed state
    errors, cpu = None, None
    if job is not None:
        uo = None
        if args.oracle_steps > 0:
            dt_o, uo, gpo, threads = job.step(state_u, state_t + prob.dt)
            cpu = {"value": 1.0 / dt_o, "unit": "steps/s", "cores": threads, "host_cores": host_cores(),
                   "kind": "oracle",
                   "sample": f"1 oracle step (sparse LU solves) of the same workload from the GPU path's developed "
                             f"state (t = {state_t:.3f}); its {job.t_setup:.1f}s set-up (mesh refinement, "
                             f"matrices, LU of the mass and coarse matrices) excluded; the oracle's sparse LU is "
                             f"sequential, so it uses {threads} of the host's {host_cores()} cores"}
        job.close()
        if uo is not None:
            errors = {"after": "one step from the developed state", "rtol": args.rtol}
            paths = [(args.precision, f)] + ([] if other is None else [(("fp64" if prec == L.CGP_MIXED else "mixed"),
                                                                          other[0])])
            for name, fl in paths:
                u1, gp1 = one_step_with_gradient(L, fl, torch.from_numpy(state_u).to(dev),
                                                 torch.from_numpy(state_p).to(dev), stream)
                errors[name] = {"u_rel_l2": rel(u1, uo), "gradp_rel_l2": rel(gp1, gpo)}

    info = f.info
    nnz, n = info.nnz_fine, info.n_fine
    vbytes = 4 if prec == L.CGP_MIXED else 8
    alg_mom = momentum_alg_bytes(nnz, n, vbytes, r["mom_it"], r["mom_out"])
    mom_launch_ms = r["mom"]
    achieved = alg_mom / (mom_launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    tname = "float" if prec == L.CGP_MIXED else "double"
    mom_kernel = f"k_bicgstab<{tname}, 1, {'true' if info.solver_format == 1 else 'false'}>"
    coarse_name = {0: f"k_cg<{tname}, 1>", 1: f"k_pcg_onchip<{tname}>", 2: f"k_pcg_pipe<{tname}>",
                   3: "k_pcg_schwarz<double, float>", 4: f"k_pcg_schwarz<{tname}, {tname}>"}[info.coarse_kernel]
    # assembly 3, momentum 1, restriction 1, Poisson 1, prolongation per level, gradient 1, mass 1,
    # correction 1, two predictors of 2 launches, and the gather of u^n into the stored fine order
    launches_per_step = 9 + info.levels + (4 if f.params.warm_start >= 1 else 0) + (1 if info.fine_order == 0 else 0)
    line = {
        "metric": METRIC, "value": job_rate(1.0, ms, ws), "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == L.CGP_FP64 else "f32+f64-ir", "data": "synthetic",
        "config": {"workload": workload_config(wname, info.n_coarse, n, info.levels, prob) +
                               f", state developed by {args.develop} GPU steps from rest (t = {state_t - args.steps * prob.dt:.3f} "
                               f"at the first timed step)",
                   "rtol": args.rtol, "precision": args.precision,
                   "momentum_rtol": args.momentum_rtol if args.momentum_rtol > 0 else (
                       min(args.rtol, max(0.1 * args.rtol, 1e-14)) if args.precision == "mixed" else args.rtol),
                   "l2": "flushed before every timed step (512 MB write, then 256 MB read)",
                   "parallelism": "replicas" if ws > 1 else "1gpu",
                   "block_threads": info.block_threads, "grid_blocks": info.grid_blocks,
                   "fine_solver_format": {1: "sliced ELL", 2: "CSR"}.get(info.solver_format, "?"),
                   "fine_node_order": {0: "Hilbert curve", 1: "refinement order"}.get(info.fine_order, "?"),
                   "autotuned": bool(args.autotune), "spmv_lanes": info.spmv_lanes,
                   "coarse_kernel": coarse_name, "momentum_degree": f.params.momentum_degree,
                   "mass_degree": f.params.mass_degree,
                   "coarse_initial_guess": {0: "p^n", 1: "2 p^n - p^(n-1)", 2: "3 p^n - 3 p^(n-1) + p^(n-2)",
                                            3: "4 p^n - 6 p^(n-1) + 4 p^(n-2) - p^(n-3)"}[f.params.warm_start]},
        "coarse_solves_per_s": 1000.0 / r["poi"],
        "stage_ms": {"assembly": r["asm"], "momentum": r["mom"], "poisson": r["poi"],
                     "prolong_correct": r["corr"]},
        "iterations": {"momentum": r["mom_it"], "momentum_outer": r["mom_out"], "poisson": r["poi_it"],
                       "poisson_outer": r["poi_out"], "mass": r["mass_it"]},
        "roofline": {"kernel": mom_kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": measured_traffic(mom_kernel, wname),
                     "alg_bytes_per_launch": alg_mom, "launch_ms": mom_launch_ms,
                     "note": "momentum BiCGStab (two right-hand sides) on the fine matrix; algorithmic bytes per "
                             "BiCGStab iteration 2((v+4) nnz + 4n + 4vn) + 90n v/8 (v = bytes of the iteration "
                             "type), per FP64 refinement pass 12 nnz + 52n; achieved = those bytes x mean "
                             "iterations / the launch's CUDA-event time"},
        "coarse_solve": {"kernel": coarse_name, "bound": "latency",
                         "us_per_iter": 1000.0 * r["poi"] / max(r["poi_it"], 1.0), "grid_barriers_per_iter": 2,
                         "note": "the coarse matrix and vectors live in shared memory, registers and L2: the "
                                 "kernel is bound by grid-barrier and FP64 latency, not by HBM"},
        "e2e": {"value": job_rate(1.0, e2e_ms, ws), "unit": "steps/s",
                "h2d_bytes_per_step": (2 * n + info.n_coarse) * 8, "d2h_bytes_per_step": (2 * n + info.n_coarse) * 8,
                "note": "the same timed steps on the host clock, from the host->device copy of u^n and p^n "
                        "(pinned) to the device->host copy of u^{n+1} and p^{n+1}"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if other is not None:
        g, ro = other
        line["other_precision"] = {"precision": "fp64" if prec == L.CGP_MIXED else "mixed",
                                   "steps_per_s": 1000.0 / ro["step"], "coarse_solves_per_s": 1000.0 / ro["poi"],
                                   "stage_ms": {"assembly": ro["asm"], "momentum": ro["mom"], "poisson": ro["poi"],
                                                "prolong_correct": ro["corr"]},
                                   "iterations": {"momentum": ro["mom_it"], "poisson": ro["poi_it"],
                                                  "mass": ro["mass_it"]}}
        g.close()
    if coarse_tp is not None:
        line["coarse_solve_throughput"] = coarse_tp
    if errors is not None:
        line["errors_vs_oracle"] = errors
    if cpu is not None:
        line["cpu_baseline"] = cpu
    sv = solver_spmv(L, f, flush, stream) if not args.no_spmv else None
    f.close()
    if args.secondary and ws == 1:
        line["secondary"] = secondary_bfs33(L, Flow, dev, flush, stream, args)
    if not args.no_spmv:
        line["spmv_hbm"] = spmv_hbm(L, Flow, dev, flush, stream, fine_order=args.fine_order)
        if sv is not None:
            line["spmv_hbm"]["fine_solver_product"] = sv
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def coarse_throughput(L, Flow, make, f, other, B_log, P_log, stream, args):
    """Coarse Poisson solves/s (Eq. 21, rtol) on the workload's own logged right-hand sides, each
    solve started from the previous logged pressure (the same initial-guess policy in every arm)
    and, for the plain arm, also from zero:
      plain   - FP64 Jacobi-preconditioned CG (the paper's PCG), one solve after another;
      default - FP64 two-level Schwarz CG (this library's single-solve kernel), one after another;
      batched - this run's precision, all right-hand sides together (cgp_poisson_solve_many,
                one block per right-hand side, two-level preconditioner)."""
    import torch
    nrhs = B_log.shape[0] - 1
    Bs, X0 = B_log[1:].contiguous(), P_log[:-1].contiguous()

    def sequential(ctx, rows, zero):
        X = torch.zeros_like(Bs[:rows]) if zero else X0[:rows].clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = 0
        for k in range(rows):
            L.cgp_poisson_solve(ctx, Bs[k], X[k], stream)
            its += L.cgp_get_stats(ctx, stream, check=True).poisson_iters
        e1.record(stream)
        e1.synchronize()
        return rows * 1000.0 / e0.elapsed_time(e1), its / rows

    jac = make(L.CGP_FP64, coarse_solver=5)
    rows_plain = min(nrhs, 8)
    plain, plain_it = sequential(jac.ctx, rows_plain, False)
    plain0, plain0_it = sequential(jac.ctx, rows_plain, True)
    jac.close()
    fp64 = other[0] if (other is not None and other[0].params.precision == L.CGP_FP64) else f
    dflt, dflt_it = sequential(fp64.ctx, min(nrhs, 64), False)
    X = X0.clone()
    its = torch.zeros(nrhs, dtype=torch.int32, device=Bs.device)
    st = torch.zeros(nrhs, dtype=torch.int32, device=Bs.device)
    L.cgp_poisson_solve_many(f.ctx, Bs[:2], X[:2], None, None, None, stream)   # set-up outside the timing
    X = X0.clone()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.cgp_poisson_solve_many(f.ctx, Bs, X, its, None, st, stream)
    e1.record(stream)
    e1.synchronize()
    if int(st.max().item()) != L.CGP_OK:
        raise RuntimeError(f"batched coarse solve status {int(st.max().item())}")
    batched = nrhs * 1000.0 / e0.elapsed_time(e1)
    return {"right_hand_sides": nrhs, "initial_guess": "previous logged pressure (all arms), plain also from zero",
            "plain_fp64_jacobi_sequential": plain, "plain_iters": plain_it,
            "plain_fp64_jacobi_zero_start": plain0, "plain_zero_iters": plain0_it,
            "default_fp64_schwarz_sequential": dflt, "default_iters": dflt_it,
            "batched_" + args.precision: batched, "batched_iters": float(its.double().mean().item()),
            "ratio_batched_vs_plain_same_guess": batched / plain,
            "ratio_batched_vs_plain_zero_start": batched / plain0,
            "ratio_batched_vs_default_fp64": batched / dflt}


def secondary_bfs33(L, Flow, dev, flush, stream, args):
    """The backward-facing-step channel (65,308 / 259,117 nodes, l = 1) in FP64 and in
    FP32+IR side by side, each after 100 developing steps: steps/s, coarse solves/s, and the relative
    L2 error of one more step of each from the FP64 state against one oracle step."""
    import torch
    coarse, prob, _ = ci.workload("bfs33")
    out = {"workload": "bfs33 (65,308 / 259,117 nodes, l=1, Re=400, dt=0.005), state after 100 steps"}
    flows = {}
    for name, prec in (("fp64", L.CGP_FP64), ("mixed", L.CGP_MIXED)):
        f = Flow(coarse, prob, precision=prec, rtol=args.rtol, device=dev)
        for _ in range(100):
            f.step(1, stream)
        L.cgp_get_stats(f.ctx, stream, check=True)
        r = timed_steps(L, f, max(10, args.steps // 2), flush, stream)
        out[name] = {"steps_per_s": 1000.0 / r["step"], "coarse_solves_per_s": 1000.0 / r["poi"],
                     "e2e_steps_per_s": 1000.0 / r["e2e"],
                     "iterations": {"momentum": r["mom_it"], "poisson": r["poi_it"], "mass": r["mass_it"]}}
        flows[name] = f
    if not args.no_cpu_baseline:
        from oracle import cgp as ocgp
        f64 = flows["fp64"]
        u0, p0, t0 = f64.u.cpu().numpy().copy(), f64.pc.clone(), f64.t
        orc = ocgp.CGPOracle(coarse.xy, coarse.tri, prob.rho, prob.mu, prob.dt, prob.levels, prob.vel_bc, prob.p_bc)
        ref = orc.step(u0, t0 + prob.dt)
        errs = {"after": "one step from the FP64 path's state", "rtol": args.rtol}
        for name, f in flows.items():
            u1, gp1 = one_step_with_gradient(L, f, torch.from_numpy(u0).to(dev), p0, stream)
            errs[name] = {"u_rel_l2": rel(u1, ref.u), "gradp_rel_l2": rel(gp1, ref.gp)}
        out["errors_vs_oracle"] = errs
    for f in flows.values():
        f.close()
    return out


def batch_launches_per_step(flows) -> int:
    """Kernels of one batched step of one-level instances with the injection restriction (the
    batch64 workload): the gather of u^n into the stored fine order (when the instances renumber),
    the colour-scheduled assembly, the two predictor launches, the momentum solve, the batched
    restriction, the batched two-level coarse CG, the prolongation per level and the gradient, the
    mass solve and the correction: one launch each for all instances."""
    lv = max(f.info.levels for f in flows)
    renumber = any(f.info.fine_order == 0 for f in flows)
    predict = any(f.params.warm_start >= 1 for f in flows)
    return (1 if renumber else 0) + 1 + (2 if predict else 0) + 1 + 1 + 1 + lv + 1 + 1 + 1


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
    flows = [Flow(m, p, precision=prec, rtol=args.rtol, device=dev, fine_order=args.fine_order,
                  momentum_rtol=args.momentum_rtol) for m, p in cases]
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

    # per-instance error against the oracle: one more batched step from the current states of a
    # sample of instances spread over the sizes, against one oracle step from the same states
    errs = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import cgp as ocgp
        sizes = np.array([f.info.n_coarse for f in flows])
        order = np.argsort(sizes, kind="stable")
        sample = [int(order[k]) for k in np.linspace(0, n_inst - 1, 4).round().astype(int)]
        states = {i: (flows[i].u.cpu().numpy().copy(), flows[i].t) for i in sample}
        b.step(1, stream)
        b.stats(check=True)
        errs = {"after": "one batched step from the timed run's final states", "rtol": args.rtol}
        for i in sample:
            m, p = cases[i]
            orc = ocgp.CGPOracle(m.xy, m.tri, p.rho, p.mu, p.dt, p.levels, p.vel_bc, p.p_bc)
            ref = orc.step(states[i][0], states[i][1] + p.dt)
            errs[f"instance {i} ({int(sizes[i])} coarse nodes)"] = rel(flows[i].u.cpu().numpy(), ref.u)

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
        "gpu_launches": batch_launches_per_step(flows) * args.steps, "clocks": clk.summary(),
    }
    if errs is not None:
        line["errors_vs_oracle"] = errs
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
    of the residual-form network (it corrects a base guess from that guess's residual) by the
    tensor-core kernels, then 256 held-out right-hand sides solved together to rtol by the
    multi-right-hand-side CG from zero, previous-step, cubic-extrapolation and network-corrected
    starts (network inference time included in the network starts' solves/s)."""
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
    f = Flow(mesh, problems[0], rtol=args.rtol)
    base = {"previous": Pp, "cubic": warmstart.history_base(P, run, 3)}
    idx = torch.nonzero(test).flatten()
    idx = idx[torch.randperm(idx.numel(), generator=torch.Generator().manual_seed(5)).to(idx.device)[:256]]
    Bt, Pt = B[idx].contiguous(), P[idx].contiguous()
    starts = {"zero": torch.zeros_like(Bt), "previous": base["previous"][idx].contiguous(),
              "cubic": base["cubic"][idx].contiguous()}
    train_s, losses, extra = {}, {}, {}
    for name in ("previous", "cubic"):
        w = L.cgp_ws_create(n, 512, 256)
        L.cgp_ws_set_params(w, ci.mlp_init_params(n, 512, 4))
        L.cgp_ws_set_mask(w, held)
        t0 = time.perf_counter()
        hist = warmstart.train_residual(w, f.ctx, B[~test].contiguous(), P[~test].contiguous(),
                                        base[name][~test].contiguous(), epochs=args.epochs, batch=256, lr=1e-3)
        torch.cuda.synchronize()
        train_s[name], losses[name] = time.perf_counter() - t0, [hist[0], hist[-1]]
        nets, ms = warmstart.network_starts(w, f.ctx, Bt, {name: starts[name]})
        starts.update(nets)
        extra.update(ms)
        L.cgp_ws_destroy(w)
    out = warmstart.evaluate(f, starts, Bt, Pt, extra)
    f.close()
    best = min(out, key=lambda k: out[k]["iters_mean"])
    line = {"metric": "coarse Poisson solves/s at rtol with zero / previous-step / cubic / learned warm starts",
            "value": out[best]["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16 network, f64 CG", "data": "synthetic",
            "config": {"workload": f"cavity129 (16,641 coarse nodes), {args.runs} runs x {args.run_steps} steps, "
                                   f"Re U[100,1000], residual-form network 16641-512-512-16641 GELU, batch 256, "
                                   f"{args.epochs} epochs; 256 held-out right-hand sides solved together",
                       "rtol": args.rtol, "best_start": best},
            "pairs": int(B.shape[0]), "gen_s": t_gen, "train_s": train_s, "loss_first_last": losses,
            "results": out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["bfs33", "cylinder", "cavity33", "batch64", "warmstart", "spmv"])
    ap.add_argument("--runs", type=int, default=100)
    ap.add_argument("--run-steps", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--develop", type=int, default=300)        # GPU steps from rest before the warm-up
    ap.add_argument("--oracle-steps", type=int, default=1)     # oracle steps from the developed state
    ap.add_argument("--no-other-precision", dest="other_precision", action="store_false")
    ap.add_argument("--no-secondary", dest="secondary", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--no-coarse-throughput", dest="coarse_throughput", action="store_false")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--coarse-solver", type=int, default=0)
    ap.add_argument("--precond-degree", type=int, default=0)
    ap.add_argument("--precond-ratio", type=float, default=0.0)
    ap.add_argument("--warm-start", type=int, default=-1)
    ap.add_argument("--inner-rtol", type=float, default=0.0)   # 0: the library default (1e-4)
    ap.add_argument("--mass-degree", type=int, default=0)      # 0: the library default (4)   # -1: the library default (1, extrapolation)
    ap.add_argument("--momentum-degree", type=int, default=0)  # 0: the library default
    ap.add_argument("--solver-format", type=int, default=0)    # 0: automatic, 1: sliced ELL, 2: CSR
    ap.add_argument("--fine-order", type=int, default=0)       # 0: Hilbert-curve storage, 1: refinement order
    ap.add_argument("--momentum-rtol", type=float, default=0.0)   # 0: rtol
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
        print(json.dumps(spmv_hbm(L, Flow, "cuda:0", flush, torch.cuda.current_stream(), reps=args.steps,
                                  fine_order=args.fine_order)), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
