"""Learned warm start for the coarse Poisson solve: data logging, training and evaluation.

The solver generates its own training data: several runs of one coarse mesh at different
Reynolds numbers are advanced together by the batched step, and every step's coarse right-hand
side b_c and pressure p_c (and the previous step's pressure) are logged on the device. The network
works in residual form: it corrects a base guess (the previous step's pressure or its
extrapolation in time) from that guess's residual b - K x_base, trained by
``cgp_ws_train_step_residual`` (tcgen05 kernels). Its gain is measured by the iteration count of the
coarse CG, which always runs to the same tolerance whatever its initial guess; the held-out
right-hand sides are solved together by ``cgp_poisson_solve_many``. All arithmetic runs in the
CUDA library; this module only orchestrates calls and keeps torch device tensors.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import cgp as L
from .flow import Batch, Flow


def generate(mesh, problems, steps: int, device: str = "cuda:0", rtol: float = 1e-8, precision: int = L.CGP_FP64):
    """Advance one Flow per problem together for ``steps`` steps and log, per run and step,
    (b_c, p_c, p_c of the previous step). Returns ``(B, P, Pprev, run_id)`` device tensors."""
    flows = [Flow(mesh, p, precision=precision, rtol=rtol, device=device) for p in problems]
    batch = Batch(flows)
    n = flows[0].info.n_coarse
    rows = len(flows) * steps
    B = torch.empty(rows, n, dtype=torch.float64, device=device)
    P = torch.empty_like(B)
    Pprev = torch.empty_like(B)
    run_id = torch.arange(len(flows), device=device).repeat_interleave(steps)
    for k in range(steps):
        for i, f in enumerate(flows):
            Pprev[i * steps + k].copy_(f.pc)
        batch.step(1)
        for i, f in enumerate(flows):
            L.cgp_copy_coarse_rhs(f.ctx, B[i * steps + k])
            P[i * steps + k].copy_(f.pc)
    batch.stats(check=True)
    held = flows[0].p_mask.copy()
    batch.close()
    for f in flows:
        f.close()
    return B, P, Pprev, run_id, held


def train(ws: int, B, P, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0, log=None):
    """Adam on shuffled minibatches (cosine-decayed step size). Returns the per-epoch mean loss."""
    n_rows = B.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=B.device)
    hist = []
    total = epochs * (n_rows // batch)
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n_rows, generator=g).to(B.device)
        acc = []
        for s in range(0, n_rows - batch + 1, batch):
            idx = perm[s:s + batch]
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(total, 1)))
            L.cgp_ws_train_step(ws, B[idx].contiguous(), P[idx].contiguous(), lr_t, loss)
            acc.append(loss.clone())
            step += 1
        hist.append(float(torch.stack(acc).mean().item()))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    if L.cgp_ws_status(ws) != L.CGP_OK:
        raise RuntimeError("tensor-core pipeline timeout during training")
    return hist


def train_residual(ws: int, ctx: int, B, P, Base, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0,
                   log=None):
    """Adam on shuffled minibatches of the residual form: input r = b - K x_base, target p - x_base
    (cgp_ws_train_step_residual; ``ctx`` supplies the coarse matrix). Returns the per-epoch mean loss."""
    n_rows = B.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=B.device)
    hist = []
    total = epochs * (n_rows // batch)
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n_rows, generator=g).to(B.device)
        acc = []
        for s in range(0, n_rows - batch + 1, batch):
            idx = perm[s:s + batch]
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(total, 1)))
            L.cgp_ws_train_step_residual(ws, ctx, B[idx].contiguous(), P[idx].contiguous(), Base[idx].contiguous(),
                                         lr_t, loss)
            acc.append(loss.clone())
            step += 1
        hist.append(float(torch.stack(acc).mean().item()))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    if L.cgp_ws_status(ws) != L.CGP_OK:
        raise RuntimeError("tensor-core pipeline timeout during training")
    return hist


def history_base(P, run_id, order: int):
    """Per logged row, the extrapolation in time of the run's earlier pressures (order 0: the
    previous step's pressure; 1..3: linear / quadratic / cubic, lower while the run is young; zero
    on a run's first step), computed by cgp_extrapolate. Rows of a run are consecutive steps."""
    rows = P.shape[0]
    out = torch.zeros_like(P)
    rid = run_id.cpu().numpy()
    k_of = np.zeros(rows, dtype=np.int64)
    for r in range(1, rows):
        k_of[r] = k_of[r - 1] + 1 if rid[r] == rid[r - 1] else 0
    for r in range(rows):
        k = int(k_of[r])
        if k == 0:
            continue
        o = min(order, k - 1)
        L.cgp_extrapolate(o, [P[r - 1 - j] for j in range(o + 1)], out[r])
    return out


def evaluate(flow: Flow, starts: dict, B, P, extra_ms: dict | None = None):
    """Coarse CG (the context's rtol) for every row of B from each initial guess in ``starts``
    (name -> [rows][n] tensor), all rows of a start solved together by cgp_poisson_solve_many
    (one block per right-hand side). Returns per start the mean iterations, solves/s (plus
    ``extra_ms[name]``, e.g. the network's inference, in the time), the maximum relative residual
    and the relative error against the logged pressures."""
    out = {}
    rows = B.shape[0]
    iters = torch.zeros(rows, dtype=torch.int32, device=B.device)
    rel = torch.zeros(rows, dtype=torch.float64, device=B.device)
    status = torch.zeros(rows, dtype=torch.int32, device=B.device)
    for name, X0 in starts.items():
        X = X0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.cgp_poisson_solve_many(flow.ctx, B, X, iters, rel, status)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) + (extra_ms or {}).get(name, 0.0)
        if int(status.max().item()) != L.CGP_OK:
            raise RuntimeError(f"coarse solve from the {name} start: status {int(status.max().item())}")
        err = float((torch.linalg.norm(X - P) / torch.linalg.norm(P)).item())
        out[name] = {"iters_mean": float(iters.double().mean().item()), "solves_per_s": rows * 1000.0 / ms,
                     "max_rel_res": float(rel.max().item()), "rel_err_vs_logged": err, "time_ms": ms}
    return out


def network_starts(ws: int, ctx: int, B, bases: dict):
    """The network's corrections of the given bases (name -> [rows][n]) in batches of the network's
    capacity, timed; returns ({"network+" + name: X0}, {"network+" + name: ms})."""
    starts, times = {}, {}
    for name, base in bases.items():
        X0 = torch.empty_like(B)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for s in range(0, B.shape[0], 256):
            L.cgp_ws_forward_residual(ws, ctx, B[s:s + 256], base[s:s + 256], X0[s:s + 256])
        e1.record()
        e1.synchronize()
        starts["network+" + name] = X0
        times["network+" + name] = e0.elapsed_time(e1)
    return starts, times
