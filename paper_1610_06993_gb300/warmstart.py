"""Learned warm start for the coarse Poisson solve: data logging, training and evaluation.

The solver generates its own training data: several runs of one coarse mesh at different
Reynolds numbers are advanced together by the batched step, and every step's coarse right-hand
side b_c and pressure p_c (and the previous step's pressure) are logged on the device. The network
is trained by ``cgp_ws_train_step`` (tcgen05 kernels) and judged by the iteration count of the
coarse CG, which always runs to the same tolerance whatever its initial guess. All arithmetic runs
in the CUDA library; this module only orchestrates calls and keeps torch device tensors.
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


def evaluate(flow: Flow, ws: int | None, B, P, Pprev):
    """Coarse CG from three initial guesses on the rows of B: zero, the previous step's pressure,
    and the network's prediction (if ``ws``). Returns per-start mean iterations, solves/s (the
    network's inference time included) and the maximum relative residual reached."""
    out = {}
    starts = {"zero": torch.zeros_like(B), "previous": Pprev.clone()}
    t_inf = 0.0
    if ws is not None:
        x0 = torch.empty_like(B)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.cgp_ws_forward(ws, B, x0)
        e1.record()
        e1.synchronize()
        t_inf = e0.elapsed_time(e1)
        starts["network"] = x0
    for name, X in starts.items():
        its, rr = [], 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ms = 0.0
        for r in range(B.shape[0]):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            L.cgp_poisson_solve(flow.ctx, B[r], X[r])
            e1.record()
            st = flow.stats(check=True)
            ms += e0.elapsed_time(e1)
            its.append(st.poisson_iters)
            rr = max(rr, st.poisson_rel_res)
        if name == "network":
            ms += t_inf
        err = float((torch.linalg.norm(X - P) / torch.linalg.norm(P)).item())
        out[name] = {"iters_mean": float(np.mean(its)), "solves_per_s": B.shape[0] * 1000.0 / ms,
                     "max_rel_res": rr, "rel_err_vs_logged": err, "time_ms": ms,
                     "wall_s": time.perf_counter() - t0}
    if ws is not None:
        out["network"]["inference_ms_per_batch"] = t_inf
    return out
