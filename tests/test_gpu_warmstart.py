"""The learned warm start, end to end on a small case: pairs logged by the batched solver, the
network trained in residual form (it corrects the previous step's pressure from that guess's
residual b - K p^{n-1}) by the tcgen05 kernels, and its gain on held-out runs. Every start is
solved by the batched multi-right-hand-side CG to the same tolerance, which decides each error."""
import os

import numpy as np
import pytest
import torch

import cgp_inputs as ci
from oracle import cgp as ocgp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_06993_gb300 import cgp
    if not os.path.exists(cgp.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    cgp.load()
    return cgp


def test_solve_many_matches_oracle(L):
    """cgp_poisson_solve_many: every right-hand side reaches the oracle's direct solve of Eq. 21
    (rtol 1e-12: the two-level preconditioner's coarse part runs in FP32, so the attainable FP64
    residual of these rough right-hand sides sits near 1e-13; energy-norm error <= sqrt(kappa)
    rtol with kappa ~ 1e3 on the 33x33-node cavity)."""
    from paper_1610_06993_gb300.flow import Flow
    coarse, prob, _ = ci.workload("cavity33")
    res, orc = ocgp.run(coarse, prob, 3, return_oracle=True)
    rng = np.random.default_rng(4)
    b = orc.coarse.M @ rng.standard_normal((orc.n_coarse, 7))
    b[orc.p_mask, :] = 0.0
    b = np.ascontiguousarray(b.T)
    b[0] = res.b_c
    ref = np.stack([orc.poisson(r) for r in b])
    f = Flow(coarse, prob, rtol=1e-12)
    B = torch.tensor(b, device="cuda")
    X = torch.zeros_like(B)
    its = torch.zeros(B.shape[0], dtype=torch.int32, device="cuda")
    rel = torch.zeros(B.shape[0], dtype=torch.float64, device="cuda")
    st = torch.full((B.shape[0],), -1, dtype=torch.int32, device="cuda")
    L.cgp_poisson_solve_many(f.ctx, B, X, its, rel, st)
    torch.cuda.synchronize()
    f.close()
    assert (st == 0).all() and float(rel.max()) <= 1e-12 and int(its.min()) > 0, (st, rel)
    e = np.linalg.norm(X.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert e.max() < 1e-10, e


def test_residual_network_beats_previous_step_start(L):
    from paper_1610_06993_gb300 import warmstart
    from paper_1610_06993_gb300.flow import Flow
    mesh = ci.cavity_mesh(33, 1000)
    res = np.linspace(100.0, 1000.0, 10)
    problems = [ci.cavity_problem(float(r), 0.005, 1) for r in res]
    steps = 30
    B, P, Pp, run, held = warmstart.generate(mesh, problems, steps)
    test_runs = {2, 7}
    te = torch.tensor([int(r) in test_runs for r in run.cpu().numpy()], device=B.device)
    n = B.shape[1]
    f = Flow(mesh, problems[0], rtol=1e-8)
    ws = L.cgp_ws_create(n, 128, 256)
    L.cgp_ws_set_params(ws, ci.mlp_init_params(n, 128, 21))
    L.cgp_ws_set_mask(ws, held)
    hist = warmstart.train_residual(ws, f.ctx, B[~te].contiguous(), P[~te].contiguous(), Pp[~te].contiguous(),
                                    epochs=60, batch=40, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    Bt, Pt = B[te].contiguous(), P[te].contiguous()
    bases = {"previous": Pp[te].contiguous(), "cubic": warmstart.history_base(P, run, 3)[te].contiguous()}
    nets, net_ms = warmstart.network_starts(ws, f.ctx, Bt, {"previous": bases["previous"]})
    starts = {"zero": torch.zeros_like(Bt), **bases, **nets}
    out = warmstart.evaluate(f, starts, Bt, Pt, net_ms)
    f.close()
    L.cgp_ws_destroy(ws)
    for name, r in out.items():
        assert r["max_rel_res"] <= 1e-8 and r["rel_err_vs_logged"] < 1e-6, (name, r)
    assert out["network+previous"]["iters_mean"] < out["previous"]["iters_mean"], out
    assert out["previous"]["iters_mean"] < out["zero"]["iters_mean"], out
