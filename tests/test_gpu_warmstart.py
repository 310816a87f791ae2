"""The learned warm start, end to end on a small case: pairs logged by the batched solver, training
by the tcgen05 kernels, and the gain over a zero initial guess on held-out runs (the coarse CG
still converges to the same tolerance from every start)."""
import os

import numpy as np
import pytest
import torch

import cgp_inputs as ci

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


def test_network_warm_start_beats_zero_start(L):
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
    ws = L.cgp_ws_create(n, 128, 256)
    L.cgp_ws_set_params(ws, ci.mlp_init_params(n, 128, 21))
    L.cgp_ws_set_mask(ws, held)
    hist = warmstart.train(ws, B[~te].contiguous(), P[~te].contiguous(), epochs=60, batch=40, lr=2e-3)
    assert hist[-1] < 0.2 * hist[0]
    f = Flow(mesh, problems[0], rtol=1e-8)
    out = warmstart.evaluate(f, ws, B[te].contiguous(), P[te].contiguous(), Pp[te].contiguous())
    f.close()
    L.cgp_ws_destroy(ws)
    for name, r in out.items():
        assert r["max_rel_res"] <= 1e-8 and r["rel_err_vs_logged"] < 1e-6, (name, r)
    assert out["network"]["iters_mean"] < out["zero"]["iters_mean"], out
