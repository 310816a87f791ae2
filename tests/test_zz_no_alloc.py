"""The allocation-free CG entry point against the oracle's exact coarse pressure solve.

cgp_cg_solve_noalloc serves callers that must not allocate device memory: they bring their own
CSR matrix and vectors, and the solver's scratch comes from a fixed static device array. Here it
gets the coarse pressure matrix of the 33x33-node cavity (the stiffness of Eq. 21 with the pinned
node eliminated symmetrically) and two right-hand sides in a row, and each solution is compared
with the oracle's direct solve of the same system. Later calls run on the scratch contents left
by the earlier ones: a call that stops at max_iter, a call with a NaN right-hand side, a matrix
with a zero diagonal entry, each reporting its status through the device output, and then a good
solve again. This file is collected last so a failure here never hides the other tests.
"""
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


@pytest.fixture(scope="module")
def system():
    coarse, prob, _ = ci.workload("cavity33")
    res5, orc = ocgp.run(coarse, prob, 5, return_oracle=True)
    res6 = orc.step(res5.u, 6 * prob.dt)
    K = ocgp._bc_sym(orc.coarse.K, orc.p_mask).tocsr()
    K.sort_indices()
    return K, (res5, res6)


def dev(a, dt):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def solve(L, rp, ci_, val, b, max_iter=20000, rtol=1e-13):
    x = torch.zeros_like(b)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    iters = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    relres = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    L.cgp_cg_solve_noalloc(rp, ci_, val, b, x, rtol, max_iter, status, iters, relres)
    torch.cuda.synchronize()
    return x, int(status.item()), int(iters.item()), float(relres.item())


def test_noalloc_cg_matches_oracle(L, system):
    K, results = system
    rp, ci_, val = dev(K.indptr, torch.int32), dev(K.indices, torch.int32), dev(K.data, torch.float64)
    for res in results:
        x, status, iters, relres = solve(L, rp, ci_, val, dev(res.b_c, torch.float64))
        assert status == L.CGP_OK and relres <= 1e-13 and iters > 0, (status, relres, iters)
        err = np.linalg.norm(x.cpu().numpy() - res.p_c) / np.linalg.norm(res.p_c)
        assert err < 1e-11, err


def test_noalloc_failure_statuses_then_recovers(L, system):
    K, results = system
    rp, ci_, val = dev(K.indptr, torch.int32), dev(K.indices, torch.int32), dev(K.data, torch.float64)
    b = dev(results[0].b_c, torch.float64)
    # max_iter = 1 at a tight tolerance: the solve stops, writes x and its residual
    x, status, iters, relres = solve(L, rp, ci_, val, b, max_iter=1)
    assert status == L.CGP_ERR_NOT_CONVERGED and iters == 1 and 1e-13 < relres < 1.0, (status, iters, relres)
    assert torch.isfinite(x).all()
    # a NaN in the right-hand side
    bn = b.clone()
    bn[17] = float("nan")
    _, status, _, _ = solve(L, rp, ci_, val, bn, max_iter=100)
    assert status == L.CGP_ERR_NAN, status
    # a row whose stored diagonal is zero: not an SPD matrix
    bad = K.data.copy()
    row = 40
    bad[K.indptr[row] + np.nonzero(K.indices[K.indptr[row]:K.indptr[row + 1]] == row)[0][0]] = 0.0
    _, status, _, _ = solve(L, rp, ci_, dev(bad, torch.float64), b, max_iter=50)
    assert status == L.CGP_ERR_ARG, status
    # the scratch left by the failed calls does not affect the next solve
    x, status, iters, relres = solve(L, rp, ci_, val, b)
    assert status == L.CGP_OK and relres <= 1e-13, (status, relres)
    err = np.linalg.norm(x.cpu().numpy() - results[0].p_c) / np.linalg.norm(results[0].p_c)
    assert err < 1e-11, err


def test_noalloc_rejects_oversize(L):
    n = 65537
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(L.CGPError) as e:
        L.cgp_cg_solve_noalloc(rp, rp, z, z, z, 1e-8, 10)
    assert e.value.code == L.CGP_ERR_ARG
