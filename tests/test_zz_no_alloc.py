"""The allocation-free CG entry point agrees with the library's coarse Poisson solve.

cgp_cg_solve_noalloc serves callers that must not allocate device memory: they bring their own
CSR matrix and vectors, and the solver's scratch comes from a fixed static device array. Here it
gets the coarse pressure matrix of the 33x33-node cavity (the stiffness of Eq. 21 with the pinned
node eliminated symmetrically) and two right-hand sides in a row, and each solution is compared
with cgp_poisson_solve on the same right-hand side. The second call runs on the scratch contents
left by the first. This file is collected last so a failure here never hides the other tests.
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


def test_noalloc_cg_matches_poisson_solve(L):
    from paper_1610_06993_gb300.flow import Flow

    coarse, prob, _ = ci.workload("cavity33")
    res5, orc = ocgp.run(coarse, prob, 5, return_oracle=True)
    res6 = orc.step(res5.u, 6 * prob.dt)
    K = ocgp._bc_sym(orc.coarse.K, orc.p_mask).tocsr()
    K.sort_indices()
    dev = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    rp, ci_, val = dev(K.indptr, torch.int32), dev(K.indices, torch.int32), dev(K.data, torch.float64)
    f = Flow(coarse, prob, rtol=1e-13)
    for b_host in (res5.b_c, res6.b_c):
        b = dev(b_host, torch.float64)
        x_ref = torch.zeros_like(b)
        L.cgp_poisson_solve(f.ctx, b, x_ref)
        assert f.stats(check=True).poisson_rel_res <= 1e-13
        x = torch.zeros_like(b)
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        iters = torch.zeros(1, dtype=torch.int32, device="cuda")
        relres = torch.zeros(1, dtype=torch.float64, device="cuda")
        L.cgp_cg_solve_noalloc(rp, ci_, val, b, x, 1e-13, 20000, status, iters, relres)
        torch.cuda.synchronize()
        assert int(status.item()) == L.CGP_OK and float(relres.item()) <= 1e-13 and int(iters.item()) > 0
        err = (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item()
        assert err < 1e-11, err
    f.close()


def test_noalloc_rejects_oversize(L):
    n = 65537
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(L.CGPError) as e:
        L.cgp_cg_solve_noalloc(rp, rp, z, z, z, 1e-8, 10)
    assert e.value.code == L.CGP_ERR_ARG
