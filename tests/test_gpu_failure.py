"""Failure detection of the bounded device waits, without faulting the GPU.

Every grid barrier of the persistent kernels gives up after a bounded wait and records
CGP_ERR_TIMEOUT instead of spinning forever. cgp_wait_probe runs that barrier on a context's own
persistent launch shape with a target of more arrivals than blocks (a wait that nothing can
satisfy): the wait must run out within its limit, the status must come back to the host, and the
context must stay usable (a following run still matches the oracle).
"""
import os
import time

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


def test_barrier_wait_runs_out_and_context_stays_usable(L):
    from paper_1610_06993_gb300.flow import Flow
    coarse, prob = ci.bfs_mesh(4, 1001), ci.bfs_problem(400.0, 0.005, 1)
    f = Flow(coarse, prob, rtol=1e-13)
    assert f.info.grid_blocks > 1
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    # a barrier every block can pass
    L.cgp_wait_probe(f.ctx, 0, 50.0, status)
    torch.cuda.synchronize()
    assert int(status.item()) == L.CGP_OK
    # one block short: nothing can complete the barrier; the wait must end by itself
    for limit_ms in (20.0, 250.0):
        status.fill_(-1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.cgp_wait_probe(f.ctx, 1, limit_ms, status)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert int(status.item()) == L.CGP_ERR_TIMEOUT
        assert limit_ms * 1e-3 <= dt < limit_ms * 1e-3 + 2.0, (limit_ms, dt)
    # the context is still usable: its own statistics are untouched and a run matches the oracle
    f.step(5)
    st = f.stats(check=True)
    assert st.barrier_status == L.CGP_OK
    ref = ocgp.run(coarse, prob, 5)
    e = float(np.linalg.norm(f.u.cpu().numpy() - ref.u) / np.linalg.norm(ref.u))
    f.close()
    assert e < 1e-10, e


def test_wait_probe_rejects_bad_arguments(L):
    from paper_1610_06993_gb300.flow import Flow
    coarse, prob, _ = ci.workload("cavity33")
    f = Flow(coarse, prob)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for missing, limit in ((-1, 10.0), (2000, 10.0), (1, 0.0), (1, 20000.0)):
        with pytest.raises(L.CGPError) as e:
            L.cgp_wait_probe(f.ctx, missing, limit, status)
        assert e.value.code == L.CGP_ERR_ARG
    f.close()
