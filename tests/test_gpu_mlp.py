"""GPU parity of the warm-start network: the tcgen05 BF16 GEMM and the network's forward pass,
back-propagated gradients and Adam update against the FP64 oracle (oracle/mlp.py) on the same
BF16-rounded inputs and weights.

Tolerances. The GEMM multiplies BF16 values exactly and adds each K = 16 tensor-core step into an
FP32 accumulator; that addition may truncate rather than round, so the error can grow linearly in
the number of steps: bound 1e-5 + 2^-24 K/16 relative L2 (7e-5 at K = 16,768; observed 1.9e-5,
and < 1e-5 for K <= 640). The network stores h1, h2 and dz in BF16
on both sides; the FP32 (GPU) and FP64 (oracle) pre-activations differ by ~1e-6 relative, which
flips the BF16 rounding of a few elements by one unit (2^-8 relative): 2e-3 relative L2 for the
outputs and gradients covers that with margin."""
import os

import numpy as np
import pytest
import torch

import cgp_inputs as ci
from oracle import mlp

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / max(np.linalg.norm(b), 1e-300))


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


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 640), (128, 512, 16768), (16768, 128, 256)])
def test_gemm_bf16_tcgen05(L, M, N, K):
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    Cd = torch.empty(M, N, dtype=torch.float32, device="cuda")
    L.cgp_gemm_bf16(A.cuda(), B.cuda(), Cd)
    torch.cuda.synchronize()
    ref = A.double().numpy() @ B.double().numpy().T
    assert rel(Cd.cpu().numpy(), ref) < 1e-5 + 2.0 ** -24 * K / 16


def test_gemm_rejects_unaligned_shapes(L):
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(100, 128, dtype=torch.float32, device="cuda")
    with pytest.raises(L.CGPError):
        L.cgp_gemm_bf16(A, torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda"), C)


def _problem(n=200, H=128, B=64, seed=5):
    params = ci.mlp_init_params(n, H, seed)
    rng = np.random.default_rng(seed)
    params[1] = (0.05 * rng.standard_normal(H)).astype(np.float32)
    params[3] = (0.05 * rng.standard_normal(H)).astype(np.float32)
    params[5] = (0.05 * rng.standard_normal(n)).astype(np.float32)
    b = rng.standard_normal((B, n))
    p = rng.standard_normal((B, n))
    held = np.zeros(n, dtype=np.uint8)
    held[0] = 1
    return params, b, p, held


def test_network_forward_grads_adam(L):
    n, H, B = 200, 128, 64
    params, b, p, held = _problem(n, H, B)
    w = L.cgp_ws_create(n, H, 128)
    L.cgp_ws_set_params(w, params)
    L.cgp_ws_set_mask(w, held)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    pd = torch.tensor(p, dtype=torch.float64, device="cuda")
    out = torch.empty_like(bd)
    L.cgp_ws_forward(w, bd, out)
    assert L.cgp_ws_status(w) == 0
    P64 = [q.astype(np.float64) for q in params]
    mask = (1 - held).astype(np.float64)
    ref, _ = mlp.forward(P64, b, mask, bf16=True)
    assert rel(out.cpu().numpy(), ref) < 2e-3
    # gradients only (lr = 0), then one Adam step
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    L.cgp_ws_train_step(w, bd, pd, 0.0, loss)
    Lref, gref = mlp.loss_and_grads(P64, b, p, mask, bf16=True)
    assert abs(loss.item() - Lref) < 2e-3 * abs(Lref)
    g = L.cgp_ws_get_grads(w, n, H)
    for k, (a, r) in enumerate(zip(g, gref)):
        assert rel(a, r) < 2e-3, (k, rel(a, r))
    L.cgp_ws_train_step(w, bd, pd, 1e-3)
    g1 = L.cgp_ws_get_grads(w, n, H)
    new = L.cgp_ws_get_params(w, n, H)
    zeros = [np.zeros_like(q) for q in P64]
    want, _, _ = mlp.adam_step(P64, [x.astype(np.float64) for x in g1], zeros, [z.copy() for z in zeros], 1, 1e-3)
    for k, (a, r) in enumerate(zip(new, want)):
        assert np.abs(a - r).max() < 1e-6 + 1e-6 * np.abs(r).max(), k
    assert L.cgp_ws_status(w) == 0
    L.cgp_ws_destroy(w)


def test_training_reduces_loss(L):
    """A few hundred Adam steps on a fixed linear target map drive the loss down."""
    n, H, B = 256, 128, 128
    rng = np.random.default_rng(9)
    Amat = rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal((B, n))
    p = b @ Amat.T
    w = L.cgp_ws_create(n, H, B)
    L.cgp_ws_set_params(w, ci.mlp_init_params(n, H, 11))
    L.cgp_ws_set_mask(w, np.zeros(n, np.uint8))
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    pd = torch.tensor(p, dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    L.cgp_ws_train_step(w, bd, pd, 0.0, loss)
    l0 = loss.item()
    for _ in range(300):
        L.cgp_ws_train_step(w, bd, pd, 2e-3, loss)
    l1 = loss.item()
    assert L.cgp_ws_status(w) == 0
    L.cgp_ws_destroy(w)
    assert l1 < 0.2 * l0, (l0, l1)
