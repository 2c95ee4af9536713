"""The library's atom-pair MLP kernels (BF16 weights, FP32 accumulation)
against the FP64 reference in oracle/mlp_ref.py: forward values, loss and
every gradient component; an Adam run lowers the loss."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2407_21445_gb300 as fk
    from oracle import mlp_ref
    return torch, fk, mlp_ref


def test_mlp_forward_and_gradients_match_reference(env):
    torch, fk, ref = env
    rng = np.random.default_rng(5)
    nin, H, nout, B = 37, 64, 45, 300
    net = fk.MLP(nin, H, nout, 512, seed=3)
    p = net.params()
    X = rng.normal(0, 1, (B, nin)).astype(np.float32)
    T = rng.normal(0, 1, (B, nout)).astype(np.float32)
    M = (rng.uniform(0, 1, (B, nout)) > 0.25).astype(np.float32)
    Xt, Tt, Mt = (torch.tensor(a, device="cuda") for a in (X, T, M))
    Y = net.forward(Xt).cpu().numpy()
    Yr, _ = ref.forward(p.astype(np.float64), X.astype(np.float64), nin, H, nout, weights_bf16=True)
    assert np.abs(Y - Yr).max() <= 1e-4 * max(1.0, np.abs(Yr).max())
    net.zero_grad()
    loss = net.loss_backward(Xt, Tt, Mt, norm=float(M.sum()))
    g = net.grads()
    lr_, gr = ref.loss_and_grad(p.astype(np.float64), X.astype(np.float64), T, M, float(M.sum()), nin, H, nout,
                                weights_bf16=True)
    assert abs(loss - lr_) <= 1e-4 * lr_
    err = np.abs(g - gr).max() / np.abs(gr).max()
    assert err < 1e-3, err


def test_mlp_training_lowers_loss(env):
    torch, fk, ref = env
    rng = np.random.default_rng(7)
    nin, H, nout, B = 8, 32, 4, 1024
    X = rng.normal(0, 1, (B, nin)).astype(np.float32)
    W = rng.normal(0, 1, (nin, nout))
    T = np.tanh(X @ W).astype(np.float32)
    net = fk.MLP(nin, H, nout, B, seed=1)
    Xt, Tt = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    l0 = net.loss_backward(Xt, Tt)
    net.zero_grad()
    for _ in range(300):
        net.loss_backward(Xt, Tt)
        net.step(lr=3e-3)
    l1 = net.loss_backward(Xt, Tt)
    assert l1 < 0.1 * l0, (l0, l1)
