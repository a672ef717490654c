"""Pins of the oracle's MLP, loss, gradients and Adam: against torch's float64 autograd and
optimizer (library routines) and central finite differences on the full loss.  CPU only."""
import numpy as np
import pytest
import torch

import synth
from oracle import adam, encode, mlp, schedule, train


def _torch_mlp(params, dims):
    layers = []
    for (W, b) in mlp.unpack(params, dims):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W))
            lin.bias.copy_(torch.from_numpy(b))
        layers += [lin, torch.nn.ReLU()]
    return torch.nn.Sequential(*layers[:-1])


@pytest.mark.parametrize("dims", [[8, 32, 32, 1], [32, 64, 64, 1], [64, 64, 64, 64, 1]])
def test_mlp_forward_backward_vs_torch(dims):
    rng = np.random.default_rng(0)
    p = synth.init_mlp(3, dims).astype(np.float64)
    x = rng.standard_normal((257, dims[0]))
    tgt = rng.standard_normal(257)
    y, a, z = mlp.forward(p, dims, x)
    L, gy = mlp.mse(y, tgt)
    g, gx = mlp.backward(p, dims, a, z, gy)

    net = _torch_mlp(p, dims)
    xt = torch.from_numpy(x).requires_grad_(True)
    yt = net(xt)[:, 0]
    Lt = torch.nn.functional.mse_loss(yt, torch.from_numpy(tgt))
    Lt.backward()
    gt = np.concatenate([np.concatenate([m.weight.grad.numpy().ravel(), m.bias.grad.numpy()])
                         for m in net if isinstance(m, torch.nn.Linear)])
    assert np.allclose(y, yt.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert abs(L - Lt.item()) <= 1e-13 * abs(L)
    assert np.allclose(g, gt, rtol=1e-11, atol=1e-14)
    assert np.allclose(gx, xt.grad.numpy(), rtol=1e-11, atol=1e-14)


def test_adam_vs_torch():
    rng = np.random.default_rng(1)
    n = 1000
    p = rng.standard_normal(n)
    m = np.zeros(n)
    v = np.zeros(n)
    pt = torch.from_numpy(p.copy()).requires_grad_(True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.99), eps=1e-8)
    for k in range(1, 8):
        g = rng.standard_normal(n)
        g[rng.random(n) < 0.3] = 0.0  # untouched rows still move
        p, m, v = adam.step(p, g, m, v, k, 1e-2, 0.9, 0.99, 1e-8)
        pt.grad = torch.from_numpy(g.copy())
        opt.step()
        assert np.allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)


def _small_model(seed=0):
    levels = [[3, 3, 3, 2], [5, 5, 4, 3], [9, 7, 6, 4]]
    dims = [6, 16, 16, 1]
    F = 2
    b, rows = schedule.bases(levels)
    table = synth.init_tables(seed, rows * F, r=0.5).astype(np.float64).reshape(rows, F)
    p = synth.init_mlp(seed, dims).astype(np.float64)
    co = synth.coords(seed, 96)
    tgt = synth.uniform(seed, 7, 96, -1, 1).astype(np.float64)
    return levels, b, F, dims, table, p, co, tgt


def test_gradients_vs_central_differences():
    # The loss is piecewise quadratic in each single parameter (ReLU MLP, encoding linear in the
    # table), so the central difference with h = 1e-3 equals the derivative unless a ReLU flips
    # within +-h; such points are detected with h/10 and skipped.
    levels, b, F, dims, table, p, co, tgt = _small_model()
    L, _, g_mlp, (rows, g_rows) = train.loss_and_grads(levels, b, F, dims, table, p, co, tgt)
    g_tab = np.zeros_like(table)
    g_tab[rows] = g_rows
    rng = np.random.default_rng(9)
    picks = [("t", int(r), int(f)) for r, f in zip(rng.choice(rows, 40), rng.integers(0, F, 40))]
    picks += [("m", int(i), 0) for i in rng.choice(p.size, 24, replace=False)]

    def loss_at(kind, i, f, delta):
        t2, p2 = table.copy(), p.copy()
        if kind == "t":
            t2[i, f] += delta
        else:
            p2[i] += delta
        return train.loss_and_grads(levels, b, F, dims, t2, p2, co, tgt)[0]

    checked = 0
    for kind, i, f in picks:
        an = g_tab[i, f] if kind == "t" else g_mlp[i]
        fd = [(loss_at(kind, i, f, h) - loss_at(kind, i, f, -h)) / (2 * h) for h in (1e-3, 1e-4)]
        if abs(fd[0] - fd[1]) > 1e-6 * max(abs(fd[0]), 1e-12) + 1e-15:
            continue  # kink within h
        assert abs(fd[0] - an) <= 1e-6 * max(abs(an), 1e-9) + 1e-13, (kind, i, f, fd[0], an)
        checked += 1
    assert checked >= 48


def test_train_step_decreases_loss():
    levels, b, F, dims, table, p, co, tgt = _small_model(1)
    model = train.Model(levels, F, dims, table, p)
    losses = [train.train_step(model, co, tgt) for _ in range(30)]
    assert losses[-1] < 0.5 * losses[0]
