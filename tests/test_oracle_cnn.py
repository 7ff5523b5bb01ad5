"""Pins of the oracle's CNN warm-start network (forward and hand-derived backward).

References: an independent float64 PyTorch-CPU restatement of the same
network with autograd, central finite differences of the loss, and the
identity of the network with a zero head."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
F = torch.nn.functional

S = 0.02


def torch_net(p, x, s):
    """Same network written with torch ops (float64, CPU)."""
    i = 0
    W = []
    for cin, cout in synth.CNN_LAYERS:
        w = p[i:i + cout * cin * 9].view(cout, cin, 3, 3)
        i += cout * cin * 9
        b = p[i:i + cout]
        i += cout
        W.append((w, b))
    wh, bh = p[i:i + 32], p[i + 32]
    conv = lambda t, k: F.relu(F.conv2d(t, W[k][0], W[k][1], padding=1))
    t = x[None, None] / s
    e1 = conv(conv(t, 0), 1)
    e2 = conv(conv(F.avg_pool2d(e1, 2), 2), 3)
    bt = conv(conv(F.avg_pool2d(e2, 2), 4), 5)
    d2 = conv(conv(torch.cat([F.interpolate(bt, scale_factor=2, mode="nearest"), e2], 1), 6), 7)
    d1 = conv(conv(torch.cat([F.interpolate(d2, scale_factor=2, mode="nearest"), e1], 1), 8), 9)
    h = torch.einsum("c,nchw->nhw", wh, d1)[0] + bh
    return x + s * h


def _params(seed):
    p = synth.cnn_init(seed)
    p[-33:] = np.random.default_rng(seed + 1).standard_normal(33) * 0.1
    return p


def test_forward_and_gradient_match_torch_autograd():
    rng = np.random.default_rng(0)
    p = _params(1)
    x = 0.02 * rng.random((12, 16))
    tgt = x * 1.05 + 0.001 * rng.standard_normal(x.shape)
    out = oracle.cnn_forward(p, x, S)
    loss, g = oracle.cnn_loss_grad(p, x, tgt, S)
    pt = torch.tensor(p, requires_grad=True)
    ot = torch_net(pt, torch.tensor(x), S)
    np.testing.assert_allclose(out, ot.detach().numpy(), rtol=1e-12, atol=1e-15)
    lt = ((ot - torch.tensor(tgt)) ** 2).mean()
    lt.backward()
    assert abs(loss - float(lt)) <= 1e-12 * abs(loss)
    np.testing.assert_allclose(g, pt.grad.numpy(), rtol=1e-9, atol=1e-16)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = _params(3)
    x = 0.02 * rng.random((8, 8))
    tgt = x * 1.1
    _, g = oracle.cnn_loss_grad(p, x, tgt, S)
    picks = rng.choice(p.size, 12, replace=False).tolist() + [p.size - 1, p.size - 20]
    h = 1e-6
    for i in picks:
        pp = p.copy()
        pp[i] += h
        lp, _ = oracle.cnn_loss_grad(pp, x, tgt, S)
        pp[i] -= 2 * h
        lm, _ = oracle.cnn_loss_grad(pp, x, tgt, S)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-9) + 1e-13


def test_untrained_net_is_the_identity_and_head_bias_shifts():
    x = 0.02 * np.random.default_rng(4).random((8, 12))
    p = synth.cnn_init(5)
    np.testing.assert_array_equal(oracle.cnn_forward(p, x, S), x)
    p[-1] = 0.5
    np.testing.assert_allclose(oracle.cnn_forward(p, x, S), x + S * 0.5, rtol=0, atol=1e-15)
    assert oracle.cnn_num_params() == 470977 == synth.cnn_num_params() == synth.cnn_init(0).size
