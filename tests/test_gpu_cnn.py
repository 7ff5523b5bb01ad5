"""GPU parity of the CNN warm start (BF16 tensor-core kernels, FP32
accumulation) against the FP64 oracle, through the C ABI.

Tolerances follow from BF16: unit roundoff u = 2^-8; every layer rounds its
weights and its output activations, about sqrt(2) u / sqrt(3) ~ 2.3e-3
relative per layer, and the ten 3x3 layers compound to ~sqrt(10) x that,
~1.5e-2 on the network's residual.  Bounds: 3e-2 relative L2 on the residual
x_out - x, 8e-2 on the gradient (the backward pass rounds the incoming
gradients too) and 1.2e-1 per layer block."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402

S = 0.02


def _params(seed):
    p = synth.cnn_init(seed)
    rng = np.random.default_rng(seed + 1)
    p[-33:] = rng.standard_normal(33) * 0.3
    # non-zero biases so every path of the network is exercised
    o = 0
    for cin, cout in synth.CNN_LAYERS:
        o += cout * cin * 9
        p[o:o + cout] = 0.05 * rng.standard_normal(cout)
        o += cout
    return p


@pytest.fixture(scope="module")
def net():
    return dect.Cnn(max_pixels=4 * 64 * 64)


@pytest.mark.parametrize("B,H,W", [(1, 16, 16), (2, 32, 24), (3, 64, 64)])
def test_forward_matches_oracle(net, B, H, W):
    rng = np.random.default_rng(B * H)
    p = _params(7)
    x = (0.02 * rng.random((B, H, W))).astype(np.float32)
    net.set_params(p.astype(np.float32))
    out = net.forward(torch.tensor(x, device="cuda"), S).cpu().numpy()
    for b in range(B):
        ref = oracle.cnn_forward(p.astype(np.float32).astype(np.float64), x[b].astype(np.float64), S)
        res_gpu, res_ref = out[b] - x[b], ref - x[b]
        assert np.linalg.norm(res_gpu - res_ref) <= 3e-2 * np.linalg.norm(res_ref)


def test_forward_matches_oracle_beyond_one_grid_pass():
    """B H W above the elementwise kernels' capped grid (152 x 16 blocks of
    256 threads cover 19456 pixels of 32 input channels): every pixel of the
    second image lies beyond one pass of the grid."""
    B, H, W = 2, 128, 96
    rng = np.random.default_rng(5)
    p = _params(9)
    x = (0.02 * rng.random((B, H, W))).astype(np.float32)
    big = dect.Cnn(max_pixels=B * H * W)
    big.set_params(p.astype(np.float32))
    out = big.forward(torch.tensor(x, device="cuda"), S).cpu().numpy()
    big.close()
    for b in range(B):
        ref = oracle.cnn_forward(p.astype(np.float32).astype(np.float64), x[b].astype(np.float64), S)
        res_gpu, res_ref = out[b] - x[b], ref - x[b]
        assert np.linalg.norm(res_gpu - res_ref) <= 3e-2 * np.linalg.norm(res_ref), b
        # the last rows as well (a stale input there would leave the norm test
        # to the first rows)
        assert np.linalg.norm(res_gpu[-16:] - res_ref[-16:]) <= 3e-2 * np.linalg.norm(res_ref[-16:]), b


def test_gradient_matches_oracle(net):
    rng = np.random.default_rng(3)
    p = _params(11).astype(np.float32)
    B, H, W = 2, 32, 32
    x = (0.02 * rng.random((B, H, W))).astype(np.float32)
    t = (x * 1.05 + 0.001 * rng.standard_normal(x.shape)).astype(np.float32)
    net.set_params(p)
    loss, g = net.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), S, want_grad=True)
    # the batch loss is the mean over all pixels: average the per-image oracle gradients
    gref = np.zeros(p.size)
    lref = 0.0
    for b in range(B):
        l, gb = oracle.cnn_loss_grad(p.astype(np.float64), x[b].astype(np.float64), t[b].astype(np.float64), S)
        gref += gb / B
        lref += l / B
    assert abs(loss - lref) <= 3e-2 * lref
    assert np.linalg.norm(g - gref) <= 8e-2 * np.linalg.norm(gref)
    # per layer as well (each layer's gradient block)
    o = 0
    for cin, cout in synth.CNN_LAYERS:
        n = cout * cin * 9
        blk = slice(o, o + n)
        assert np.linalg.norm(g[blk] - gref[blk]) <= 1.2e-1 * np.linalg.norm(gref[blk]) + 1e-12
        o += n + cout


def test_training_reduces_the_loss(net):
    rng = np.random.default_rng(5)
    B, H, W = 4, 32, 32
    x = (0.02 * rng.random((B, H, W))).astype(np.float32)
    t = x * 1.1
    net.set_params(synth.cnn_init(13).astype(np.float32))
    xt, tt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    l0 = net.loss_grad(xt, tt, S)
    for _ in range(30):
        net.loss_grad(xt, tt, S)
        net.adam_step(1e-3)
    l1 = net.loss_grad(xt, tt, S)
    assert l1 < 0.5 * l0
