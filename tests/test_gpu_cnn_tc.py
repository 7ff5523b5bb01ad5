"""The two convolution kernels of the CNN warm start: the tensor-memory
implicit GEMM (tcgen05, the default) and the warp-level mma.sync one.

Both form the same BF16 products and accumulate them in FP32, in different
orders, so their FP32 sums differ by a few units of FP32 roundoff and a
layer's BF16 output differs in the last bit where the sum lies near a
rounding boundary: about 2^-9 relative for those elements, far below the
BF16 error against the FP64 oracle (tests/test_gpu_cnn.py).  Bounds: 1e-2
relative L2 on the network's residual and on the gradient.  The
oracle parity of the default path is checked again here at sizes with
several tiles and ragged edges in both directions at every level."""
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
    o = 0
    for cin, cout in synth.CNN_LAYERS:
        o += cout * cin * 9
        p[o:o + cout] = 0.05 * rng.standard_normal(cout)
        o += cout
    return p.astype(np.float32)


@pytest.fixture(scope="module")
def net():
    n = dect.Cnn(max_pixels=16 * 128 * 128)
    yield n
    n.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_default_path_is_tcgen05(net):
    assert net.conv_path == dect.Cnn.CONV_TCGEN05
    with pytest.raises(dect.DectError):
        net.conv_path = 7


@pytest.mark.parametrize("B,H,W", [(1, 8, 8), (2, 40, 56), (3, 72, 36), (16, 128, 128)])
def test_forward_paths_agree(net, B, H, W):
    rng = np.random.default_rng(H * W + B)
    net.set_params(_params(3))
    x = torch.tensor((0.02 * rng.random((B, H, W))).astype(np.float32), device="cuda")
    outs = {}
    for path in (dect.Cnn.CONV_MMA_SYNC, dect.Cnn.CONV_TCGEN05):
        net.conv_path = path
        outs[path] = net.forward(x, S).cpu().numpy()
    xs = x.cpu().numpy()
    r_tc, r_ms = outs[dect.Cnn.CONV_TCGEN05] - xs, outs[dect.Cnn.CONV_MMA_SYNC] - xs
    assert np.all(np.isfinite(r_tc))
    # both paths round every layer's activations to BF16 (unit roundoff
    # 2^-9 = 2e-3) after FP32 sums taken in different orders, so an element
    # can land one BF16 step apart in each of the ten layers; measured 6.6e-3
    # at 16 x 128^2 (each path is also held to the FP64 oracle)
    assert _rel(r_tc, r_ms) <= 1e-2


def test_gradient_paths_agree(net):
    rng = np.random.default_rng(9)
    B, H, W = 4, 48, 80
    p = _params(5)
    x = torch.tensor((0.02 * rng.random((B, H, W))).astype(np.float32), device="cuda")
    t = x * 1.05
    res = {}
    for path in (dect.Cnn.CONV_MMA_SYNC, dect.Cnn.CONV_TCGEN05):
        net.conv_path = path
        net.set_params(p)
        res[path] = net.loss_grad(x, t, S, want_grad=True)
    (l_tc, g_tc), (l_ms, g_ms) = res[dect.Cnn.CONV_TCGEN05], res[dect.Cnn.CONV_MMA_SYNC]
    assert abs(l_tc - l_ms) <= 4e-3 * l_ms
    assert _rel(g_tc, g_ms) <= 1e-2
    net.conv_path = dect.Cnn.CONV_TCGEN05


@pytest.mark.parametrize("B,H,W", [(2, 40, 56)])
def test_tcgen05_forward_matches_oracle(net, B, H, W):
    rng = np.random.default_rng(21)
    p = _params(7)
    x = (0.02 * rng.random((B, H, W))).astype(np.float32)
    net.conv_path = dect.Cnn.CONV_TCGEN05
    net.set_params(p)
    out = net.forward(torch.tensor(x, device="cuda"), S).cpu().numpy()
    for b in range(B):
        ref = oracle.cnn_forward(p.astype(np.float64), x[b].astype(np.float64), S)
        assert np.linalg.norm((out[b] - x[b]) - (ref - x[b])) <= 3e-2 * np.linalg.norm(ref - x[b])
    net.check()
