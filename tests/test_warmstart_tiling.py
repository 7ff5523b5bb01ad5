"""Host logic of the tile-wise warm start (warmstart.apply_tiled and
tile_pairs), on the CPU: the network is the FP64 oracle's forward pass
behind the same call the library's network offers.

The network is local: its receptive field reaches 23 pixels (two 3x3
convolutions at each of three levels, two 2x2 poolings, nearest
up-sampling), and translating the input by a multiple of 4 translates the
output.  Tiles computed from crops with a halo of at least 23 pixels that
start at multiples of 4 must therefore equal the whole image's output
exactly; a halo smaller than the receptive field must not."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

from paper_1607_01650_gb300 import warmstart as ws  # noqa: E402


def _params():
    rng = np.random.default_rng(4)
    p = synth.cnn_init(2)
    p[-33:] = rng.standard_normal(33) * 0.3
    o = 0
    for cin, cout in synth.CNN_LAYERS:
        o += cout * cin * 9
        p[o:o + cout] = 0.05 * rng.standard_normal(cout)
        o += cout
    return p


class OracleNet:
    """forward(x [B, H, W], scale) of the oracle's network, one image at a
    time; max_pixels bounds a call as the library's workspace does."""

    def __init__(self, params, max_pixels):
        self.params = params
        self.max_pixels = max_pixels
        self.calls = []

    def forward(self, x, scale):
        assert x.shape[0] * x.shape[1] * x.shape[2] <= self.max_pixels
        self.calls.append(tuple(x.shape))
        return torch.stack([torch.from_numpy(oracle.cnn_forward(self.params, xi.numpy(), scale)) for xi in x])


@pytest.fixture(scope="module")
def case():
    g = synth.tiny_geometry(n=32)
    u = synth.rasterize(synth.random_ellipse_phantom(g, seed=5, axis_range=(3.0, 10.0)), 32, 1.0, supersample=2)
    rng = np.random.default_rng(6)
    img = np.kron(u[0] + 2.0 * u[1], np.ones((2, 2)))[:64, :56]
    x = torch.from_numpy(0.02 * img + 1e-3 * rng.standard_normal(img.shape))[None]
    net = OracleNet(_params(), max_pixels=64 * 56)
    return net, x, net.forward(x, ws.SCALE)


def test_tiles_with_a_halo_beyond_the_receptive_field_equal_the_whole_image(case):
    net, x, whole = case
    # 24 x 24 tiles leave ragged tiles on both sides (64 = 2 x 24 + 16, 56 = 2 x 24 + 8)
    tiled = ws.apply_tiled(net, x, ws.SCALE, tile=24, halo=24)
    assert torch.equal(tiled, whole)


def test_a_halo_inside_the_receptive_field_changes_the_output(case):
    net, x, whole = case
    tiled = ws.apply_tiled(net, x, ws.SCALE, tile=24, halo=8)
    d = (tiled - whole).abs()
    assert float(d.max()) > 1e-6
    # pixels 24 or more from every inner edge of their crop still agree: the
    # first tile's crop is [0, 32)^2, so its top-left 8 x 8
    assert float(d[0, :8, :8].max()) == 0.0


def test_crops_batch_by_shape_within_the_workspace(case):
    net, x, _ = case
    small = OracleNet(net.params, max_pixels=2 * 48 * 48)
    ws.apply_tiled(small, x, ws.SCALE, tile=24, halo=24)
    assert all(b * h * w <= small.max_pixels for b, h, w in small.calls)
    assert sum(b for b, _, _ in small.calls) == 9  # 3 x 3 tiles, each once


def test_arguments_must_keep_the_pooling_period():
    net = OracleNet(_params(), max_pixels=1 << 20)
    x = torch.zeros((1, 16, 16), dtype=torch.float64)
    for tile, halo in ((6, 4), (8, 6)):
        with pytest.raises(ValueError):
            ws.apply_tiled(net, x, ws.SCALE, tile=tile, halo=halo)


def test_tile_pairs_cuts_every_image_into_its_blocks():
    rng = np.random.default_rng(0)
    a = torch.from_numpy(rng.standard_normal((3, 8, 12)))
    b = a + 1.0
    p = ws.tile_pairs(ws.Pairs(a, b), 4)
    assert p.x0.shape == (3 * 2 * 3, 4, 4) and p.xstar.shape == p.x0.shape
    # block (i, j) of image n is sample n * 6 + i * 3 + j
    for n in range(3):
        for i in range(2):
            for j in range(3):
                assert torch.equal(p.x0[n * 6 + i * 3 + j], a[n, 4 * i:4 * i + 4, 4 * j:4 * j + 4])
                assert torch.equal(p.xstar[n * 6 + i * 3 + j], b[n, 4 * i:4 * i + 4, 4 * j:4 * j + 4])
    with pytest.raises(ValueError):
        ws.tile_pairs(ws.Pairs(a, b), 5)
