"""CNN warm start for ADM-TV (the learned part of the workload; the paper has
no counterpart).

Pairs are produced by the method itself: for seeded random phantoms, the
image after a few ADM iterations (x0) and after many (x*).  The network
(``Cnn``) learns x0 -> x*; at run time ADM then continues from the network's
output.  Everything on the GPU path runs in libdect's kernels (ADM, the
network's forward/backward and Adam); this module only sequences calls.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

from . import AdmParams, Cnn, Plan, adm_tv

SCALE = 0.02  # 1/mm: typical attenuation, the network's input scale


@dataclasses.dataclass
class Pairs:
    x0: "object"      # torch [S*2, H, W] float32 CUDA: short-ADM images (both energies)
    xstar: "object"   # torch [S*2, H, W]: long-ADM images


def make_pairs(plan: Plan, sinograms, params: AdmParams, k0: int = 20, kstar: int = 300,
               chunk: int = 16) -> Pairs:
    """ADM with k0 and with kstar iterations (fixed counts) from zero for every
    slice of sinograms [S, 2, nv, nb] (CUDA float32).  Returns both energies as
    separate images."""
    import torch
    g = plan.geom
    S = sinograms.shape[0]
    x0 = torch.empty((S, 2, g.n, g.n), device=sinograms.device)
    xs = torch.empty_like(x0)
    p0 = dataclasses.replace(params, max_iter=k0, rel_obj_tol=0.0, warm_start=False)
    ps = dataclasses.replace(params, max_iter=kstar, rel_obj_tol=0.0, warm_start=False)
    for c in range(0, S, chunk):
        m = sinograms[c:c + chunk].contiguous()
        a, _ = adm_tv(plan, m, p0)
        b, _ = adm_tv(plan, m, ps)
        x0[c:c + chunk] = a
        xs[c:c + chunk] = b
    return Pairs(x0.reshape(S * 2, g.n, g.n).contiguous(), xs.reshape(S * 2, g.n, g.n).contiguous())


def tile_pairs(pairs: Pairs, tile: int) -> Pairs:
    """Cut every image of `pairs` into non-overlapping tile x tile blocks (the
    image sides a multiple of `tile`): training samples of a size the
    network's workspace holds, from images too large to train on whole."""
    def cut(x):
        n, H, W = x.shape
        if H % tile or W % tile:
            raise ValueError("image sides must be multiples of the tile")
        t = x.reshape(n, H // tile, tile, W // tile, tile).permute(0, 1, 3, 2, 4)
        return t.reshape(-1, tile, tile).contiguous()
    return Pairs(cut(pairs.x0), cut(pairs.xstar))


def apply_tiled(net: Cnn, x, scale: float = SCALE, tile: int = 256, halo: int = 32):
    """The network's output for x [B, H, W], computed tile by tile: each
    tile x tile block from a crop with `halo` pixels of context on each
    side, clipped to the image.  The network's receptive field (two 3x3
    convolutions at each of three levels, about 23 pixels) lies within the
    halo and the crops start at multiples of 4 (the two 2 x 2 poolings), so
    every output pixel equals that of the whole image; the network's
    workspace then bounds the crop, not the image (crops of one shape are
    batched up to that size)."""
    import torch
    B, H, W = x.shape
    if tile % 4 or halo % 4 or H % 4 or W % 4:
        raise ValueError("tile, halo and image sides must be multiples of 4")
    out = torch.empty_like(x)
    jobs = {}
    for b in range(B):
        for ty in range(0, H, tile):
            for tx in range(0, W, tile):
                y0, y1 = max(ty - halo, 0), min(ty + tile + halo, H)
                x0, x1 = max(tx - halo, 0), min(tx + tile + halo, W)
                jobs.setdefault((y1 - y0, x1 - x0), []).append((b, y0, x0, ty, tx))
    for (h, w), lst in jobs.items():
        per = max(1, net.max_pixels // (h * w))
        for i in range(0, len(lst), per):
            part = lst[i:i + per]
            crops = torch.stack([x[b, y0:y0 + h, x0:x0 + w] for b, y0, x0, _, _ in part]).contiguous()
            y = net.forward(crops, scale)
            for k, (b, y0, x0, ty, tx) in enumerate(part):
                th, tw = min(tile, H - ty), min(tile, W - tx)
                out[b, ty:ty + th, tx:tx + tw] = y[k, ty - y0:ty - y0 + th, tx - x0:tx - x0 + tw]
    return out


def train(net: Cnn, pairs: Pairs, epochs: int = 4, batch: int = 16, lr: float = 3e-4,
          seed: int = 0, log=None) -> List[float]:
    """Adam on the mean-squared error between net(x0) and x*; returns the mean
    loss of each epoch.  The network starts as the identity (zero head), whose
    error is already small; lr = 3e-4 descends smoothly from there (the
    epoch loss falls about 17-fold over 8 epochs on 4096 pairs at 256^2)."""
    import torch
    n = pairs.x0.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = torch.tensor(rng.permutation(n), device=pairs.x0.device)
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = order[i:i + batch]
            x = pairs.x0.index_select(0, idx).contiguous()
            t = pairs.xstar.index_select(0, idx).contiguous()
            tot += net.loss_grad(x, t, SCALE)
            net.adam_step(lr)
            cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log("epoch %d loss %.4g" % (ep, losses[-1]))
    return losses


def warm_started_adm(net: Cnn, plan: Plan, sinograms, params: AdmParams, k0: int = 20, tile: int = 0):
    """ADM with the CNN warm start: k0 plain iterations, the network, then ADM
    (with params' stopping rule) from the network's output.  tile > 0: the
    network runs tile-wise (apply_tiled).  Returns (x [S, 2, n, n], reports
    of the final ADM, k0)."""
    import torch
    g = plan.geom
    S = sinograms.shape[0]
    p0 = dataclasses.replace(params, max_iter=k0, rel_obj_tol=0.0, warm_start=False)
    x0, _ = adm_tv(plan, sinograms, p0)
    x0 = x0.reshape(S * 2, g.n, g.n).contiguous()
    xh = apply_tiled(net, x0, SCALE, tile) if tile > 0 else net.forward(x0, SCALE)
    pw = dataclasses.replace(params, warm_start=True)
    x, reps = adm_tv(plan, sinograms, pw, x=xh.reshape(S, 2, g.n, g.n).contiguous())
    return x, reps, k0
