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


def train(net: Cnn, pairs: Pairs, epochs: int = 4, batch: int = 16, lr: float = 3e-4,
          seed: int = 0, log=None) -> List[float]:
    """Adam on the mean-squared error between net(x0) and x*; returns the mean
    loss of each epoch.  The network starts as the identity (zero head), whose
    error is already small; at lr = 1e-3 the first steps push the loss well
    above it and the run's outcome then depends on the last bits of the
    arithmetic (the two convolution paths ended at 951 and 816 warm-started
    ADM iterations), while at 3e-4 and 1e-4 both paths descend smoothly to
    the same loss (800-820 iterations against 996 from zero at 512^2)."""
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


def warm_started_adm(net: Cnn, plan: Plan, sinograms, params: AdmParams, k0: int = 20):
    """ADM with the CNN warm start: k0 plain iterations, the network, then ADM
    (with params' stopping rule) from the network's output.  Returns
    (x [S, 2, n, n], reports of the final ADM, k0)."""
    import torch
    g = plan.geom
    S = sinograms.shape[0]
    p0 = dataclasses.replace(params, max_iter=k0, rel_obj_tol=0.0, warm_start=False)
    x0, _ = adm_tv(plan, sinograms, p0)
    xh = net.forward(x0.reshape(S * 2, g.n, g.n).contiguous(), SCALE)
    pw = dataclasses.replace(params, warm_start=True)
    x, reps = adm_tv(plan, sinograms, pw, x=xh.reshape(S, 2, g.n, g.n).contiguous())
    return x, reps, k0
