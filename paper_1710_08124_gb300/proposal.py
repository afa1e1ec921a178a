"""Training data and training loop of the learned top-m proposal.

The labels are produced by the method itself: each observation is restored
for t = 0 .. T-1 iterations of Algorithm 1 (exhaustive selection), and the
exact Gaussian selection (Eq. 14) of every patch of the estimate x_t is taken
at that iteration's beta_t = lambda * beta_mult[t] / sigma^2.  Every step runs
in libepll (``restore``, ``patch_step``, ``Proposal.train_step``); this module
only arranges the calls and the sample order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import (PAPER_BETA, SUBSET_ALL, BF16X3, SELECT_EXHAUSTIVE, GMM, Options, Proposal, patch_step,
               restore)


def denoise_lambda(sigma: float) -> float:
    """lambda of the beta schedule for denoising (A = I): min{1, 250 sigma_255^2}
    (Sec. "Parameter settings"; the library computes the same on the device)."""
    return min(1.0, 250.0 * (255.0 * sigma) ** 2)


@dataclass
class Pairs:
    """Labelled patches: images [n_img, H, W] (the estimates x_t) and, per
    sample, its image, anchor, log(1/beta) and exact selection."""
    images: "torch.Tensor"
    img_idx: "torch.Tensor"
    anchors: "torch.Tensor"
    log_ib: "torch.Tensor"
    labels: "torch.Tensor"

    def __len__(self):
        return int(self.labels.numel())


def make_pairs(g: GMM, observations, sigmas, beta_mult=PAPER_BETA, options: Options | None = None) -> Pairs:
    """(patch, exact selection) pairs from denoising trajectories.

    observations: list of float32 CUDA tensors [H, W] (one size), noisy images;
    sigmas: their noise levels.  For every observation y and iteration t the
    estimate x_t (x_0 = y; x_t = ``restore`` with the first t multipliers) and
    all its H*W patches are labelled by the exhaustive selection at beta_t.
    """
    import torch
    o = options or Options(precision=BF16X3)
    o = Options(**{**o.__dict__, "select": SELECT_EXHAUSTIVE, "subset": SUBSET_ALL})
    H, W = observations[0].shape
    ims, idx, anc, lib_, lab = [], [], [], [], []
    for y, sigma in zip(observations, sigmas):
        if tuple(y.shape) != (H, W):
            raise ValueError("observations must share one size")
        lam = denoise_lambda(float(sigma))
        for t in range(len(beta_mult)):
            x = y if t == 0 else restore(g, y, float(sigma), beta_mult[:t], options=o)
            beta = lam * beta_mult[t] / float(sigma) ** 2
            _, an, ks, _ = patch_step(g, x, beta, o)
            k = len(ims)
            ims.append(x.clone())
            idx.append(torch.full((an.numel(),), k, dtype=torch.int32, device=y.device))
            anc.append(an.clone())
            lib_.append(torch.full((an.numel(),), -math.log(beta), dtype=torch.float32, device=y.device))
            lab.append(ks.clone())
    return Pairs(torch.stack(ims), torch.cat(idx), torch.cat(anc), torch.cat(lib_), torch.cat(lab))


def train(p: Proposal, data: Pairs, steps: int, batch: int = 4096, lr: float = 2e-3,
          weight_decay: float = 1e-4, seed: int = 0, warmup: int = 50, log_every: int = 0):
    """AdamW on shuffled minibatches (epochs of a seeded permutation), with a
    linear warm-up and a cosine decay of the learning rate.  Returns the
    losses that were read (every ``log_every`` steps, and the last step)."""
    import torch
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    n = len(data)
    perm = torch.randperm(n, generator=gen).to(torch.int32).to(data.labels.device)
    pos, losses = 0, []
    for s in range(steps):
        if pos + batch > n:
            perm = torch.randperm(n, generator=gen).to(torch.int32).to(data.labels.device)
            pos = 0
        sel = perm[pos:pos + batch]
        pos += batch
        f = (s + 1) / warmup if s < warmup else 0.5 * (1 + math.cos(math.pi * (s - warmup) / max(1, steps - warmup)))
        want = (log_every and s % log_every == 0) or s == steps - 1
        loss = p.train_step(data.images, data.img_idx, data.anchors, data.log_ib, data.labels, sel,
                            lr * max(f, 0.02), weight_decay, want_loss=bool(want))
        if want:
            losses.append((s, loss))
    return losses


def hit_rate(cand, labels) -> float:
    """Fraction of patches whose exact selection is among the proposals."""
    return float((cand == labels[:, None]).any(dim=1).float().mean().item())
