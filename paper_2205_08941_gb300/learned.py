"""Orchestration of the learned initial guess: training-set assembly, the training loop and
the guarded start (learned guess, or the Palser-Manolopoulos start when the learned one is
judged poor).  All arithmetic runs in libcq's kernels (cq_guess_*, cq_lnv_*); this module
only sequences calls and moves minibatch indices.
"""
from __future__ import annotations

import torch

from . import cq


def training_set(guess: cq.Guess, samples):
    """Descriptors and pair-frame targets of converged L's: samples = [(pL, L), ...]."""
    descs, targs = [], []
    for pL, L in samples:
        d, f, _ = guess.descriptors(pL)
        descs.append(d)
        targs.append(guess.targets(pL, L, f))
    return torch.cat(descs), torch.cat(targs)


def train(guess: cq.Guess, desc, targets, epochs=40, batch=8192, lr=2e-3, seed=0,
          lr_decay=0.93):
    """Adam on shuffled minibatches; returns the loss history (one value per epoch)."""
    guess.fit_scale(desc, targets)
    n = desc.shape[0]
    gen = torch.Generator(device=desc.device)
    gen.manual_seed(seed)
    hist = []
    rate = lr
    guess.loss_sum(reset=True)
    for _ in range(epochs):
        perm = torch.randperm(n, device=desc.device, generator=gen)
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            if idx.numel() < 64:
                continue
            # asynchronous: the epoch's loss is read once, from the device-side sums
            guess.train_step(desc[idx].contiguous(), targets[idx].contiguous(), rate, loss=False)
        sq, rows = guess.loss_sum(reset=True)
        hist.append(sq / max(rows * cq.Guess.N_OUT, 1))
        rate *= lr_decay
    return hist


def accept_learned(s_learned, s_pm, n_electrons, ratio=10.0) -> bool:
    """The guard of the learned start: its RMS gradient (after the electron-number
    corrections) at most `ratio` times the PM start's, and its electron count within 1 % of
    n_electrons.  A NaN in either state fails the test."""
    return bool(s_learned["gnorm"] <= ratio * s_pm["gnorm"]
                and abs(s_learned["n_elec"] - n_electrons) <= 0.01 * n_electrons)


def guarded_start(ctx: cq.Context, guess: cq.Guess, pS, S, H, pT, T, pL, L, n_electrons,
                  prec=cq.CQ_FP64, ratio=10.0):
    """LNV object started from the learned guess, unless its RMS gradient after the
    electron-number corrections exceeds `ratio` times that of the PM start or its
    electron count is off by more than 1 % -- then from the PM start.

    Returns (lnv, used_learned, info)."""
    L_pm = ctx.zeros(pL)
    ctx.pm_guess(pS, S, H, pT, T, pL, L_pm, n_electrons / 2.0)
    if prec != cq.CQ_FP64:
        ctx.release_cache()  # the FP64 task lists of the set-up: tensor-core steps need none
    probe = ctx.lnv(pS, S, H, pL, L_pm, n_electrons, prec)
    s_pm = probe.state()
    probe.close()
    guess.apply(pL, L)
    lnv = ctx.lnv(pS, S, H, pL, L, n_electrons, prec)
    s_ml = lnv.state()
    ok = accept_learned(s_ml, s_pm, n_electrons, ratio)
    info = {"gnorm_pm": s_pm["gnorm"], "gnorm_learned": s_ml["gnorm"],
            "E_pm": s_pm["energy"], "E_learned": s_ml["energy"]}
    if ok:
        return lnv, True, info
    lnv.close()
    L.copy_(L_pm)
    return ctx.lnv(pS, S, H, pL, L, n_electrons, prec), False, info
