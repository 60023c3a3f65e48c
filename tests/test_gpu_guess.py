"""Learned initial guess on the GPU against its oracle, and its gain over the
Palser-Manolopoulos start counted in LNV iterations.

Tolerances: descriptors and frames are computed in FP64 and stored/accumulated in FP32
(relative 1e-5); the network in FP32-weight test mode matches the FP64 oracle to 1e-4
(outputs) / 1e-3 (gradients, FP32 accumulation over the batch); with BF16 weights the
outputs match to 1e-2 of their scale.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import guess as G
from paper_2205_08941_gb300 import cq, learned
from paper_2205_08941_gb300 import inputs as I

from helpers import gpu_pattern, layout_index, to_oracle, upload_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08941_gb300 import build
    build.build()
    c = cq.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small(ctx):
    cell = I.diamond_cell(2, a=10.26, sigma=0.12, seed=9, norb=9)
    po = O.Pattern.of_cell(cell, 8.0)
    pg = gpu_pattern(ctx, cell, 8.0)
    return cell, po, pg


def test_descriptors_frames_targets_match_oracle(ctx, small):
    cell, po, pg = small
    g = cq.Guess(ctx, seed=1)
    desc, frames, pairs = g.descriptors(pg)
    ref_pairs = G.pairs_of(po)
    assert np.array_equal(pairs.cpu().numpy(), ref_pairs)
    L = O.scatter(po, I.random_blocks(cell, 8.0, 4))
    idx = layout_index(pg, po)
    Lg = torch.zeros(pg.n_values, dtype=torch.float64, device="cuda:0")
    Lg[idx] = torch.tensor(L, device="cuda:0")
    targ = g.targets(pg, Lg, frames).cpu().numpy()
    d, f = desc.cpu().numpy(), frames.cpu().numpy()
    for q, b in enumerate(ref_pairs):
        F, fd = G.frame_and_descriptor(po, b)
        assert np.allclose(f[q].reshape(3, 3), F, atol=2e-6)
        assert np.allclose(d[q], fd, rtol=1e-5, atol=1e-5 * max(1.0, np.abs(fd).max()))
        assert np.allclose(targ[q], G.target(F, G.block(po, L, b)), atol=2e-6)
    g.close()


def _net_case(ctx, fp32):
    rng = np.random.default_rng(7)
    g = cq.Guess(ctx, seed=3, fp32_weights=fp32)
    X = rng.normal(size=(300, 64)).astype(np.float32) * 2 + 1
    T = rng.normal(size=(300, 81)).astype(np.float32)
    im, isc = rng.normal(size=64).astype(np.float32), (1 + rng.random(64)).astype(np.float32)
    om, osc = rng.normal(size=81).astype(np.float32), (1 + rng.random(81)).astype(np.float32)
    g.set_scale(im, isc, om, osc)
    w, b = g.params()
    b = rng.normal(size=b.shape).astype(np.float32) * 0.1
    g.set_params(w, b)
    return g, X, T, (im, isc, om, osc), w, b


def test_network_fp32_mode_matches_oracle(ctx):
    g, X, T, (im, isc, om, osc), w, b = _net_case(ctx, True)
    Xg, Tg = torch.tensor(X, device="cuda:0"), torch.tensor(T, device="cuda:0")
    Y = g.forward(Xg).cpu().numpy()
    Yo, _ = G.forward(w, b, X, im, isc)
    assert np.abs(Y - Yo).max() <= 1e-4 * max(1.0, np.abs(Yo).max())
    loss, gw, gb = g.train_step(Xg, Tg, 0.0, grads=True)
    lo, gwo, gbo = G.loss_and_grads(w, b, X, T, im, isc, om, osc)
    assert loss == pytest.approx(lo, rel=1e-4)
    assert np.abs(gw - gwo).max() <= 1e-3 * np.abs(gwo).max()
    assert np.abs(gb - gbo).max() <= 1e-3 * np.abs(gbo).max()
    g.close()


def test_network_bf16_mode_within_bf16_tolerance(ctx):
    """BF16 weights: every contraction runs on the tensor cores (tcgen05, BF16 inputs, FP32
    accumulation).  Outputs to 1e-2 of their scale; loss to 1e-2; weight and bias gradients
    to 3e-2 of their largest entry (BF16 rounds the activations, dZ and the weights to 2^-9
    relative before FP32 accumulation over the batch)."""
    g, X, T, (im, isc, om, osc), w, b = _net_case(ctx, False)
    Xg, Tg = torch.tensor(X, device="cuda:0"), torch.tensor(T, device="cuda:0")
    Y = g.forward(Xg).cpu().numpy()
    Yo, _ = G.forward(w, b, X, im, isc)
    assert np.abs(Y - Yo).max() <= 1e-2 * max(1.0, np.abs(Yo).max())
    loss, gw, gb = g.train_step(Xg, Tg, 0.0, grads=True)
    lo, gwo, gbo = G.loss_and_grads(w, b, X, T, im, isc, om, osc)
    assert loss == pytest.approx(lo, rel=1e-2)
    assert np.abs(gw - gwo).max() <= 3e-2 * np.abs(gwo).max()
    assert np.abs(gb - gbo).max() <= 3e-2 * np.abs(gbo).max()
    g.close()


def test_loss_sums_of_asynchronous_steps_match_the_step_losses(ctx):
    """Steps that read nothing back still add their squared-error sums and rows on the
    device: with lr = 0 (weights fixed) the running sums of three such steps equal the
    losses the same batches report one by one, and a reset starts them again at zero."""
    g, X, T, _, _, _ = _net_case(ctx, True)
    Xg, Tg = torch.tensor(X, device="cuda:0"), torch.tensor(T, device="cuda:0")
    cuts = [(0, 100), (100, 220), (220, 300)]
    g.loss_sum(reset=True)
    want = sum(g.train_step(Xg[a:b].contiguous(), Tg[a:b].contiguous(), 0.0) * (b - a) * 81
               for a, b in cuts)
    g.loss_sum(reset=True)
    for a, b in cuts:
        assert g.train_step(Xg[a:b].contiguous(), Tg[a:b].contiguous(), 0.0, loss=False) is None
    sq, rows = g.loss_sum(reset=True)
    assert rows == 300
    assert sq == pytest.approx(want, rel=1e-5)
    assert g.loss_sum(reset=False) == (0.0, 0)
    g.close()


# ---------------------------------------------------------------- training and gain

def _solve(ctx, cell, steps=40, start=None, guess=None, gtol=1e-6):
    """Hotelling + start + LNV until the RMS gradient is below gtol; returns iterations."""
    Spb, Hpb = I.overlap_hamiltonian(cell, I.silicon_model(14.0))
    pS, pL = gpu_pattern(ctx, cell, 14.0), gpu_pattern(ctx, cell, 16.0)
    S, H = upload_pairs(ctx, pS, Spb), upload_pairs(ctx, pS, Hpb)
    T = ctx.zeros(pL)
    ctx.hotelling_init(pS, S, pL, T)
    for _ in range(12):
        ctx.hotelling_step(pS, S, pL, T)
    ne = 4.0 * cell.n_atoms
    L = ctx.zeros(pL)
    used = None
    if guess is None:
        ctx.pm_guess(pS, S, H, pL, T, pL, L, ne / 2.0)
        lnv = ctx.lnv(pS, S, H, pL, L, ne)
    else:
        lnv, used, _ = learned.guarded_start(ctx, guess, pS, S, H, pL, T, pL, L, ne)
    it = 0
    st = lnv.state()
    while st["gnorm"] > gtol and it < steps:
        st = lnv.step()
        it += 1
    E = st["energy"]
    lnv.close()
    return it, E, pL, L, used


def test_learned_guess_saves_lnv_iterations(ctx):
    # training data: converged L of thermally displaced 216-atom SZP cells (sigma 0.1-0.3)
    rng = np.random.default_rng(1000)
    samples = []
    for k in range(5):
        cell = I.diamond_cell(3, a=10.26, sigma=float(rng.uniform(0.1, 0.3)), seed=1000 + k,
                              norb=9)
        _, _, pL, L, _ = _solve(ctx, cell, steps=60, gtol=1e-7)
        samples.append((pL, L))
    g = cq.Guess(ctx, seed=11)
    desc, targ = learned.training_set(g, samples)
    hist = learned.train(g, desc, targ, epochs=60, batch=4096, lr=2e-3, lr_decay=0.96)
    assert hist[-1] < 0.5 * hist[0]
    # held-out cell
    cell = I.diamond_cell(3, a=10.26, sigma=0.2, seed=4242, norb=9)
    it_pm, E_pm, *_ = _solve(ctx, cell, steps=80)
    it_ml, E_ml, _, _, used = _solve(ctx, cell, steps=80, guess=g)
    print(f"learned-guess gain: loss {hist[0]:.4f} -> {hist[-1]:.4f}, LNV iterations to "
          f"RMS gradient 1e-6: PM start {it_pm}, learned start {it_ml} (used={used})")
    assert used
    assert abs(E_ml - E_pm) / cell.n_atoms < 1e-9
    assert it_ml < it_pm, (it_ml, it_pm)
    g.close()
