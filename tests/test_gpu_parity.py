"""CUDA path against the CPU oracle on the same seeded inputs, through the C ABI.

Tolerances: patterns, task counts and branch decisions are compared exactly; block products
per block with ||dC_ij||_F <= 1e-12 max(||C_ij||_F, 1e-3 sum_k ||A_ik|| ||B_kj||) (the
relative 1e-12 bound, widened only where a block is small by cancellation); traces and
energies to 1e-10 Ha per atom.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_08941_gb300 import cq
from paper_2205_08941_gb300 import inputs as I

from helpers import (assert_product_close, block_errors, from_oracle, gpu_pattern,
                     layout_index, natural_scale, to_oracle, upload_pairs)

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
def si64():
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    S, H = I.overlap_hamiltonian(cell, I.silicon_model(10.0))
    return cell, S, H


def mixed_cell():
    cell = I.diamond_cell(2, a=10.26, sigma=0.2, seed=7, norb=4)
    rng = np.random.default_rng(11)
    cell.nb = rng.choice(np.array([1, 4, 5, 9, 13], dtype=np.int32), size=cell.n_atoms)
    return cell


class Both:
    """A pattern on both paths plus the layout map between them."""

    def __init__(self, ctx, cell, r):
        self.o = O.Pattern.of_cell(cell, r)
        self.g = gpu_pattern(ctx, cell, r)
        self.idx = layout_index(self.g, self.o)

    def up(self, ctx, vals):
        return from_oracle(ctx, self.g, self.idx, vals)

    def down(self, t):
        return to_oracle(t, self.idx)


# ------------------------------------------------------------------ A1 patterns

@pytest.mark.parametrize("r", [0.0, 3.0, 10.0, 12.0, 16.5, 22.0, 32.0])
def test_pattern_bitexact_si64(ctx, si64, r):
    b = Both(ctx, si64[0], r)  # layout_index asserts row_ptr and col equal
    rp, col, off, tr = b.g.export()
    tr = tr.cpu().numpy()
    assert np.array_equal(tr[tr], np.arange(b.o.nnzb))
    assert np.array_equal(b.o.row[tr], b.o.col)
    assert int(off[0]) == 0 and np.all(off.cpu().numpy() % 2 == 0)


def test_pattern_bitexact_512_and_mixed(ctx):
    cell = I.diamond_cell(4, a=10.26, sigma=0.1, seed=2, norb=9)
    for r in (14.0, 16.0, 30.0):
        Both(ctx, cell, r)
    m = mixed_cell()
    for r in (7.0, 13.0):
        Both(ctx, m, r)


# ------------------------------------------------------------------ A2/A3 product

def _random(cell, r, seed, sym=False):
    return I.random_blocks(cell, r, seed, symmetric=sym)


@pytest.mark.parametrize("ranges", [(12.0, 10.0, 22.0), (12.0, 10.0, 12.0), (22.0, 10.0, 32.0),
                                    (32.0, 22.0, 12.0), (6.0, 8.0, 5.0)])
def test_bsmm_parity_si64(ctx, si64, ranges):
    cell = si64[0]
    A_, B_, C_ = (Both(ctx, cell, r) for r in ranges)
    A = O.scatter(A_.o, _random(cell, ranges[0], 1))
    B = O.scatter(B_.o, _random(cell, ranges[1], 2))
    C0 = O.scatter(C_.o, _random(cell, ranges[2], 3))
    ref = O.bsmm(-0.7, A_.o, A, B_.o, B, 1.3, C_.o, C0.copy())
    Cg = C_.up(ctx, C0)
    ctx.bsmm(-0.7, A_.g, A_.up(ctx, A), B_.g, B_.up(ctx, B), 1.3, C_.g, Cg)
    got = C_.down(Cg)
    scale = natural_scale(A_.o, A, B_.o, B, C_.o)
    assert_product_close(C_.o, got, ref, 0.7 * scale + 1.3 * np.abs(
        np.sqrt(np.bincount(np.repeat(np.arange(C_.o.nnzb), np.diff(C_.o.off)),
                            weights=C0 ** 2, minlength=C_.o.nnzb))))
    t, f = ctx.bsmm_work(A_.g, B_.g, C_.g)
    assert (t, f) == O.triplets(A_.o, B_.o, C_.o)


def test_bsmm_parity_mixed_basis(ctx):
    cell = mixed_cell()
    A_, B_, C_ = (Both(ctx, cell, r) for r in (9.0, 7.0, 13.0))
    A = O.scatter(A_.o, _random(cell, 9.0, 4))
    B = O.scatter(B_.o, _random(cell, 7.0, 5))
    ref = O.bsmm(1.0, A_.o, A, B_.o, B, 0.0, C_.o)
    Cg = ctx.empty(C_.g)
    ctx.bsmm(1.0, A_.g, A_.up(ctx, A), B_.g, B_.up(ctx, B), 0.0, C_.g, Cg)
    assert_product_close(C_.o, C_.down(Cg), ref, natural_scale(A_.o, A, B_.o, B, C_.o))


def test_bsmm_szp_512_long_segments(ctx):
    # 9x9 blocks, segments from ~30 to ~800 tasks (every lane-split width)
    cell = I.diamond_cell(4, a=10.26, sigma=0.1, seed=2, norb=9)
    for ranges in ((16.0, 14.0, 30.0), (30.0, 30.0, 16.0)):
        A_, B_, C_ = (Both(ctx, cell, r) for r in ranges)
        A = O.scatter(A_.o, _random(cell, ranges[0], 6))
        B = O.scatter(B_.o, _random(cell, ranges[1], 7))
        rows = np.arange(0, cell.n_atoms, 37, dtype=np.int32)
        ref = O.bsmm(1.0, A_.o, A, B_.o, B, 0.0, C_.o, rows=rows)
        Cg = ctx.empty(C_.g)
        ctx.bsmm(1.0, A_.g, A_.up(ctx, A), B_.g, B_.up(ctx, B), 0.0, C_.g, Cg)
        scale = natural_scale(A_.o, A, B_.o, B, C_.o, rows=rows)
        assert_product_close(C_.o, C_.down(Cg), ref, scale, rows=rows)


def test_bsmm_deterministic(ctx, si64):
    cell = si64[0]
    A_, B_, C_ = (Both(ctx, cell, r) for r in (12.0, 10.0, 22.0))
    A = A_.up(ctx, O.scatter(A_.o, _random(cell, 12.0, 1)))
    B = B_.up(ctx, O.scatter(B_.o, _random(cell, 10.0, 2)))
    c_a, c_b = ctx.empty(C_.g), ctx.empty(C_.g)
    ctx.bsmm(1.0, A_.g, A, B_.g, B, 0.0, C_.g, c_a)
    ctx.bsmm(1.0, A_.g, A, B_.g, B, 0.0, C_.g, c_b)
    assert torch.equal(c_a[C_.idx], c_b[C_.idx])


# ------------------------------------------------------------------ K5 traces, dots

def test_trace_and_dot_parity(ctx):
    cell = mixed_cell()
    A_, B_ = Both(ctx, cell, 9.0), Both(ctx, cell, 6.0)
    A = O.scatter(A_.o, _random(cell, 9.0, 8))
    B = O.scatter(B_.o, _random(cell, 6.0, 9))
    t = ctx.trace_prod(A_.g, A_.up(ctx, A), B_.g, B_.up(ctx, B))
    assert t == pytest.approx(O.trace_prod(A_.o, A, B_.o, B), rel=1e-13, abs=1e-13)
    d = ctx.dot(A_.g, A_.up(ctx, A), A_.up(ctx, A))
    assert d == pytest.approx(O.dot(A, A), rel=1e-13)


# ------------------------------------------------------------------ A4 Hotelling, A7

def _setup_si64(ctx, si64, rl=12.0):
    cell, Spb, Hpb = si64
    pS, pL = Both(ctx, cell, 10.0), Both(ctx, cell, rl)
    S_o, H_o = O.scatter(pS.o, Spb), O.scatter(pS.o, Hpb)
    S_g, H_g = upload_pairs(ctx, pS.g, Spb), upload_pairs(ctx, pS.g, Hpb)
    assert np.array_equal(pS.down(S_g), S_o)
    return cell, pS, pL, S_o, H_o, S_g, H_g


@pytest.mark.parametrize("rt", [12.0, 18.0])
def test_hotelling_parity_si64(ctx, si64, rt):
    cell, pS, pT, S_o, _, S_g, _ = _setup_si64(ctx, si64, rt)
    pV = O.Pattern.of_cell(cell, 10.0 + rt)
    T_o = O.hotelling_init(pS.o, S_o, pT.o)
    T_g = ctx.zeros(pT.g)
    ctx.hotelling_init(pS.g, S_g, pT.g, T_g)
    assert np.array_equal(pT.down(T_g), T_o)
    for _ in range(10):
        T_o, r_o = O.hotelling_step(pS.o, S_o, pT.o, T_o, pV)
        r_g = ctx.hotelling_step(pS.g, S_g, pT.g, T_g)
        assert r_g == pytest.approx(r_o, rel=1e-11, abs=1e-14)
    err, nrm = block_errors(pT.o, pT.down(T_g), T_o)
    assert err.max() < 1e-12 * nrm.max()


def test_overlap_inverse_cg_parity_si64(ctx, si64):
    """Least-squares inverse on P_T by CG: residual and gradient histories and the final T
    against the oracle, from a symmetric start that does not commute with S."""
    cell, pS, pT, S_o, _, S_g, _ = _setup_si64(ctx, si64, 12.0)
    pV = O.Pattern.of_cell(cell, 22.0)
    T0 = (O.hotelling_init(pS.o, S_o, pT.o)
          + 0.05 * O.scatter(pT.o, I.random_blocks(cell, 12.0, 31)))
    T_o, r_o, g_o = O.overlap_inverse_cg(pS.o, S_o, pT.o, T0, pV, 25)
    T_g = pT.up(ctx, T0)
    r0, g0 = ctx.overlap_inverse_cg(pS.g, S_g, pT.g, T_g, 0)   # no step: start values only
    assert len(r0) == 1 and r0[0] == pytest.approx(r_o[0], rel=1e-12)
    assert np.array_equal(pT.down(T_g), T0)
    r_g, g_g = ctx.overlap_inverse_cg(pS.g, S_g, pT.g, T_g, 25)
    assert len(r_g) == len(r_o) == 26
    assert r_g == pytest.approx(r_o, rel=1e-9)
    assert g_g == pytest.approx(g_o, rel=1e-6, abs=1e-12 * g_o[0])
    err, nrm = block_errors(pT.o, pT.down(T_g), T_o)
    assert err.max() < 1e-10 * nrm.max()
    # the reported residual is the one of the T returned (Hotelling reports the incoming T's)
    assert ctx.hotelling_step(pS.g, S_g, pT.g, T_g.clone()) == pytest.approx(r_g[-1], rel=1e-10)


def test_pm_guess_and_mcweeny_parity_si64(ctx, si64):
    cell, pS, pL, S_o, H_o, S_g, H_g = _setup_si64(ctx, si64, 12.0)
    pX, pU, p2L = (O.Pattern.of_cell(cell, r) for r in (22.0, 32.0, 24.0))
    T_o = O.hotelling_init(pS.o, S_o, pL.o)
    T_g = ctx.zeros(pL.g)
    ctx.hotelling_init(pS.g, S_g, pL.g, T_g)
    for _ in range(10):
        T_o, _ = O.hotelling_step(pS.o, S_o, pL.o, T_o, pX)
        ctx.hotelling_step(pS.g, S_g, pL.g, T_g)
    L_o = O.pm_guess(pS.o, S_o, H_o, pL.o, T_o, pX, pL.o, 128.0)
    L_g = ctx.zeros(pL.g)
    ctx.pm_guess(pS.g, S_g, H_g, pL.g, T_g, pL.g, L_g, 128.0)
    err, nrm = block_errors(pL.o, pL.down(L_g), L_o)
    assert err.max() < 1e-12 * nrm.max()
    M_o = O.mcweeny_step(pS.o, S_o, pL.o, L_o, pX, pU, p2L)
    ctx.mcweeny_step(pS.g, S_g, pL.g, L_g)
    err, nrm = block_errors(pL.o, pL.down(L_g), M_o)
    assert err.max() < 1e-12 * nrm.max()


# ------------------------------------------------------------------ A5/A6 LNV

def test_lnv_parity_si64_20_steps(ctx, si64):
    cell, pS, pL, S_o, H_o, S_g, H_g = _setup_si64(ctx, si64, 12.0)
    pX, pU = O.Pattern.of_cell(cell, 22.0), O.Pattern.of_cell(cell, 32.0)
    T_o = O.hotelling_init(pS.o, S_o, pL.o)
    for _ in range(10):
        T_o, _ = O.hotelling_step(pS.o, S_o, pL.o, T_o, pX)
    L0 = O.pm_guess(pS.o, S_o, H_o, pL.o, T_o, pX, pL.o, 128.0)
    lo = O.LNV(pS.o, S_o, H_o, pL.o, L0, 256.0, pX, pU)
    L_g = pL.up(ctx, L0)  # identical start on both paths
    lg = ctx.lnv(pS.g, S_g, H_g, pL.g, L_g, 256.0)
    st = lg.state()
    tol = 1e-10 * cell.n_atoms
    assert st["energy"] == pytest.approx(lo.E, abs=tol)
    assert st["n_corr"] == lo.n_corrections_initial
    for k in range(20):
        ro = lo.step()
        rg = lg.step()
        assert rg["energy"] == pytest.approx(ro["E"], abs=tol), k
        assert rg["n_elec"] == pytest.approx(ro["N"], abs=tol), k
        assert (rg["restart"], rg["fallback"], rg["n_corr"]) == (
            int(ro["restart"]), int(ro["fallback"]), ro["n_corr"]), k
        # the RMS gradient is a difference of O(1) terms: compare it to 1e-9 Ha absolute,
        # two decades under the 1e-8 convergence threshold
        assert rg["gnorm"] == pytest.approx(ro["gnorm"], rel=1e-5, abs=1e-9), k
    err, nrm = block_errors(pL.o, pL.down(L_g), lo.L)
    assert err.max() < 1e-8 * nrm.max()


def _lnv_pair_si64(ctx, si64):
    """Oracle and GPU LNV objects on the 64-atom cell from the same PM start, with the
    Hotelling T (12 steps, on P_L) both sides precondition with."""
    cell, pS, pL, S_o, H_o, S_g, H_g = _setup_si64(ctx, si64, 12.0)
    pX, pU = O.Pattern.of_cell(cell, 22.0), O.Pattern.of_cell(cell, 32.0)
    T_o = O.hotelling_init(pS.o, S_o, pL.o)
    for _ in range(12):
        T_o, _ = O.hotelling_step(pS.o, S_o, pL.o, T_o, pX)
    L0 = O.pm_guess(pS.o, S_o, H_o, pL.o, T_o, pX, pL.o, 128.0)
    lo = O.LNV(pS.o, S_o, H_o, pL.o, L0, 256.0, pX, pU)
    L_g = pL.up(ctx, L0)
    lg = ctx.lnv(pS.g, S_g, H_g, pL.g, L_g, 256.0)
    return cell, pS, pL, T_o, pL.up(ctx, T_o), lo, lg, L_g


def test_preconditioned_lnv_parity_si64(ctx, si64):
    """Search directions from Z = sym(mask_L(T G T)): the GPU steps follow the oracle's
    step by step, and reach the 1e-8 RMS gradient in fewer steps than the plain gradient
    (Development Priorities: overlap inversion feeding the density-matrix minimisation)."""
    cell, pS, pL, T_o, T_g, lo, lg, L_g = _lnv_pair_si64(ctx, si64)
    lo.set_preconditioner(pL.o, T_o, O.Pattern.of_cell(cell, 24.0))
    lg.set_preconditioner(pL.g, T_g)
    tol = 1e-10 * cell.n_atoms
    for k in range(15):
        ro, rg = lo.step(), lg.step()
        assert rg["energy"] == pytest.approx(ro["E"], abs=tol), k
        assert rg["n_elec"] == pytest.approx(ro["N"], abs=tol), k
        assert (rg["restart"], rg["fallback"], rg["n_corr"]) == (
            int(ro["restart"]), int(ro["fallback"]), ro["n_corr"]), k
        assert rg["gnorm"] == pytest.approx(ro["gnorm"], rel=1e-5, abs=1e-9), k
    err, nrm = block_errors(pL.o, pL.down(L_g), lo.L)
    assert err.max() < 1e-8 * nrm.max()
    # the step's flop count includes the two preconditioner products; switching the
    # preconditioner off removes them
    with_t = lg.step_flops()
    lg.set_preconditioner(None, None)
    plain_flops = lg.step_flops()
    assert with_t > plain_flops > 0

    def steps_to(lnv, cap=60):
        k = 0
        while lnv.state()["gnorm"] > 1e-8 and k < cap:
            lnv.step()
            k += 1
        return k

    _, _, _, _, T2, _, pre, _ = _lnv_pair_si64(ctx, si64)
    pre.set_preconditioner(pL.g, T2)
    _, _, _, _, _, _, plain, _ = _lnv_pair_si64(ctx, si64)
    n_pre, n_plain = steps_to(pre), steps_to(plain)
    assert pre.state()["gnorm"] <= 1e-8 and plain.state()["gnorm"] <= 1e-8
    assert n_pre < n_plain, (n_pre, n_plain)
    assert pre.state()["energy"] == pytest.approx(plain.state()["energy"], abs=tol)


def test_identity_preconditioner_gives_the_plain_steps_si64(ctx, si64):
    cell, pS, pL, T_o, T_g, lo, lg, L_g = _lnv_pair_si64(ctx, si64)
    ident = pL.up(ctx, O.identity(pL.o))
    _, _, _, _, _, _, plain, _ = _lnv_pair_si64(ctx, si64)
    lg.set_preconditioner(pL.g, ident)
    for k in range(6):
        a, b = plain.step(), lg.step()
        assert b["energy"] == pytest.approx(a["energy"], abs=1e-10 * cell.n_atoms), k
        assert b["alpha"] == pytest.approx(a["alpha"], rel=1e-8), k
        assert (b["restart"], b["fallback"], b["n_corr"]) == (a["restart"], a["fallback"],
                                                              a["n_corr"]), k
    other = Both(ctx, I.diamond_cell(2, a=10.26, sigma=0.05, seed=99, norb=4), 12.0)
    with pytest.raises(cq.CQError) as e:   # T on another geometry is refused
        lg.set_preconditioner(other.g, ctx.zeros(other.g))
    assert e.value.status == 2


def test_failed_preconditioner_set_leaves_the_plain_step_si64(ctx, si64):
    """A set that fails (T on a pattern of another context) switches the preconditioner off
    instead of leaving a half-updated one: the next step is the plain step from the same L,
    although a valid, non-trivial T was set before."""
    cell, pS, pL, T_o, T_g, lo, lg, L_g = _lnv_pair_si64(ctx, si64)
    _, _, _, _, _, _, plain, _ = _lnv_pair_si64(ctx, si64)
    lg.set_preconditioner(pL.g, T_g)
    c2 = cq.Context(0)
    try:
        foreign = gpu_pattern(c2, cell, 12.0)
        with pytest.raises(cq.CQError) as e:
            lg.set_preconditioner(foreign, c2.zeros(foreign))
        assert e.value.status == 2
        a, b = plain.step(), lg.step()
        assert b["energy"] == a["energy"] and b["alpha"] == a["alpha"], (a, b)
        assert (b["restart"], b["fallback"], b["n_corr"]) == (a["restart"], a["fallback"],
                                                              a["n_corr"])
        assert b["flops"] == a["flops"]
    finally:
        c2.close()


# ------------------------------------------------------------------ error paths

def test_errors_are_reported_not_raised_on_device(ctx, si64):
    cell = si64[0]
    p = gpu_pattern(ctx, cell, 5.0)
    pb = I.random_blocks(cell, 10.0, 1)
    with pytest.raises(cq.CQError) as e:
        upload_pairs(ctx, p, pb)          # pairs beyond the pattern's range
    assert e.value.status == 2
    other = I.diamond_cell(2, a=10.26, sigma=0.05, seed=99, norb=4)
    q = gpu_pattern(ctx, other, 5.0)
    A = ctx.zeros(p)
    with pytest.raises(cq.CQError) as e:
        ctx.bsmm(1.0, p, A, q, ctx.zeros(q), 0.0, p, ctx.zeros(p))
    assert e.value.status == 2
    with pytest.raises(cq.CQError) as e:
        ctx.bsmm(1.0, p, A, p, A, 0.0, p, A)  # C aliases A
    assert e.value.status == 1
    c2 = cq.Context(0)
    c2.set_mem_limit(1 << 20)
    big = I.diamond_cell(4, a=10.26, sigma=0.1, seed=2, norb=9)
    with pytest.raises(cq.CQError) as e:
        gpu_pattern(c2, big, 30.0)
    assert e.value.status == 3
    c2.close()
