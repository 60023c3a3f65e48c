"""Emulated-FP64 products (CQ_FP64_EMU: eight BF16 digit planes per value on the tensor
cores, exact level sums, three-float drains) against the FP64 oracle, to the FP64 product
bound of the other parity tests: per block
||dC_ij||_F <= 1e-12 max(||C_ij||_F, 1e-3 sum_k ||A_ik||_F ||B_kj||_F).

The digits carry every value to 2^-64 of its scale group's largest magnitude, the merged
high levels round near 2^-64 of it and the dropped digit products lie below that, so the
emulated product meets the FP64 bound while the magnitudes inside a scale group (one scalar
row of A, or column of B, over sixteen atoms of K) stay within about 2^14 of one another --
the smooth decay of the method's matrices does (the 44-bohr S.X products reach values
several decades below their group's largest at the edge of the lens).  Beyond that the
error follows the group's largest value; a test states that weaker guarantee.  Cases: the 64-atom sp cell over several range
triples with alpha and beta, the 512-atom SZP cell (long k-sums, sampled rows), blocks that
no triplet reaches (exactly beta C), non-finite values (NaN where FP64 gives NaN, only in
the same scalar row), and twenty LNV steps from the oracle's start (energies to 1e-10
Ha/atom and the same step decisions as the oracle, as for FP64 products).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_08941_gb300 import cq
from paper_2205_08941_gb300 import inputs as I

from helpers import (assert_product_close, block_errors, from_oracle, gpu_pattern,
                     layout_index, natural_scale, to_oracle, upload_pairs)

pytestmark = pytest.mark.gpu
EMU = cq.CQ_FP64_EMU


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08941_gb300 import build
    build.build()
    c = cq.Context(0)
    yield c
    c.close()


class Both:
    def __init__(self, ctx, cell, r):
        self.o = O.Pattern.of_cell(cell, r)
        self.g = gpu_pattern(ctx, cell, r)
        self.idx = layout_index(self.g, self.o)

    def up(self, ctx, vals):
        return from_oracle(ctx, self.g, self.idx, vals)

    def down(self, t):
        return to_oracle(t, self.idx)


def _check(ctx, cell, ranges, seeds=(1, 2, 3), alpha=1.0, beta=0.0, rows=None, scale_by=1.0):
    A_, B_, C_ = (Both(ctx, cell, r) for r in ranges)
    A = scale_by * O.scatter(A_.o, I.random_blocks(cell, ranges[0], seeds[0], symmetric=False))
    B = O.scatter(B_.o, I.random_blocks(cell, ranges[1], seeds[1], symmetric=False))
    C0 = O.scatter(C_.o, I.random_blocks(cell, ranges[2], seeds[2], symmetric=False))
    ref = O.bsmm(alpha, A_.o, A, B_.o, B, beta, C_.o, C0.copy(), rows=rows)
    Cg = C_.up(ctx, C0)
    ctx.bsmm(alpha, A_.g, A_.up(ctx, A), B_.g, B_.up(ctx, B), beta, C_.g, Cg, prec=EMU)
    got = C_.down(Cg)
    scale = abs(alpha) * natural_scale(A_.o, A, B_.o, B, C_.o, rows=rows)
    if beta != 0.0:
        scale = scale + abs(beta) * np.abs(C0).max()
    return assert_product_close(C_.o, got, ref, scale, rows=rows)


@pytest.mark.parametrize("ranges", [(12.0, 10.0, 22.0), (12.0, 10.0, 12.0), (22.0, 22.0, 12.0),
                                    (6.0, 8.0, 5.0)])
def test_emu_parity_sp_cell(ctx, ranges):
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    _check(ctx, cell, ranges, alpha=-0.7, beta=1.3)


@pytest.mark.parametrize("ranges", [(16.0, 14.0, 30.0), (30.0, 30.0, 16.0), (14.0, 30.0, 44.0)])
def test_emu_parity_szp_512(ctx, ranges):
    cell = I.diamond_cell(4, a=10.26, sigma=0.1, seed=2, norb=9)
    rows = np.arange(0, cell.n_atoms, 29, dtype=np.int32)
    _check(ctx, cell, ranges, rows=rows)


def _wide(ctx, decades, seed=4):
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    A_, B_, C_ = (Both(ctx, cell, r) for r in (12.0, 10.0, 22.0))
    rng = np.random.default_rng(seed)
    A = O.scatter(A_.o, I.random_blocks(cell, 12.0, 1, symmetric=False))
    A *= np.repeat(10.0 ** rng.uniform(-decades, decades, A_.o.nnzb), np.diff(A_.o.off))
    B = O.scatter(B_.o, I.random_blocks(cell, 10.0, 2, symmetric=False))
    ref = O.bsmm(1.0, A_.o, A, B_.o, B, 0.0, C_.o)
    Cg = ctx.zeros(C_.g)
    ctx.bsmm(1.0, A_.g, A_.up(ctx, A), B_.g, B_.up(ctx, B), 0.0, C_.g, Cg, prec=EMU)
    return A_, A, B_, B, C_, C_.down(Cg), ref


def test_emu_spread_magnitudes_within_the_fp64_bound(ctx):
    """Operand blocks spread over four decades (10^(+-2) per block, inside the 2^14 that the
    digits' 2^-64 resolution of a scale group's largest value allows): the FP64 bound."""
    A_, A, B_, B, C_, got, ref = _wide(ctx, 2.0)
    assert_product_close(C_.o, got, ref, natural_scale(A_.o, A, B_.o, B, C_.o))


def test_emu_error_follows_the_scale_groups_largest_value(ctx):
    """Twelve decades (10^(+-6) per block) exceed that: a small term sharing a scale group
    with a large one keeps only 2^-64 of the large one's magnitude.  The error then stays
    within 1e-15 of sum_k max_k' ||A_ik'|| ||B_kj|| (each row's largest A block standing in
    for its scale group's), the guarantee the construction gives."""
    A_, A, B_, B, C_, got, ref = _wide(ctx, 6.0)
    err, _ = block_errors(C_.o, got, ref)
    po = A_.o
    nrm = np.sqrt(np.bincount(np.repeat(np.arange(po.nnzb), np.diff(po.off)), weights=A ** 2,
                              minlength=po.nnzb))
    rowmax = np.zeros(po.n)
    np.maximum.at(rowmax, po.row, nrm)
    ones = lambda p: O.Pattern(p.pos, p.box, np.ones(p.n, dtype=np.int32), p.range)
    bn = np.sqrt(np.bincount(np.repeat(np.arange(B_.o.nnzb), np.diff(B_.o.off)), weights=B ** 2,
                             minlength=B_.o.nnzb))
    scale_row = O.bsmm(1.0, ones(po), rowmax[po.row], ones(B_.o), bn, 0.0, ones(C_.o))
    assert (err <= 1e-15 * scale_row).all(), (err / np.maximum(scale_row, 1e-300)).max()


def test_emu_blocks_without_triplets_get_exactly_beta_c(ctx):
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    A_, B_, C_ = (Both(ctx, cell, r) for r in (5.0, 5.0, 12.0))
    A = O.scatter(A_.o, I.random_blocks(cell, 5.0, 1, symmetric=False))
    B = O.scatter(B_.o, I.random_blocks(cell, 5.0, 2, symmetric=False))
    C0 = O.scatter(C_.o, I.random_blocks(cell, 12.0, 3, symmetric=False))
    scale = natural_scale(A_.o, A, B_.o, B, C_.o)
    empty = scale == 0.0
    assert empty.any() and not empty.all()
    ev = np.repeat(empty, np.diff(C_.o.off))
    Ag, Bg = A_.up(ctx, A), B_.up(ctx, B)
    for beta in (0.0, 1.3):
        ref = O.bsmm(-0.7, A_.o, A, B_.o, B, beta, C_.o, C0.copy())
        Cg = C_.up(ctx, C0)
        ctx.bsmm(-0.7, A_.g, Ag, B_.g, Bg, beta, C_.g, Cg, prec=EMU)
        got = C_.down(Cg)
        assert np.array_equal(got[ev], beta * C0[ev]), beta
        assert_product_close(C_.o, got, ref, 0.7 * scale + beta * np.abs(ref).max())


def test_emu_carries_non_finite_values_as_nan(ctx):
    """An infinity or a NaN in A poisons its scale group (one scalar row of A over sixteen
    atoms of K): every C value the FP64 product makes NaN is NaN, and NaN appears only in the
    same scalar row."""
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    A_, B_, C_ = (Both(ctx, cell, r) for r in (12.0, 10.0, 22.0))
    A = O.scatter(A_.o, I.random_blocks(cell, 12.0, 1, symmetric=False))
    B = O.scatter(B_.o, I.random_blocks(cell, 10.0, 2, symmetric=False))
    blk = 37
    i_atom = int(A_.o.row[blk])
    pos = int(A_.o.off[blk]) + 1 * int(cell.nb[int(A_.o.col[blk])]) + 2
    An = A.copy()
    An[pos] = np.nan
    reach = np.isnan(O.bsmm(1.0, A_.o, An, B_.o, B, 0.0, C_.o))
    assert reach.any()
    row1 = np.zeros(C_.o.n_values, dtype=bool)
    for b in np.nonzero(C_.o.row == i_atom)[0]:
        nj = int(cell.nb[int(C_.o.col[b])])
        row1[int(C_.o.off[b]) + nj:int(C_.o.off[b]) + 2 * nj] = True
    Bg = B_.up(ctx, B)
    for bad in (-np.inf, np.nan):
        Ab = A.copy()
        Ab[pos] = bad
        Cg = ctx.zeros(C_.g)
        ctx.bsmm(1.0, A_.g, A_.up(ctx, Ab), B_.g, Bg, 0.0, C_.g, Cg, prec=EMU)
        got = C_.down(Cg)
        assert np.isnan(got[reach]).all(), bad
        assert np.isfinite(got[~row1]).all(), bad


def test_emu_lnv_matches_the_oracle_20_steps(ctx):
    """LNV with every product emulated follows the FP64 oracle as the FP64 products do."""
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    Spb, Hpb = I.overlap_hamiltonian(cell, I.silicon_model(10.0))
    pS, pL = Both(ctx, cell, 10.0), Both(ctx, cell, 12.0)
    pX, pU = O.Pattern.of_cell(cell, 22.0), O.Pattern.of_cell(cell, 32.0)
    S_o, H_o = O.scatter(pS.o, Spb), O.scatter(pS.o, Hpb)
    T_o = O.hotelling_init(pS.o, S_o, pL.o)
    for _ in range(10):
        T_o, _ = O.hotelling_step(pS.o, S_o, pL.o, T_o, pX)
    L0 = O.pm_guess(pS.o, S_o, H_o, pL.o, T_o, pX, pL.o, 128.0)
    lo = O.LNV(pS.o, S_o, H_o, pL.o, L0, 256.0, pX, pU)
    S_g, H_g = upload_pairs(ctx, pS.g, Spb), upload_pairs(ctx, pS.g, Hpb)
    L_g = pL.up(ctx, L0)
    lg = ctx.lnv(pS.g, S_g, H_g, pL.g, L_g, 256.0, prec=EMU)
    tol = 1e-10 * cell.n_atoms
    assert lg.state()["energy"] == pytest.approx(lo.E, abs=tol)
    for k in range(20):
        ro, rg = lo.step(), lg.step()
        assert rg["energy"] == pytest.approx(ro["E"], abs=tol), k
        assert rg["n_elec"] == pytest.approx(ro["N"], abs=tol), k
        assert (rg["restart"], rg["fallback"], rg["n_corr"]) == (
            int(ro["restart"]), int(ro["fallback"]), ro["n_corr"]), k
        assert rg["gnorm"] == pytest.approx(ro["gnorm"], rel=1e-5, abs=1e-9), k
    lg.close()
