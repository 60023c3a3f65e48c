"""Split-BF16 tensor-core product (three BF16 terms per FP64 value, six cross products,
FP32 accumulation drained into double-float sums) against the FP64 oracle.

Error model per product term a*b: operand truncation after three terms and the dropped
cross terms (A1B2, A2B1, A2B2) give at most ~4 * 2^-24 |a||b| (2.4e-7); FP32 accumulation
over one drain period (4 chunks of 3 K steps = 12 accumulations per split product into
the tensor-memory accumulator, 72 in all) adds at most 72 * 2^-24 (4.3e-6) of the summed
magnitudes.  The per-block bound tested is therefore
||dC_ij||_F <= 1e-5 * sum_k ||A_ik||_F ||B_kj||_F, and the typical (RMS) error is checked at
1e-6 of the same scale.
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


def _check_split(ctx, cell, ranges, seeds=(1, 2, 3), alpha=1.0, beta=0.0, rows=None):
    A_, B_, C_ = (Both(ctx, cell, r) for r in ranges)
    A = O.scatter(A_.o, I.random_blocks(cell, ranges[0], seeds[0], symmetric=False))
    B = O.scatter(B_.o, I.random_blocks(cell, ranges[1], seeds[1], symmetric=False))
    C0 = O.scatter(C_.o, I.random_blocks(cell, ranges[2], seeds[2], symmetric=False))
    ref = O.bsmm(alpha, A_.o, A, B_.o, B, beta, C_.o, C0.copy(), rows=rows)
    Cg = C_.up(ctx, C0)
    ctx.bsmm(alpha, A_.g, A_.up(ctx, A), B_.g, B_.up(ctx, B), beta, C_.g, Cg,
             prec=cq.CQ_SPLIT_BF16X3)
    got = C_.down(Cg)
    err, _ = block_errors(C_.o, got, ref)
    scale = abs(alpha) * natural_scale(A_.o, A, B_.o, B, C_.o, rows=rows)
    if rows is not None:
        sel = np.isin(C_.o.row, rows)
        err, scale = err[sel], scale[sel]
    rel = err / np.maximum(scale, 1e-300)
    assert rel.max() <= 1e-5, rel.max()
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, np.sqrt(np.mean(rel ** 2))
    return rel


@pytest.mark.parametrize("ranges", [(12.0, 10.0, 22.0), (12.0, 10.0, 12.0), (22.0, 22.0, 12.0),
                                    (6.0, 8.0, 5.0)])
def test_split_parity_sp_cell(ctx, ranges):
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    _check_split(ctx, cell, ranges, alpha=-0.7, beta=1.3)


@pytest.mark.parametrize("ranges", [(16.0, 14.0, 30.0), (30.0, 30.0, 16.0), (14.0, 30.0, 44.0)])
def test_split_parity_szp_512(ctx, ranges):
    cell = I.diamond_cell(4, a=10.26, sigma=0.1, seed=2, norb=9)
    rows = np.arange(0, cell.n_atoms, 29, dtype=np.int32)
    _check_split(ctx, cell, ranges, rows=rows)


def test_blocks_without_triplets_get_exactly_beta_c(ctx):
    """P_C reaches beyond r_A + r_B, so some C blocks have no (i, k, j) at all (and some
    split tiles may have no K chunk): those must come out as exactly beta C_ij (zero for
    beta = 0) in both precisions, the others as the product."""
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    A_, B_, C_ = (Both(ctx, cell, r) for r in (5.0, 5.0, 12.0))
    A = O.scatter(A_.o, I.random_blocks(cell, 5.0, 1, symmetric=False))
    B = O.scatter(B_.o, I.random_blocks(cell, 5.0, 2, symmetric=False))
    C0 = O.scatter(C_.o, I.random_blocks(cell, 12.0, 3, symmetric=False))
    scale = natural_scale(A_.o, A, B_.o, B, C_.o)
    empty = scale == 0.0                       # no triplet reaches these blocks
    assert empty.any() and not empty.all()
    ev = np.repeat(empty, np.diff(C_.o.off))
    Ag, Bg = A_.up(ctx, A), B_.up(ctx, B)
    for prec in (cq.CQ_FP64, cq.CQ_SPLIT_BF16X3):
        for beta in (0.0, 1.3):
            ref = O.bsmm(-0.7, A_.o, A, B_.o, B, beta, C_.o, C0.copy())
            Cg = C_.up(ctx, C0)
            ctx.bsmm(-0.7, A_.g, Ag, B_.g, Bg, beta, C_.g, Cg, prec=prec)
            got = C_.down(Cg)
            assert np.array_equal(got[ev], beta * C0[ev]), (prec, beta)
            if prec == cq.CQ_FP64:
                assert_product_close(C_.o, got, ref, 0.7 * scale + beta * np.abs(ref).max())
            else:
                err, _ = block_errors(C_.o, got, ref)
                assert (err[~empty] <= 1e-5 * 0.7 * scale[~empty]).all(), (prec, beta)


def test_split_carries_out_of_range_values_as_nan(ctx):
    """A value beyond the split's range (or infinite, or NaN) in A turns every C value it
    reaches into NaN instead of vanishing: all values the FP64 oracle makes NaN for a NaN
    there, and only values of the same scalar row (the densified tile may also reach blocks
    of that row that the masked product leaves out)."""
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    A_, B_, C_ = (Both(ctx, cell, r) for r in (12.0, 10.0, 22.0))
    A = O.scatter(A_.o, I.random_blocks(cell, 12.0, 1, symmetric=False))
    B = O.scatter(B_.o, I.random_blocks(cell, 10.0, 2, symmetric=False))
    blk = 37                                   # an off-diagonal block of A, its value (1, 2)
    i_atom = int(A_.o.row[blk])
    pos = int(A_.o.off[blk]) + 1 * int(cell.nb[int(A_.o.col[blk])]) + 2
    An = A.copy()
    An[pos] = np.nan
    reach = np.isnan(O.bsmm(1.0, A_.o, An, B_.o, B, 0.0, C_.o))
    assert reach.any()
    # C values of scalar row 1 of atom i_atom (blocks (i_atom, j) of P_C)
    row1 = np.zeros(C_.o.n_values, dtype=bool)
    for b in np.nonzero(C_.o.row == i_atom)[0]:
        nj = int(cell.nb[int(C_.o.col[b])])
        row1[int(C_.o.off[b]) + nj:int(C_.o.off[b]) + 2 * nj] = True
    assert not (reach & ~row1).any()
    Bg = B_.up(ctx, B)
    for bad in (1e300, -np.inf, np.nan):
        Ab = A.copy()
        Ab[pos] = bad
        Cg = ctx.zeros(C_.g)
        ctx.bsmm(1.0, A_.g, A_.up(ctx, Ab), B_.g, Bg, 0.0, C_.g, Cg,
                 prec=cq.CQ_SPLIT_BF16X3)
        got = C_.down(Cg)
        assert np.isnan(got[reach]).all(), bad
        assert np.isfinite(got[~row1]).all(), bad


@pytest.mark.parametrize("species,ranges", [((5, 9, 13), (12.0, 10.0, 22.0)),
                                            ((5, 9, 13), (22.0, 22.0, 12.0)),
                                            ((4, 9), (12.0, 10.0, 12.0)),
                                            ((13,), (12.0, 10.0, 22.0))])
def test_split_parity_mixed_basis(ctx, species, ranges):
    """Atoms of different orbital counts, and uniform counts other than 4 and 9, take the
    mixed path (atom groups of varying slot counts, tails of 1 to 5 values packed into
    16-value tail groups): same error model as the uniform products, on a 216-atom cell
    whose groups and tail groups end ragged."""
    cell = I.mixed_cell((3, 3, 3), 0.05, 0.1, 41, species=species)
    _check_split(ctx, cell, ranges, alpha=-0.7, beta=1.3)


def test_split_lnv_then_fp64_refinement(ctx):
    """Mixed-precision LNV on the 64-atom sp cell tracks the FP64 oracle to FP32-class
    accuracy; FP64 refinement steps then reach the oracle's converged energy."""
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
    for _ in range(40):
        lo.step()
    E_ref = lo.E
    S_g, H_g = upload_pairs(ctx, pS.g, Spb), upload_pairs(ctx, pS.g, Hpb)
    L_g = pL.up(ctx, L0)
    lg = ctx.lnv(pS.g, S_g, H_g, pL.g, L_g, 256.0, prec=cq.CQ_SPLIT_BF16X3)
    for _ in range(25):
        r = lg.step()
    e_mixed = abs(r["energy"] - E_ref) / cell.n_atoms
    assert e_mixed < 1e-5, e_mixed
    lg.set_precision(cq.CQ_FP64)
    for _ in range(15):
        r = lg.step()
    assert abs(r["energy"] - E_ref) / cell.n_atoms < 1e-9
    assert abs(r["n_elec"] - 256.0) < 1e-7


def test_timed_out_wait_is_reported_and_the_next_product_is_clean(ctx):
    """The error path of the tensor-core waits, run for real: with the test hook on, every
    split kernel's first wait is on a barrier that nothing completes and gives up after 2000
    cycles; the CTA retires its issued copies, frees its tensor memory and returns, and the
    next synchronising call reports CQ_ERR_TIMEOUT.  With the hook off again the same
    product on the same context is correct."""
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    A_, B_, C_ = (Both(ctx, cell, r) for r in (12.0, 10.0, 22.0))
    A = O.scatter(A_.o, I.random_blocks(cell, 12.0, 1, symmetric=False))
    B = O.scatter(B_.o, I.random_blocks(cell, 10.0, 2, symmetric=False))
    Ag, Bg = A_.up(ctx, A), B_.up(ctx, B)
    Cg = ctx.zeros(C_.g)
    ctx.set_test_wait(2000)
    try:
        ctx.bsmm(1.0, A_.g, Ag, B_.g, Bg, 0.0, C_.g, Cg, prec=cq.CQ_SPLIT_BF16X3)
        with pytest.raises(cq.CQError) as e:
            ctx.sync()
        assert e.value.status == 6, e.value
    finally:
        ctx.set_test_wait(0)
    ctx.sync()  # the flag was cleared by the report
    ctx.bsmm(1.0, A_.g, Ag, B_.g, Bg, 0.0, C_.g, Cg, prec=cq.CQ_SPLIT_BF16X3)
    ctx.sync()
    ref = O.bsmm(1.0, A_.o, A, B_.o, B, 0.0, C_.o)
    err, _ = block_errors(C_.o, C_.down(Cg), ref)
    scale = natural_scale(A_.o, A, B_.o, B, C_.o)
    assert (err / np.maximum(scale, 1e-300)).max() <= 1e-5
