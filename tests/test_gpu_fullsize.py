"""Block products at the full size the benchmark times (4096-atom Si SZP, 9 orbitals per
atom, S on 14 bohr, L on 16, X on 30), against the oracle on 32 sampled output atom rows
spread over the cell (the oracle computes only those rows).

The product types of the LNV evaluation in the benchmark's launch configuration: L.S on
P_X (short segments), X.X on P_L (the long-segment regime of the R products, whose k-sums
run over ~800 blocks), and the two 44-bohr products that dominate the step: S.X on P_U
(r_U = 44, 10.5M output blocks) and U.Y back onto P_L, with U the oracle's S.X on the
sampled rows (zero elsewhere: a C row of U.Y needs only the same row of U).  FP64 and
emulated FP64 to the product tolerance of the other parity tests; split-BF16 to its error
model (per block <= 1e-5 of sum_k ||A_ik|| ||B_kj||, RMS <= 1e-6).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_08941_gb300 import cq
from paper_2205_08941_gb300 import inputs as I

from helpers import (assert_product_close, block_errors, from_oracle, gpu_pattern,
                     layout_index, natural_scale, to_oracle)

pytestmark = pytest.mark.gpu
ROWS = np.unique(np.linspace(0, 4095, 32).astype(np.int32))


class Both:
    def __init__(self, ctx, cell, r):
        self.o = O.Pattern.of_cell(cell, r)
        self.g = gpu_pattern(ctx, cell, r)
        self.idx = layout_index(self.g, self.o)

    def up(self, ctx, vals):
        return from_oracle(ctx, self.g, self.idx, vals)

    def down(self, t):
        return to_oracle(t, self.idx)


@pytest.fixture(scope="module")
def data():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08941_gb300 import build
    build.build()
    ctx = cq.Context(0)
    cell = I.diamond_cell(8, a=10.26, sigma=0.1, seed=2, norb=9)
    P = {r: Both(ctx, cell, r) for r in (14.0, 16.0, 30.0)}
    vals = {r: O.scatter(P[r].o, I.random_blocks(cell, r, seed, symmetric=False))
            for r, seed in ((14.0, 1), (16.0, 2), (30.0, 3))}
    dev = {r: P[r].up(ctx, vals[r]) for r in P}
    yield ctx, P, vals, dev
    ctx.close()


def _check(data, ra, rb, rc, prec):
    ctx, P, vals, dev = data
    A_, B_, C_ = P[ra], P[rb], P[rc]
    ref = O.bsmm(1.0, A_.o, vals[ra], B_.o, vals[rb], 0.0, C_.o, rows=ROWS)
    Cg = ctx.zeros(C_.g)
    ctx.bsmm(1.0, A_.g, dev[ra], B_.g, dev[rb], 0.0, C_.g, Cg, prec=prec)
    got = C_.down(Cg)
    scale = natural_scale(A_.o, vals[ra], B_.o, vals[rb], C_.o, rows=ROWS)
    if prec in (cq.CQ_FP64, cq.CQ_FP64_EMU):
        assert_product_close(C_.o, got, ref, scale, rows=ROWS)
        return
    err, _ = block_errors(C_.o, got, ref)
    sel = np.isin(C_.o.row, ROWS)
    rel = err[sel] / np.maximum(scale[sel], 1e-300)
    assert rel.max() <= 1e-5, rel.max()
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, np.sqrt(np.mean(rel ** 2))


@pytest.mark.parametrize("prec", [cq.CQ_FP64, cq.CQ_SPLIT_BF16X3, cq.CQ_FP64_EMU])
def test_fullsize_l_times_s_on_p_x(data, prec):
    _check(data, 16.0, 14.0, 30.0, prec)


@pytest.mark.parametrize("prec", [cq.CQ_FP64, cq.CQ_SPLIT_BF16X3, cq.CQ_FP64_EMU])
def test_fullsize_x_times_x_on_p_l(data, prec):
    _check(data, 30.0, 30.0, 16.0, prec)


class Rows:
    """A pattern on both paths with the value indices of the sampled rows only (a full
    index of the 44-bohr pattern would be 850M entries)."""

    def __init__(self, ctx, cell, r, rows):
        self.o = O.Pattern.of_cell(cell, r)
        self.g = gpu_pattern(ctx, cell, r)
        rp, col, off, _ = self.g.export()
        assert np.array_equal(rp.cpu().numpy(), self.o.rp)
        assert np.array_equal(col.cpu().numpy(), self.o.col)
        po = self.o
        blocks = np.concatenate([np.arange(po.rp[i], po.rp[i + 1]) for i in rows])
        sizes = np.diff(po.off)[blocks]
        within = np.arange(int(sizes.sum())) - np.repeat(np.cumsum(sizes) - sizes, sizes)
        self.oidx = np.repeat(po.off[blocks], sizes) + within
        goff = off.cpu().numpy()[blocks]
        self.gidx = torch.tensor(np.repeat(goff, sizes) + within, device="cuda:0")
        self.blocks, self.sizes = blocks, sizes

    def rows_of(self, t):
        return t[self.gidx].cpu().numpy()


def _norms81(v, n_blocks):
    """Block norms of a 9x9-block value array in oracle layout (81 values per block)."""
    out = np.empty(n_blocks)
    step = 1 << 20
    for b0 in range(0, n_blocks, step):
        x = v[81 * b0:81 * min(n_blocks, b0 + step)].reshape(-1, 81)
        out[b0:b0 + x.shape[0]] = np.sqrt(np.einsum("ij,ij->i", x, x))
    return out


def _scale_rows(pA, normA, pB, normB, pC, rows):
    """sum_k ||A_ik|| ||B_kj|| on the sampled rows, by the oracle on one-orbital patterns."""
    ones = lambda p: O.Pattern(p.pos, p.box, np.ones(p.n, dtype=np.int32), p.range)
    return O.bsmm(1.0, ones(pA), normA, ones(pB), normB, 0.0, ones(pC), rows=rows)


def _compare_rows(pC, sel_blocks, sizes, got, ref, scale, prec):
    blk = np.repeat(np.arange(len(sel_blocks)), sizes)
    err = np.sqrt(np.bincount(blk, weights=(got - ref) ** 2, minlength=len(sel_blocks)))
    nrm = np.sqrt(np.bincount(blk, weights=ref ** 2, minlength=len(sel_blocks)))
    sc = scale[sel_blocks]
    if prec in (cq.CQ_FP64, cq.CQ_FP64_EMU):
        bound = 1e-12 * np.maximum(nrm, 1e-3 * sc)
        bad = np.nonzero(err > bound)[0]
        assert bad.size == 0, (bad[:5], err[bad[:5]], bound[bad[:5]])
        return
    rel = err / np.maximum(sc, 1e-300)
    assert rel.max() <= 1e-5, rel.max()
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, np.sqrt(np.mean(rel ** 2))


@pytest.fixture(scope="module")
def u_data(data):
    ctx, P, vals, dev = data
    cell = I.diamond_cell(8, a=10.26, sigma=0.1, seed=2, norb=9)
    P44 = Rows(ctx, cell, 44.0, ROWS)
    # U = S.X on the sampled rows by the oracle (zero elsewhere)
    U_o = O.bsmm(1.0, P[14.0].o, vals[14.0], P[30.0].o, vals[30.0], 0.0, P44.o, rows=ROWS)
    n14, n30 = _norms81(vals[14.0], P[14.0].o.nnzb), _norms81(vals[30.0], P[30.0].o.nnzb)
    yield P44, U_o, n14, n30


@pytest.mark.parametrize("prec", [cq.CQ_FP64, cq.CQ_SPLIT_BF16X3, cq.CQ_FP64_EMU])
def test_fullsize_s_times_x_on_p_u(data, u_data, prec):
    ctx, P, vals, dev = data
    P44, U_o, n14, n30 = u_data
    Ug = ctx.zeros(P44.g)
    ctx.bsmm(1.0, P[14.0].g, dev[14.0], P[30.0].g, dev[30.0], 0.0, P44.g, Ug, prec=prec)
    scale = _scale_rows(P[14.0].o, n14, P[30.0].o, n30, P44.o, ROWS)
    _compare_rows(P44.o, P44.blocks, P44.sizes, P44.rows_of(Ug), U_o[P44.oidx], scale, prec)
    del Ug


@pytest.mark.parametrize("prec", [cq.CQ_FP64, cq.CQ_SPLIT_BF16X3, cq.CQ_FP64_EMU])
def test_fullsize_u_times_y_on_p_l(data, u_data, prec):
    ctx, P, vals, dev = data
    P44, U_o, n14, n30 = u_data
    Ug = ctx.zeros(P44.g)
    Ug[P44.gidx] = torch.tensor(U_o[P44.oidx], device="cuda:0")
    C_ = P[16.0]
    ref = O.bsmm(1.0, P44.o, U_o, P[30.0].o, vals[30.0], 0.0, C_.o, rows=ROWS)
    Cg = ctx.zeros(C_.g)
    ctx.bsmm(1.0, P44.g, Ug, P[30.0].g, dev[30.0], 0.0, C_.g, Cg, prec=prec)
    got = C_.down(Cg)
    nU = np.zeros(P44.o.nnzb)
    nU[P44.blocks] = np.sqrt(np.bincount(np.repeat(np.arange(len(P44.blocks)), P44.sizes),
                                         weights=U_o[P44.oidx] ** 2,
                                         minlength=len(P44.blocks)))
    scale = _scale_rows(P44.o, nU, P[30.0].o, n30, C_.o, ROWS)
    sel = np.nonzero(np.isin(C_.o.row, ROWS))[0]
    sizes = np.diff(C_.o.off)[sel]
    within = np.arange(int(sizes.sum())) - np.repeat(np.cumsum(sizes) - sizes, sizes)
    oidx = np.repeat(C_.o.off[sel], sizes) + within
    _compare_rows(C_.o, sel, sizes, got[oidx], ref[oidx], scale, prec)
    del Ug
