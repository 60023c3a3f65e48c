"""Block products at the full size the benchmark times (4096-atom Si SZP, 9 orbitals per
atom, S on 14 bohr, L on 16, X on 30), against the oracle on 32 sampled output atom rows
spread over the cell (the oracle computes only those rows).

Two product types of the LNV evaluation in the benchmark's launch configuration: L.S on
P_X (short segments) and X.X on P_L (the long-segment regime of the R products, whose
k-sums run over ~800 blocks).  FP64 to the product tolerance of the other parity tests;
split-BF16 to its error model (per block <= 1e-5 of sum_k ||A_ik|| ||B_kj||, RMS <= 1e-6).
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
    if prec == cq.CQ_FP64:
        assert_product_close(C_.o, got, ref, scale, rows=ROWS)
        return
    err, _ = block_errors(C_.o, got, ref)
    sel = np.isin(C_.o.row, ROWS)
    rel = err[sel] / np.maximum(scale[sel], 1e-300)
    assert rel.max() <= 1e-5, rel.max()
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, np.sqrt(np.mean(rel ** 2))


@pytest.mark.parametrize("prec", [cq.CQ_FP64, cq.CQ_SPLIT_BF16X3])
def test_fullsize_l_times_s_on_p_x(data, prec):
    _check(data, 16.0, 14.0, 30.0, prec)


@pytest.mark.parametrize("prec", [cq.CQ_FP64, cq.CQ_SPLIT_BF16X3])
def test_fullsize_x_times_x_on_p_l(data, prec):
    _check(data, 30.0, 30.0, 16.0, prec)
