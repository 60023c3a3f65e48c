"""Test-side plumbing: move seeded inputs onto both paths and compare their values.

Both the CUDA library and the oracle store blocks in (i, j) order on identical patterns; the
CUDA layout pads odd-sized blocks to an even length, the oracle's does not.  The index maps
below only reorder memory; no arithmetic of the method happens here.
"""
import numpy as np
import torch

import oracle as O
from paper_2205_08941_gb300 import cq


def dev_cell(cell, device="cuda:0"):
    pos = torch.tensor(cell.pos, dtype=torch.float64, device=device)
    nb = torch.tensor(cell.nb, dtype=torch.int32, device=device)
    return pos, nb


def gpu_pattern(ctx, cell, r):
    pos, nb = dev_cell(cell)
    return ctx.pattern(pos, cell.box, nb, r)


def upload_pairs(ctx, p, pb):
    dev = "cuda:0"
    i = torch.tensor(pb.i, dtype=torch.int32, device=dev)
    j = torch.tensor(pb.j, dtype=torch.int32, device=dev)
    off = torch.tensor(pb.off, dtype=torch.int64, device=dev)
    v = torch.tensor(pb.values, dtype=torch.float64, device=dev)
    return ctx.scatter(p, i, j, off, v)


def layout_index(pg, po: O.Pattern):
    """Index into the CUDA value array for every value of the oracle layout (same blocks)."""
    rp, col, off, tr = pg.export()
    assert np.array_equal(rp.cpu().numpy(), po.rp)
    assert np.array_equal(col.cpu().numpy(), po.col)
    sizes = np.diff(po.off)
    idx = np.repeat(off.cpu().numpy() - po.off[:-1], sizes) + np.arange(int(po.off[-1]))
    return torch.tensor(idx, dtype=torch.int64, device="cuda:0")


def to_oracle(values: torch.Tensor, idx: torch.Tensor) -> np.ndarray:
    return values[idx].cpu().numpy()


def from_oracle(ctx, pg, idx, vals: np.ndarray) -> torch.Tensor:
    out = ctx.zeros(pg)
    out[idx] = torch.tensor(vals, dtype=torch.float64, device="cuda:0")
    return out


def block_errors(po: O.Pattern, got: np.ndarray, ref: np.ndarray):
    """Per-block Frobenius norms of (got - ref) and of ref."""
    sizes = np.diff(po.off)
    blk = np.repeat(np.arange(po.nnzb), sizes)
    err = np.sqrt(np.bincount(blk, weights=(got - ref) ** 2, minlength=po.nnzb))
    nrm = np.sqrt(np.bincount(blk, weights=ref ** 2, minlength=po.nnzb))
    return err, nrm


def block_norms(po: O.Pattern, vals: np.ndarray) -> np.ndarray:
    sizes = np.diff(po.off)
    blk = np.repeat(np.arange(po.nnzb), sizes)
    return np.sqrt(np.bincount(blk, weights=vals ** 2, minlength=po.nnzb))


def natural_scale(pA, A, pB, B, pC, rows=None):
    """sum_k ||A_ik||_F ||B_kj||_F per C block: the product of block-norm matrices, computed
    by the oracle on patterns with one orbital per atom."""
    ones = lambda p: O.Pattern(p.pos, p.box, np.ones(p.n, dtype=np.int32), p.range)
    qa, qb, qc = ones(pA), ones(pB), ones(pC)
    return O.bsmm(1.0, qa, block_norms(pA, A), qb, block_norms(pB, B), 0.0, qc, rows=rows)


def assert_product_close(pC, got, ref, scale, rel=1e-12, rows=None):
    """The per-block bound of the product: ||dC_ij|| <= rel * max(||C_ij||, 1e-3 sum_k
    ||A_ik|| ||B_kj||)."""
    err, nrm = block_errors(pC, got, ref)
    bound = rel * np.maximum(nrm, 1e-3 * scale)
    if rows is not None:
        sel = np.isin(pC.row, rows)
        err, bound = err[sel], bound[sel]
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, (bad[:5], err[bad[:5]], bound[bad[:5]])
    return float((err / np.maximum(bound / rel, 1e-300)).max()) if err.size else 0.0
