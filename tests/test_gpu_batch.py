"""Batched heterogeneous cells (cells of different sizes, densities, ranges and mixed 5-, 9-
and 13-orbital species) against the oracle run cell by cell, and against the same cells
solved one at a time on the GPU."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_08941_gb300 import cq
from paper_2205_08941_gb300 import inputs as I

from helpers import block_errors, natural_scale

pytestmark = pytest.mark.gpu

CELLS = [((2, 1, 1), 0.05, 0.10, 31, 8.0), ((2, 2, 1), 0.03, 0.10, 32, 9.0),
         ((1, 2, 2), 0.06, 0.05, 33, 8.5)]


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
def cells():
    out = []
    for shape, dens, sig, seed, rs in CELLS:
        cell = I.mixed_cell(shape, dens, sig, seed)
        S, H = I.overlap_hamiltonian_species(cell, I.silicon_model(rs))
        out.append((cell, S, H, rs))
    return out


class BatchOracle:
    """Per-cell oracle patterns and the map from their values to the batch layout."""

    def __init__(self, ctx, cells, ranges):
        self.cells = cells
        pos, nb, start, boxes = I.concat_cells(cells)
        self.start = start
        dev = "cuda:0"
        self.g = ctx.pattern_batch(torch.tensor(pos, device=dev), start, boxes,
                                   torch.tensor(nb, dtype=torch.int32, device=dev), ranges)
        self.o = [O.Pattern.of_cell(c, r) for c, r in zip(cells, ranges)]
        rp, col, off, tr = self.g.export()
        rp, col, off = rp.cpu().numpy(), col.cpu().numpy(), off.cpu().numpy()
        self.idx = []
        for c, po in enumerate(self.o):
            a0, a1 = start[c], start[c + 1]
            b0, b1 = rp[a0], rp[a1]
            assert np.array_equal(rp[a0:a1 + 1] - b0, po.rp)
            assert np.array_equal(col[b0:b1] - a0, po.col)
            sizes = np.diff(po.off)
            self.idx.append(np.repeat(off[b0:b1] - po.off[:-1], sizes) + np.arange(po.off[-1]))
        self.n_values = self.g.n_values

    def up(self, per_cell):
        out = np.zeros(self.n_values)
        for ix, v in zip(self.idx, per_cell):
            out[ix] = v
        return torch.tensor(out, device="cuda:0")

    def down(self, t):
        a = t.cpu().numpy()
        return [a[ix] for ix in self.idx]


def _ranges(cells, extra):
    return [c[3] + extra for c in cells]


def test_batch_patterns_match_cellwise_oracle(ctx, cells):
    cl = [c[0] for c in cells]
    for extra in (0.0, 2.0, 12.0):
        BatchOracle(ctx, cl, _ranges(cells, extra))  # asserts inside


def test_batch_product_matches_cellwise_oracle(ctx, cells):
    cl = [c[0] for c in cells]
    A_ = BatchOracle(ctx, cl, _ranges(cells, 2.0))
    B_ = BatchOracle(ctx, cl, _ranges(cells, 0.0))
    C_ = BatchOracle(ctx, cl, [r + r0 for r, r0 in zip(_ranges(cells, 2.0), _ranges(cells, 0.0))])
    As = [O.scatter(po, I.random_blocks(c, r, 10 + k, symmetric=False))
          for k, (c, po, r) in enumerate(zip(cl, A_.o, _ranges(cells, 2.0)))]
    Bs = [O.scatter(po, I.random_blocks(c, r, 20 + k, symmetric=False))
          for k, (c, po, r) in enumerate(zip(cl, B_.o, _ranges(cells, 0.0)))]
    Cg = torch.zeros(C_.n_values, dtype=torch.float64, device="cuda:0")
    ctx.bsmm(1.0, A_.g, A_.up(As), B_.g, B_.up(Bs), 0.0, C_.g, Cg)
    for k, got in enumerate(C_.down(Cg)):
        ref = O.bsmm(1.0, A_.o[k], As[k], B_.o[k], Bs[k], 0.0, C_.o[k])
        err, nrm = block_errors(C_.o[k], got, ref)
        scale = natural_scale(A_.o[k], As[k], B_.o[k], Bs[k], C_.o[k])
        assert np.all(err <= 1e-12 * np.maximum(nrm, 1e-3 * scale))
    # per-cell traces
    t = [ctx.trace_prod(A_.g, A_.up(As), A_.g, A_.up(As))]
    ref = sum(O.trace_prod(A_.o[k], As[k], A_.o[k], As[k]) for k in range(len(cl)))
    assert t[0] == pytest.approx(ref, rel=1e-12)


def test_batch_split_product_matches_cellwise_oracle(ctx, cells):
    """Split-BF16 products on the batch (mixed 5/9/13-orbital species, cells of different
    sizes) against the FP64 oracle cell by cell, to the split's error model: every block
    within 1e-5 of sum_k ||A_ik|| ||B_kj||, RMS 1e-6 (tests/test_gpu_split.py)."""
    cl = [c[0] for c in cells]
    A_ = BatchOracle(ctx, cl, _ranges(cells, 2.0))
    B_ = BatchOracle(ctx, cl, _ranges(cells, 0.0))
    C_ = BatchOracle(ctx, cl, [r + r0 for r, r0 in zip(_ranges(cells, 2.0), _ranges(cells, 0.0))])
    As = [O.scatter(po, I.random_blocks(c, r, 10 + k, symmetric=False))
          for k, (c, po, r) in enumerate(zip(cl, A_.o, _ranges(cells, 2.0)))]
    Bs = [O.scatter(po, I.random_blocks(c, r, 20 + k, symmetric=False))
          for k, (c, po, r) in enumerate(zip(cl, B_.o, _ranges(cells, 0.0)))]
    Cs = [O.scatter(po, I.random_blocks(c, r, 30 + k, symmetric=False))
          for k, (c, po, r) in enumerate(zip(cl, C_.o, [x + y for x, y in zip(
              _ranges(cells, 2.0), _ranges(cells, 0.0))]))]
    Cg = C_.up(Cs)
    ctx.bsmm(-0.7, A_.g, A_.up(As), B_.g, B_.up(Bs), 1.3, C_.g, Cg, prec=cq.CQ_SPLIT_BF16X3)
    for k, got in enumerate(C_.down(Cg)):
        ref = O.bsmm(-0.7, A_.o[k], As[k], B_.o[k], Bs[k], 1.3, C_.o[k], Cs[k].copy())
        err, _ = block_errors(C_.o[k], got, ref)
        rel = err / np.maximum(0.7 * natural_scale(A_.o[k], As[k], B_.o[k], Bs[k], C_.o[k]),
                               1e-300)
        assert rel.max() <= 1e-5, (k, rel.max())
        assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, k


def _oracle_cell_lnv(cell, Spb, Hpb, rs, steps):
    rl = rs + 2.0
    pS, pL = O.Pattern.of_cell(cell, rs), O.Pattern.of_cell(cell, rl)
    pX, pU = O.Pattern.of_cell(cell, rl + rs), O.Pattern.of_cell(cell, 2 * rs + rl)
    S, H = O.scatter(pS, Spb), O.scatter(pS, Hpb)
    T = O.hotelling_init(pS, S, pL)
    for _ in range(10):
        T, _ = O.hotelling_step(pS, S, pL, T, pX)
    n_occ = 2.0 * cell.n_atoms
    L0 = O.pm_guess(pS, S, H, pL, T, pX, pL, n_occ)
    lnv = O.LNV(pS, S, H, pL, L0, 2 * n_occ, pX, pU)
    hist = [lnv.step() for _ in range(steps)]
    return L0, lnv, hist


def test_batch_lnv_matches_cellwise_oracle(ctx, cells):
    cl = [c[0] for c in cells]
    rs = [c[3] for c in cells]
    pS = BatchOracle(ctx, cl, rs)
    pL = BatchOracle(ctx, cl, [r + 2.0 for r in rs])
    S_g = pS.up([O.scatter(po, c[1]) for po, c in zip(pS.o, cells)])
    H_g = pS.up([O.scatter(po, c[2]) for po, c in zip(pS.o, cells)])
    T_g = torch.zeros(pL.n_values, dtype=torch.float64, device="cuda:0")
    ctx.hotelling_init(pS.g, S_g, pL.g, T_g)
    for _ in range(10):
        ctx.hotelling_step(pS.g, S_g, pL.g, T_g)
    n_occ = [2.0 * c.n_atoms for c in cl]
    L_g = torch.zeros(pL.n_values, dtype=torch.float64, device="cuda:0")
    ctx.pm_guess_cells(pS.g, S_g, H_g, pL.g, T_g, pL.g, L_g, n_occ)
    steps = 8
    refs = [_oracle_cell_lnv(c[0], c[1], c[2], c[3], steps) for c in cells]
    # the PM start per cell matches the oracle's
    for k, got in enumerate(pL.down(L_g)):
        err, nrm = block_errors(pL.o[k], got, refs[k][0])
        assert err.max() < 1e-11 * max(nrm.max(), 1.0)
    lg = ctx.lnv_cells(pS.g, S_g, H_g, pL.g, L_g, [2 * x for x in n_occ])
    for s in range(steps):
        reps = lg.step()
        for k in range(len(cl)):
            ro = refs[k][2][s]
            assert reps[k]["energy"] == pytest.approx(ro["E"], abs=1e-10 * cl[k].n_atoms), (s, k)
            assert (reps[k]["restart"], reps[k]["fallback"], reps[k]["n_corr"]) == (
                int(ro["restart"]), int(ro["fallback"]), ro["n_corr"]), (s, k)


def test_batch_split_lnv_tracks_cellwise_oracle(ctx, cells):
    """Batched LNV with split-BF16 products (mixed species) follows the FP64 oracle run cell
    by cell: every cell's energy within 2e-5 Ha/atom of the oracle's at each of 8 steps (the
    split's FP32-class product error), and its electron count within 1e-5 relative."""
    cl = [c[0] for c in cells]
    rs = [c[3] for c in cells]
    pS = BatchOracle(ctx, cl, rs)
    pL = BatchOracle(ctx, cl, [r + 2.0 for r in rs])
    S_g = pS.up([O.scatter(po, c[1]) for po, c in zip(pS.o, cells)])
    H_g = pS.up([O.scatter(po, c[2]) for po, c in zip(pS.o, cells)])
    T_g = torch.zeros(pL.n_values, dtype=torch.float64, device="cuda:0")
    ctx.hotelling_init(pS.g, S_g, pL.g, T_g)
    for _ in range(10):
        ctx.hotelling_step(pS.g, S_g, pL.g, T_g)
    n_occ = [2.0 * c.n_atoms for c in cl]
    L_g = torch.zeros(pL.n_values, dtype=torch.float64, device="cuda:0")
    ctx.pm_guess_cells(pS.g, S_g, H_g, pL.g, T_g, pL.g, L_g, n_occ)
    steps = 8
    refs = [_oracle_cell_lnv(c[0], c[1], c[2], c[3], steps) for c in cells]
    lg = ctx.lnv_cells(pS.g, S_g, H_g, pL.g, L_g, [2 * x for x in n_occ],
                       prec=cq.CQ_SPLIT_BF16X3)
    for s in range(steps):
        reps = lg.step()
        for k in range(len(cl)):
            ro = refs[k][2][s]
            assert abs(reps[k]["energy"] - ro["E"]) <= 2e-5 * cl[k].n_atoms, (s, k)
            assert abs(reps[k]["n_elec"] - 2 * n_occ[k]) <= 1e-5 * 2 * n_occ[k], (s, k)


def test_batch_equals_cells_solved_alone(ctx, cells):
    cl = [c[0] for c in cells]
    rs = [c[3] for c in cells]
    pS = BatchOracle(ctx, cl, rs)
    pL = BatchOracle(ctx, cl, [r + 2.0 for r in rs])
    Ss = [O.scatter(po, c[1]) for po, c in zip(pS.o, cells)]
    Hs = [O.scatter(po, c[2]) for po, c in zip(pS.o, cells)]
    Ls = [O.scatter(po, I.random_blocks(c, r + 2.0, 50 + k)) * 0.02
          for k, (c, po, r) in enumerate(zip(cl, pL.o, rs))]
    L_b = pL.up(Ls)
    lb = ctx.lnv_cells(pS.g, pS.up(Ss), pS.up(Hs), pL.g, L_b, [4.0 * c.n_atoms for c in cl])
    rb = [lb.step() for _ in range(3)]
    for k, (cell, r) in enumerate(zip(cl, rs)):
        dev = "cuda:0"
        pos = torch.tensor(cell.pos, device=dev)
        nb = torch.tensor(cell.nb, dtype=torch.int32, device=dev)
        qS, qL = ctx.pattern(pos, cell.box, nb, r), ctx.pattern(pos, cell.box, nb, r + 2.0)

        def single(q, po, vals):
            rp, col, off, _ = q.export()
            ix = np.repeat(off.cpu().numpy() - po.off[:-1], np.diff(po.off)) + np.arange(po.off[-1])
            t = torch.zeros(q.n_values, dtype=torch.float64, device=dev)
            t[torch.tensor(ix, device=dev)] = torch.tensor(vals, device=dev)
            return t

        L1 = single(qL, pL.o[k], Ls[k])
        l1 = ctx.lnv(qS, single(qS, pS.o[k], Ss[k]), single(qS, pS.o[k], Hs[k]), qL, L1,
                     4.0 * cell.n_atoms)
        for s in range(3):
            r1 = l1.step()
            assert r1["energy"] == pytest.approx(rb[s][k]["energy"], rel=1e-13), (k, s)
            assert r1["n_corr"] == rb[s][k]["n_corr"]
        l1.close()
