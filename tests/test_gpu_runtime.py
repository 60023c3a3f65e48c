"""Runtime features: CUDA-graph replay of LNV phases and the FP64 lane-split autotuner."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_08941_gb300 import cq
from paper_2205_08941_gb300 import inputs as I

from helpers import (assert_product_close, from_oracle, gpu_pattern, layout_index,
                     natural_scale, to_oracle, upload_pairs)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08941_gb300 import build
    build.build()


def _si64_lnv(ctx, steps, graphs):
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    Spb, Hpb = I.overlap_hamiltonian(cell, I.silicon_model(10.0))
    pS, pL = gpu_pattern(ctx, cell, 10.0), gpu_pattern(ctx, cell, 12.0)
    S, H = upload_pairs(ctx, pS, Spb), upload_pairs(ctx, pS, Hpb)
    torch.cuda.synchronize()
    T = ctx.zeros(pL)
    torch.cuda.synchronize()
    ctx.hotelling_init(pS, S, pL, T)
    for _ in range(10):
        ctx.hotelling_step(pS, S, pL, T)
    L = ctx.zeros(pL)
    torch.cuda.synchronize()
    ctx.pm_guess(pS, S, H, pL, T, pL, L, 128.0)
    ctx.set_graphs(graphs)
    lnv = ctx.lnv(pS, S, H, pL, L, 256.0)
    n0 = cq.kernel_launches()
    reps = [lnv.step() for _ in range(steps)]
    return reps, cq.kernel_launches() - n0


def test_graph_replay_matches_eager_bitwise(built):
    a = cq.Context(0, stream=torch.cuda.Stream())
    b = cq.Context(0, stream=torch.cuda.Stream())
    eager, _ = _si64_lnv(a, 6, False)
    graphed, launches = _si64_lnv(b, 6, True)
    for re, rg in zip(eager, graphed):
        assert re == rg
    assert launches > 0
    a.close()
    b.close()


def test_graphs_need_a_created_stream(built):
    c = cq.Context(0)  # torch's default stream
    with pytest.raises(cq.CQError) as e:
        c.set_graphs(True)
    assert e.value.status == 1
    c.close()


def test_autotuner_picks_a_split_and_keeps_parity(built):
    ctx = cq.Context(0)
    ctx.set_autotune(True)
    cell = I.diamond_cell(4, a=10.26, sigma=0.1, seed=2, norb=9)
    ranges = (30.0, 30.0, 16.0)
    po = [O.Pattern.of_cell(cell, r) for r in ranges]
    pg = [gpu_pattern(ctx, cell, r) for r in ranges]
    idx = [layout_index(g, o) for g, o in zip(pg, po)]
    A = O.scatter(po[0], I.random_blocks(cell, ranges[0], 6, symmetric=False))
    B = O.scatter(po[1], I.random_blocks(cell, ranges[1], 7, symmetric=False))
    Cg = ctx.empty(pg[2])
    ctx.bsmm(1.0, pg[0], from_oracle(ctx, pg[0], idx[0], A), pg[1],
             from_oracle(ctx, pg[1], idx[1], B), 0.0, pg[2], Cg)
    q, tuned = ctx.bsmm_config(*pg)
    assert tuned and q in (1, 2, 4, 8, 16, 32)
    rows = np.arange(0, cell.n_atoms, 41, dtype=np.int32)
    ref = O.bsmm(1.0, po[0], A, po[1], B, 0.0, po[2], rows=rows)
    assert_product_close(po[2], to_oracle(Cg, idx[2]), ref,
                         natural_scale(po[0], A, po[1], B, po[2], rows=rows), rows=rows)
    ctx.close()


def test_release_cache_mid_run_changes_nothing(built):
    """Dropping every cached task list, plan and scratch buffer between LNV steps (with graph
    replay on) gives bitwise the same steps as a run that keeps them, and frees memory."""
    def run(release):
        c = cq.Context(0, stream=torch.cuda.Stream())
        cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
        Spb, Hpb = I.overlap_hamiltonian(cell, I.silicon_model(10.0))
        pS, pL = gpu_pattern(c, cell, 10.0), gpu_pattern(c, cell, 12.0)
        S, H = upload_pairs(c, pS, Spb), upload_pairs(c, pS, Hpb)
        torch.cuda.synchronize()
        T = c.zeros(pL)
        torch.cuda.synchronize()
        c.hotelling_init(pS, S, pL, T)
        for _ in range(10):
            c.hotelling_step(pS, S, pL, T)
        L = c.zeros(pL)
        torch.cuda.synchronize()
        c.pm_guess(pS, S, H, pL, T, pL, L, 128.0)
        c.set_graphs(True)
        lnv = c.lnv(pS, S, H, pL, L, 256.0)
        out = []
        for k in range(6):
            if release and k == 3:
                before = c.mem_used()
                c.release_cache()
                assert c.mem_used() < before
            r = lnv.step()
            out.append((r["energy"], r["n_elec"], r["alpha"], r["n_corr"]))
        lnv.close()
        c.close()
        return out

    assert run(True) == run(False)
