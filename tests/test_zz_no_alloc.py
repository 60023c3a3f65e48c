"""The allocation-free trace (cq_trace_prod_static) against cq_trace_prod.

Callers that cannot allocate device memory when they need a trace -- code under a
framework-owned memory budget, loops that must not pay for cudaMalloc, or callers that no
longer hold the context that built their patterns -- use the static variant, whose scratch
is a fixed device array.  It must give the same trace as the
allocating entry point (within the trace tolerance of the other tests) on consecutive calls
that share that array, and reject patterns larger than the array.
"""
import numpy as np
import pytest
import torch

from paper_2205_08941_gb300 import cq
from paper_2205_08941_gb300 import inputs as I

from helpers import gpu_pattern, upload_pairs

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


def test_static_trace_matches_trace_prod_on_two_calls(ctx):
    cell = I.diamond_cell(4, a=10.26, sigma=0.1, seed=2, norb=9)
    pA, pB = gpu_pattern(ctx, cell, 16.0), gpu_pattern(ctx, cell, 14.0)
    A = upload_pairs(ctx, pA, I.random_blocks(cell, 16.0, 1, symmetric=False))
    B1 = upload_pairs(ctx, pB, I.random_blocks(cell, 14.0, 2, symmetric=False))
    B2 = upload_pairs(ctx, pB, I.random_blocks(cell, 14.0, 3, symmetric=False))
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    for B in (B1, B2):  # consecutive calls share the static scratch
        ref = ctx.trace_prod(pA, A, pB, B)
        cq.trace_prod_static(pA, A, pB, B, out)
        torch.cuda.synchronize()
        assert float(out.item()) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_static_trace_rejects_patterns_beyond_its_scratch(ctx):
    n = 65537
    rng = np.random.default_rng(0)
    box = np.array([200.0, 200.0, 200.0])
    cell = I.Cell(pos=rng.random((n, 3)) * box, box=box, nb=np.ones(n, dtype=np.int32))
    p = gpu_pattern(ctx, cell, 0.0)
    A = ctx.zeros(p)
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    with pytest.raises(cq.CQError) as e:
        cq.trace_prod_static(p, A, p, A, out)
    assert e.value.status == 1 and "65536" in str(e.value)


def test_static_trace_needs_no_context():
    """Patterns outlive the context that built them; the static trace runs on the device the
    patterns record, with no context at all."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cq.Context(0)
    cell = I.diamond_cell(2, a=10.26, sigma=0.1, seed=4, norb=9)
    pA, pB = gpu_pattern(c, cell, 12.0), gpu_pattern(c, cell, 10.0)
    A = upload_pairs(c, pA, I.random_blocks(cell, 12.0, 5, symmetric=False))
    B = upload_pairs(c, pB, I.random_blocks(cell, 10.0, 6, symmetric=False))
    ref = c.trace_prod(pA, A, pB, B)
    # destroy the C context only; the patterns stay alive
    cq.lib().cq_ctx_destroy(c.h)
    c.h = None
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    for _ in range(2):
        cq.trace_prod_static(pA, A, pB, B, out)
        torch.cuda.synchronize()
        assert float(out.item()) == pytest.approx(ref, rel=1e-12, abs=1e-12)
    pA.close()
    pB.close()
