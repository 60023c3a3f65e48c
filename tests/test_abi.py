"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/*.h.

No compute call is made here (this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cq_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libcq():
    from paper_2205_08941_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("cq_pattern_build", "cq_bsmm", "cq_trace_prod", "cq_lnv_step",
                     "cq_hotelling_step", "cq_dot", "cq_lnv_create", "cq_pm_guess",
                     "cq_mcweeny_step", "cq_pattern_scatter"):
        assert required in names


def test_library_exports_every_declared_symbol(libcq):
    missing = [n for n in declared_functions() if not hasattr(libcq, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2205_08941_gb300 import cq
    missing = [n for n in declared_functions() if n not in cq.SIGNATURES]
    assert not missing, missing


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: a missing libcq.so is an error at the first call."""
    from paper_2205_08941_gb300 import cq
    monkeypatch.setattr(cq, "LIB_PATH", str(tmp_path / "libcq.so"))
    monkeypatch.setattr(cq, "_lib", None)
    with pytest.raises(ImportError, match="missing"):
        cq.lib()


def test_context_creation_without_a_gpu_is_an_error(libcq):
    """Without a usable device the library reports CQ_ERR_CUDA (and leaves *out null); it
    never computes on the host instead."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    libcq.cq_ctx_create.restype = ctypes.c_int
    libcq.cq_ctx_create.argtypes = [ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p(1)
    assert libcq.cq_ctx_create(0, None, ctypes.byref(h)) == 4   # CQ_ERR_CUDA
    assert not h.value
    assert libcq.cq_ctx_create(0, None, None) == 1               # CQ_ERR_INVALID
