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
