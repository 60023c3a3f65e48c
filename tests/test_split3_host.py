"""The split-BF16 operand split (three BF16 terms per FP64 value), built for the host from
the same header the packing kernels use and checked against its error bounds on the CPU.

The bounds follow from the construction: a 24-bit FP32 head h, the 29 cut-off bits as an
FP32 tail l (present when its scale 2^(e - 52) is a normal FP32 number, i.e. |x| >= 2^-74),
b0 = bf16(h), b1 = bf16(h - b0), b2 = bf16(h - b0 - b1 + l); each BF16 rounding is at most
2^-8 of its argument.  So for 2^-74 <= |x| < X_max = (2 - 2^-8) 2^127 the error is at most
2^-25 |x|; without the tail at most 2^-22 |x| (2^-109 <= |x| < 2^-74); where the later
terms are BF16 subnormals at most 2^-8 |x| (down to 2^-126); below that all terms are zero;
from X_max on (b0 rounds to infinity), and for infinities and NaNs, the terms sum to NaN.
The split is odd in x, and BF16 values split exactly.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "split3_host.cu")
HDR = os.path.join(os.path.dirname(HERE), "paper_2205_08941_gb300", "csrc", "split3.cuh")
EXE = os.path.join(HERE, "_build", "split3_host")


@pytest.fixture(scope="module")
def split():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    stale = not os.path.exists(EXE) or any(os.path.getmtime(f) > os.path.getmtime(EXE)
                                           for f in (SRC, HDR))
    if stale:
        os.makedirs(os.path.dirname(EXE), exist_ok=True)
        subprocess.run([nvcc, "-O2", "-std=c++17", SRC, "-o", EXE], check=True,
                       capture_output=True)

    def run(x):
        x = np.ascontiguousarray(x, dtype="<f8")
        out = subprocess.run([EXE], input=x.tobytes(), capture_output=True, check=True).stdout
        return np.frombuffer(out, dtype="<f4").reshape(-1, 3).astype(np.float64)

    return run


def _random(rng, n, lo, hi):
    """Doubles with uniformly random exponents in [lo, hi), random 52-bit significands and
    random signs."""
    frac = rng.integers(0, 1 << 52, size=n, dtype=np.int64).astype(np.float64) / 2.0 ** 52
    x = np.ldexp(1.0 + frac, rng.integers(lo, hi, size=n))
    return np.where(rng.random(n) < 0.5, -x, x)


def test_error_bound_over_the_fp32_range(split):
    x = _random(np.random.default_rng(1), 200_000, -74, 127)
    b = split(x)
    rel = np.abs(x - b.sum(axis=1)) / np.abs(x)   # the three terms sum exactly in FP64
    assert rel.max() <= 2.0 ** -25, rel.max()
    assert np.sqrt(np.mean(rel ** 2)) <= 2.0 ** -26
    # b1 is the rounding error of b0 (at most 2^-8 |b0|); b2 that of b1 plus the tail
    # (|l| < 2^-23 |x|), with one FP32 and one BF16 rounding on top
    assert np.all(np.abs(b[:, 1]) <= 2.0 ** -8 * np.abs(b[:, 0]))
    assert np.all(np.abs(b[:, 2]) <= (2.0 ** -8 * np.abs(b[:, 1]) + 2.0 ** -23 * np.abs(x))
                  * (1 + 2.0 ** -7))


def test_small_values_drop_the_tail_then_vanish(split):
    rng = np.random.default_rng(2)
    x = _random(rng, 20_000, -109, -74)
    rel = np.abs(x - split(x).sum(axis=1)) / np.abs(x)
    assert rel.max() <= 2.0 ** -22
    x = _random(rng, 20_000, -126, -109)
    rel = np.abs(x - split(x).sum(axis=1)) / np.abs(x)
    assert rel.max() <= 2.0 ** -8 * (1 + 2.0 ** -7)
    tiny = np.concatenate([[0.0, -0.0, 2.0 ** -127, -1e-300, 5e-324],
                           _random(rng, 1000, -1074, -126)])
    assert np.all(split(tiny) == 0.0)


def test_out_of_range_and_non_finite_values_give_nan(split):
    x_max = (2.0 - 2.0 ** -8) * 2.0 ** 127
    bad = np.array([x_max, -x_max, np.nextafter(2.0 ** 128, 0.0), 2.0 ** 128, 1e300,
                    -1.7976931348623157e308, np.inf, -np.inf, np.nan])
    with np.errstate(invalid="ignore"):
        assert np.all(np.isnan(split(bad).sum(axis=1)))
    # just below X_max (the largest BF16 value and a value that rounds down to it) and the
    # smallest FP32 normal stay finite
    ok = np.array([np.nextafter(x_max, 0.0), (2.0 - 2.0 ** -7) * 2.0 ** 127, 2.0 ** -126,
                   -(2.0 ** -126)])
    b = split(ok)
    assert np.all(np.isfinite(b))
    assert np.all(np.abs(ok - b.sum(axis=1)) <= 2.0 ** -8 * np.abs(ok))


def test_odd_and_exact_on_bf16_values(split):
    x = _random(np.random.default_rng(3), 10_000, -60, 60)
    assert np.array_equal(split(-x), -split(x))
    # BF16 values (8-bit significands) are their own first term
    v = np.ldexp(np.random.default_rng(4).integers(128, 256, size=1000) / 128.0,
                 np.random.default_rng(5).integers(-100, 100, size=1000))
    b = split(v)
    assert np.array_equal(b[:, 0], v) and np.all(b[:, 1:] == 0.0)
