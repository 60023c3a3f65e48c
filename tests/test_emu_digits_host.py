"""The digit planes of the emulated-FP64 product, built for the host from the same header
the packing kernels use, checked on the CPU against what the construction fixes.

For a group exponent E with |x| < 2^E the eight planes f_p = d_p 2^(-8p) must hold
integers |d_p| <= 128 (exact in BF16), and 2^(E - 7) sum_p f_p must equal x rounded to the
grid 2^(E - 63) -- checked exactly, in integers: round(x 2^(63 - E)) against
sum_p d_p 2^(8 (7 - p)).  So |x - reconstruction| <= 2^(E - 64).  Zero gives zero planes;
infinities and NaNs give a NaN first plane (the group is poisoned); the exponent is the
smallest E with |x| < 2^E, subnormals included.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "emu_digits_host.cu")
HDR = os.path.join(os.path.dirname(HERE), "paper_2205_08941_gb300", "csrc", "emu_digits.cuh")
EXE = os.path.join(HERE, "_build", "emu_digits_host")
OWN = 99999
P = 8


@pytest.fixture(scope="module")
def digits():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    stale = not os.path.exists(EXE) or any(os.path.getmtime(f) > os.path.getmtime(EXE)
                                           for f in (SRC, HDR))
    if stale:
        os.makedirs(os.path.dirname(EXE), exist_ok=True)
        subprocess.run([nvcc, "-O2", "-std=c++17", SRC, "-o", EXE], check=True,
                       capture_output=True)

    def run(x, E):
        rec = np.zeros(len(x), dtype=[("x", "<f8"), ("E", "<i4")])
        rec["x"], rec["E"] = x, E
        out = subprocess.run([EXE], input=rec.tobytes(), capture_output=True, check=True).stdout
        o = np.frombuffer(out, dtype=[("E", "<i4"), ("f", "<f4", (P,))])
        return o["E"].astype(np.int64), o["f"].astype(np.float64)

    return run


def _exact_check(x, E, f):
    """Integers: d_p = f_p 2^(8p); sum_p d_p 2^(8(7-p)) == round(x 2^(63-E)) (ties away)."""
    for xi, Ei, fi in zip(x, E, f):
        d = [int(Fraction(float(fi[p])) * 2 ** (8 * p)) for p in range(P)]
        assert all(Fraction(float(fi[p])) * 2 ** (8 * p) == d[p] for p in range(P))
        assert all(abs(v) <= 128 for v in d), d
        Y = sum(v * 2 ** (8 * (P - 1 - p)) for p, v in enumerate(d))
        t = Fraction(float(xi)) * Fraction(2) ** (63 - int(Ei))
        r = int(abs(t) + Fraction(1, 2))           # round half away from zero
        r = -r if t < 0 else r
        assert Y == r, (xi, Ei, Y, r)
        err = abs(Fraction(float(xi)) - Fraction(2) ** (int(Ei) - 63) * Y)
        assert err <= Fraction(2) ** (int(Ei) - 64)


def test_exponent_is_the_smallest_bound(digits):
    rng = np.random.default_rng(1)
    x = np.ldexp(1.0 + rng.random(500), rng.integers(-1070, 1020, 500)) * rng.choice([-1, 1], 500)
    x = np.concatenate([x, [1.0, 0.5, 2.0 ** -1074, 3 * 2.0 ** -1074, 2.0 ** -1022,
                            np.nextafter(1.0, 0.0), 1.5]])
    E, _ = digits(x, np.full(x.size, OWN))
    for xi, e in zip(x, E):
        assert abs(xi) < 2.0 ** int(e) and abs(xi) >= 2.0 ** (int(e) - 1), (xi, e)


def test_digits_reconstruct_the_rounded_value_exactly(digits):
    rng = np.random.default_rng(2)
    n = 3000
    x = np.ldexp(1.0 + rng.random(n), rng.integers(-60, 60, n)) * rng.choice([-1, 1], n)
    own, _ = digits(x, np.full(n, OWN))
    E = own + rng.integers(0, 70, n)  # the group maximum may lie far above the value
    E2, f = digits(x, E)
    assert np.array_equal(E, E2)
    _exact_check(x, E, f)


def test_extremes_of_the_digit_range(digits):
    # values at the top of the group (|x| just below 2^E), exact digits, subnormals
    E = np.array([0, 0, 0, 0, 5, -1020, -1030, 3])
    x = np.array([np.nextafter(1.0, 0.0), -np.nextafter(1.0, 0.0), 0.5 + 2.0 ** -30,
                  -(2.0 ** -55) * 3, 17.25, 2.0 ** -1074, 5 * 2.0 ** -1074, 0.0])
    Eo, f = digits(x, E)
    _exact_check(x, Eo, f)
    assert np.all(f[-1] == 0.0)


def test_non_finite_values_poison_the_group(digits):
    x = np.array([np.inf, -np.inf, np.nan])
    E, f = digits(x, np.full(3, OWN))
    assert np.all(E == 32767)
    assert np.all(np.isnan(f[:, 0])) and np.all(f[:, 1:] == 0.0)
    Ez, fz = digits(np.array([0.0, -0.0]), np.full(2, OWN))
    assert np.all(Ez == -32768) and np.all(fz == 0.0)
