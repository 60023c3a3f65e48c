"""Pins of the CPU oracle against facts fixed by mathematics or by independent libraries.

Each test checks the oracle against something other than itself: numpy / scipy dense
linear algebra, scipy's periodic k-d tree, closed forms (Hotelling's squared residual,
Palser-Manolopoulos trace), textbook limits (the ground-state projector of a gapped
insulator, McWeeny idempotency), finite differences and the exact-cubic invariant.
The cells are the 64-atom diamond Si cell (sp, 256 orbitals) and a mixed-orbital cell.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl
from scipy.spatial import cKDTree

import oracle as O
from paper_2205_08941_gb300 import inputs as I


@pytest.fixture(scope="module")
def si64():
    cell = I.diamond_cell(2, a=10.26, sigma=0.05, seed=1, norb=4)
    S, H = I.overlap_hamiltonian(cell, I.silicon_model(10.0))
    return cell, S, H


@pytest.fixture(scope="module")
def mixed():
    cell = I.diamond_cell(2, a=10.26, sigma=0.2, seed=7, norb=4)
    rng = np.random.default_rng(11)
    cell.nb = rng.choice(np.array([1, 4, 5, 9], dtype=np.int32), size=cell.n_atoms)
    return cell


def _mask(p):
    return O.to_dense(p, np.ones(p.n_values)) != 0


# ------------------------------------------------------------------ patterns

@pytest.mark.parametrize("r", [3.0, 10.0, 12.0, 16.5])
def test_pattern_matches_periodic_kdtree(si64, r):
    cell = si64[0]
    p = O.Pattern.of_cell(cell, r)
    tree = cKDTree(cell.pos, boxsize=cell.box)
    pairs = tree.query_pairs(r, output_type="ndarray")
    ref = set(map(tuple, pairs.tolist())) | {(j, i) for i, j in pairs.tolist()}
    ref |= {(i, i) for i in range(cell.n_atoms)}
    got = set(zip(p.row.tolist(), p.col.tolist()))
    assert got == ref
    for i in range(p.n):
        cols = p.col[p.rp[i]:p.rp[i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_pattern_count_closed_form():
    # 512-atom cell: pairs per atom -> rho (4/3) pi R^3 once R spans several neighbour shells
    # (R below half the box, so each pair has one image)
    cell = I.diamond_cell(4, a=10.26, sigma=0.1, seed=2, norb=4)
    rho = 8.0 / 10.26 ** 3
    for r in (16.0, 19.0):
        p = O.Pattern.of_cell(cell, r)
        per_atom = p.nnzb / cell.n_atoms
        assert abs(per_atom - (rho * 4.0 / 3.0 * math.pi * r ** 3)) / per_atom < 0.1


def test_pattern_self_only_and_dense(si64):
    cell = si64[0]
    p0 = O.Pattern.of_cell(cell, 1e-3)
    assert p0.nnzb == cell.n_atoms and np.all(p0.row == p0.col)
    pd = O.Pattern.of_cell(cell, 18.0)  # beyond the largest minimum-image distance
    assert pd.nnzb == cell.n_atoms ** 2


# ------------------------------------------------------------------ product

@pytest.mark.parametrize("ranges", [(12.0, 10.0, 22.0), (12.0, 10.0, 12.0), (6.0, 8.0, 5.0)])
def test_bsmm_is_dense_multiply_then_mask(si64, ranges):
    cell = si64[0]
    ra, rb, rc = ranges
    pA, pB, pC = (O.Pattern.of_cell(cell, r) for r in ranges)
    A = O.scatter(pA, I.random_blocks(cell, ra, 1, symmetric=False))
    B = O.scatter(pB, I.random_blocks(cell, rb, 2, symmetric=False))
    C0 = O.scatter(pC, I.random_blocks(cell, rc, 3, symmetric=False))
    C = O.bsmm(-0.7, pA, A, pB, B, 1.3, pC, C0.copy())
    ref = (1.3 * O.to_dense(pC, C0) - 0.7 * O.to_dense(pA, A) @ O.to_dense(pB, B)) * _mask(pC)
    assert np.abs(O.to_dense(pC, C) - ref).max() < 1e-13


def test_bsmm_mixed_orbital_counts(mixed):
    cell = mixed
    pA, pB, pC = (O.Pattern.of_cell(cell, r) for r in (9.0, 7.0, 13.0))
    A = O.scatter(pA, I.random_blocks(cell, 9.0, 4, symmetric=False))
    B = O.scatter(pB, I.random_blocks(cell, 7.0, 5, symmetric=False))
    C = O.bsmm(1.0, pA, A, pB, B, 0.0, pC)
    ref = (O.to_dense(pA, A) @ O.to_dense(pB, B)) * _mask(pC)
    assert np.abs(O.to_dense(pC, C) - ref).max() < 1e-13
    t, f = O.triplets(pA, pB, pC)
    # brute-force triplet count from the boolean patterns
    a = (O.to_dense(pA, np.ones(pA.n_values)) != 0)
    nb = cell.nb
    o = np.concatenate([[0], np.cumsum(nb)])
    ab = np.zeros((cell.n_atoms,) * 2, dtype=bool)
    bb = np.zeros_like(ab)
    cb = np.zeros_like(ab)
    for p_, m in ((pA, ab), (pB, bb), (pC, cb)):
        m[p_.row, p_.col] = True
    trip = (ab.astype(np.int64) @ bb.astype(np.int64)) * cb
    assert t == int(trip.sum())
    fl = 2.0 * np.einsum("ik,kj,ij,i,k,j->", ab.astype(float), bb.astype(float),
                         cb.astype(float), nb.astype(float), nb.astype(float), nb.astype(float))
    assert f == pytest.approx(fl, rel=1e-14)
    assert a.shape[0] == o[-1]


def test_trace_and_gather(mixed):
    cell = mixed
    pA, pB = O.Pattern.of_cell(cell, 9.0), O.Pattern.of_cell(cell, 6.0)
    A = O.scatter(pA, I.random_blocks(cell, 9.0, 8, symmetric=False))
    B = O.scatter(pB, I.random_blocks(cell, 6.0, 9, symmetric=False))
    Ad, Bd = O.to_dense(pA, A), O.to_dense(pB, B)
    assert O.trace_prod(pA, A, pB, B) == pytest.approx(np.trace(Ad @ Bd), rel=1e-13, abs=1e-13)
    G = O.gather(pB, B, pA, transpose=True)
    assert np.abs(O.to_dense(pA, G) - Bd.T * _mask(pA)).max() == 0.0
    assert O.dot(A, A) == pytest.approx(np.sum(Ad * Ad), rel=1e-14)


# ------------------------------------------------------------------ Hotelling

def test_hotelling_residual_squares_and_limit(si64):
    cell, Spb, _ = si64
    pS = O.Pattern.of_cell(cell, 10.0)
    pT = O.Pattern.of_cell(cell, 18.0)   # dense T
    pV = O.Pattern.of_cell(cell, 28.0)
    S = O.scatter(pS, Spb)
    Sd = O.to_dense(pS, S)
    T = O.hotelling_init(pS, S, pT)
    eye = np.eye(Sd.shape[0])
    assert np.abs(O.to_dense(pT, T) - eye / np.abs(Sd).sum(axis=1).max()).max() < 1e-15
    for _ in range(10):
        E_n = eye - Sd @ O.to_dense(pT, T)
        T, r = O.hotelling_step(pS, S, pT, T, pV)
        assert r == pytest.approx(np.linalg.norm(E_n), rel=1e-12)
        E_next = eye - Sd @ O.to_dense(pT, T)
        assert np.linalg.norm(E_next - E_n @ E_n) < 1e-13 * max(1.0, np.linalg.norm(E_n))
    assert np.abs(O.to_dense(pT, T) - sl.inv(Sd)).max() < 1e-12


def test_hotelling_sparse_converges(si64):
    cell, Spb, _ = si64
    pS, pT = O.Pattern.of_cell(cell, 10.0), O.Pattern.of_cell(cell, 12.0)
    pV = O.Pattern.of_cell(cell, 22.0)
    S = O.scatter(pS, Spb)
    T = O.hotelling_init(pS, S, pT)
    res = []
    for _ in range(10):
        T, r = O.hotelling_step(pS, S, pT, T, pV)
        res.append(r)
    assert res[-1] < 0.05 * res[0]
    assert np.allclose(O.to_dense(pT, T), O.to_dense(pT, T).T, atol=1e-14)


# ------------------------------------------------------------------ PM and McWeeny

def _dense_setup(si64):
    cell, Spb, Hpb = si64
    pS = O.Pattern.of_cell(cell, 10.0)
    pD = O.Pattern.of_cell(cell, 18.0)
    S, H = O.scatter(pS, Spb), O.scatter(pS, Hpb)
    return cell, pS, pD, S, H


def test_pm_guess_trace_and_spectrum(si64):
    cell, pS, pD, S, H = _dense_setup(si64)
    T = O.from_dense(pD, sl.inv(O.to_dense(pS, S)))
    L0 = O.pm_guess(pS, S, H, pD, T, pD, pD, 128.0)
    LS = O.to_dense(pD, L0) @ O.to_dense(pS, S)
    assert np.trace(LS) == pytest.approx(128.0, rel=1e-12)
    ev = np.linalg.eigvals(LS).real
    assert ev.min() > -1e-10 and ev.max() < 1.0 + 1e-10


def test_mcweeny_sparse_step_is_masked_formula(si64):
    cell, Spb, _ = si64
    pS, pL = O.Pattern.of_cell(cell, 10.0), O.Pattern.of_cell(cell, 7.0)
    pX, pU, p2L = (O.Pattern.of_cell(cell, r) for r in (17.0, 27.0, 14.0))
    S = O.scatter(pS, Spb)
    L = O.scatter(pL, I.random_blocks(cell, 7.0, 3)) * 0.1
    out = O.mcweeny_step(pS, S, pL, L, pX, pU, p2L)
    Ld, Sd = O.to_dense(pL, L), O.to_dense(pS, S)
    ref = (3 * Ld @ Sd @ Ld - 2 * Ld @ Sd @ Ld @ Sd @ Ld) * _mask(pL)
    assert np.abs(O.to_dense(pL, out) - ref).max() < 1e-13


def test_mcweeny_purifies_to_idempotent(si64):
    cell, pS, pD, S, H = _dense_setup(si64)
    T = O.from_dense(pD, sl.inv(O.to_dense(pS, S)))
    L = O.pm_guess(pS, S, H, pD, T, pD, pD, 128.0)
    Sd = O.to_dense(pS, S)
    for _ in range(40):
        L = O.mcweeny_step(pS, S, pD, L, pD, pD, pD)
    LS = O.to_dense(pD, L) @ Sd
    assert np.linalg.norm(LS @ LS - LS) < 1e-12
    # half filling with the PM start: the projector holds the 128 lowest states
    e, C = sl.eigh(O.to_dense(pS, H), Sd)
    P = C[:, :128] @ C[:, :128].T
    assert np.abs(O.to_dense(pD, L) - P).max() < 1e-9


# ------------------------------------------------------------------ LNV

def _lnv_setup(si64, rl=12.0):
    cell, Spb, Hpb = si64
    pS, pL = O.Pattern.of_cell(cell, 10.0), O.Pattern.of_cell(cell, rl)
    pX, pU = O.Pattern.of_cell(cell, 10.0 + rl), O.Pattern.of_cell(cell, 20.0 + rl)
    S, H = O.scatter(pS, Spb), O.scatter(pS, Hpb)
    return cell, pS, pL, pX, pU, S, H


def test_lnv_energy_number_match_dense(si64):
    cell, pS, pL, pX, pU, S, H = _lnv_setup(si64)
    L = O.scatter(pL, I.random_blocks(cell, 12.0, 21)) * 0.05
    lnv = O.LNV.__new__(O.LNV)
    lnv.pS, lnv.S, lnv.H, lnv.pL, lnv.pX, lnv.pU = pS, S, H, pL, pX, pU
    E, N, _ = lnv.energy_number(L)
    Ld, Sd, Hd = O.to_dense(pL, L), O.to_dense(pS, S), O.to_dense(pS, H)
    K = 3 * Ld @ Sd @ Ld - 2 * Ld @ Sd @ Ld @ Sd @ Ld
    assert E == pytest.approx(2 * np.trace(K @ Hd), rel=1e-12)
    assert N == pytest.approx(2 * np.trace(K @ Sd), rel=1e-12)


def test_lnv_gradients_by_finite_differences(si64):
    cell, pS, pL, pX, pU, S, H = _lnv_setup(si64, rl=8.0)
    L = O.scatter(pL, I.random_blocks(cell, 8.0, 31)) * 0.05
    lnv = O.LNV.__new__(O.LNV)
    lnv.pS, lnv.S, lnv.H, lnv.pL, lnv.pX, lnv.pU = pS, S, H, pL, pX, pU
    lnv.L = L
    lnv.evaluate()
    Dl = O.scatter(pL, I.random_blocks(cell, 8.0, 32))
    for grad, idx in ((lnv.GE, 0), (lnv.GN, 1)):
        def f(h):
            return lnv.energy_number(L + h * Dl)[idx]
        # f is an exact cubic in h: Richardson on central differences removes the h^2 term
        d1 = (f(1e-2) - f(-1e-2)) / 2e-2
        d2 = (f(5e-3) - f(-5e-3)) / 1e-2
        fd = (4 * d2 - d1) / 3
        assert O.dot(grad, Dl) == pytest.approx(fd, rel=1e-8)


def test_lnv_line_is_exact_cubic(si64):
    cell, pS, pL, pX, pU, S, H = _lnv_setup(si64)
    L = O.scatter(pL, I.random_blocks(cell, 12.0, 41)) * 0.05
    D = O.scatter(pL, I.random_blocks(cell, 12.0, 42)) * 0.05
    lnv = O.LNV.__new__(O.LNV)
    lnv.pS, lnv.S, lnv.H, lnv.pL, lnv.pX, lnv.pU = pS, S, H, pL, pX, pU
    al = np.array([0.0, 0.3, 0.7, 1.1, 1.6])
    vals = np.array([lnv.energy_number(L + a * D)[:2] for a in al])
    for k in range(2):
        c = np.polyfit(al[:4], vals[:4, k], 3)
        assert np.polyval(c, al[4]) == pytest.approx(vals[4, k], rel=1e-10)


def test_cubic_min_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(200):
        w1 = -abs(rng.normal())
        w2, w3 = rng.normal(size=2)
        a = O.cubic_min(w1, w2, w3)
        roots = np.roots([3 * w3, 2 * w2, w1])
        good = [r.real for r in roots
                if abs(r.imag) < 1e-12 and r.real > 0 and 2 * w2 + 6 * w3 * r.real > 0]
        if a is None:
            assert not good
        else:
            assert a == pytest.approx(min(good), rel=1e-9)
    c2, c3 = O.cubic_coeffs(1.0, -2.0, 0.5, 1.0 - 1.0 + 0.75 - 0.125 * 0.5, 1.0,
                            1.0 - 2.0 + 3.0 - 0.5)
    assert (c2, c3) == (pytest.approx(3.0), pytest.approx(-0.5))


def test_lnv_converges_to_ground_state_projector(si64):
    cell, pS, pD, S, H = _dense_setup(si64)
    pT = pD
    T = O.hotelling_init(pS, S, pT)
    for _ in range(10):
        T, _ = O.hotelling_step(pS, S, pT, T, pD)
    L0 = O.pm_guess(pS, S, H, pT, T, pD, pD, 128.0)
    lnv = O.LNV(pS, S, H, pD, L0, 256.0, pD, pD)
    E_prev = lnv.E
    for _ in range(30):
        rec = lnv.step()
        if rec["n_corr"] == 0:
            assert rec["E"] <= E_prev + 1e-10
        E_prev = rec["E"]
    e, C = sl.eigh(O.to_dense(pS, H), O.to_dense(pS, S))
    assert lnv.E == pytest.approx(2.0 * e[:128].sum(), abs=1e-8)
    assert lnv.N == pytest.approx(256.0, rel=1e-10)
    P = C[:, :128] @ C[:, :128].T
    assert np.abs(O.to_dense(pD, lnv.L) - P).max() < 1e-4


def test_lnv_truncated_monotone(si64):
    cell, pS, pL, pX, pU, S, H = _lnv_setup(si64)
    pT = pL
    T = O.hotelling_init(pS, S, pT)
    for _ in range(10):
        T, _ = O.hotelling_step(pS, S, pT, T, pX)
    L0 = O.pm_guess(pS, S, H, pT, T, pX, pL, 128.0)
    lnv = O.LNV(pS, S, H, pL, L0, 256.0, pX, pU)
    E_prev = lnv.E
    for _ in range(8):
        mu, G = lnv.mu_and_g()
        rec = lnv.step()
        # Omega = E - mu N does not rise along the accepted step
        assert rec["E"] - mu * rec["N"] <= E_prev - mu * 256.0 + 1e-9
        E_prev = rec["E"]
    assert abs(lnv.N - 256.0) < 1e-8


def test_fallback_step_is_bounded_by_the_rms_change_of_L():
    """Without a minimiser of the exact cubic the step is 2 a2, capped where the RMS change
    of L over its stored values reaches 0.01."""
    rng = np.random.default_rng(8)
    D = rng.normal(size=1000)
    dd = float(D @ D)
    a = O.fallback_alpha(10.0, D.size, dd)          # 2 a2 = 20 is far beyond the cap
    assert np.sqrt(np.mean((a * D) ** 2)) == pytest.approx(0.01, rel=1e-12)
    small = 1e-6                                      # 2 a2 below the cap is kept
    assert O.fallback_alpha(small, D.size, dd) == 2.0 * small


def test_fallback_step_lowers_omega_where_the_cubic_has_no_minimiser(si64):
    """What the capped fallback step is for.  From L = 3 L_PM, far outside idempotency, the
    exact cubic of Omega = E - mu N along the first search direction has no positive
    minimiser (Omega falls without bound along D), so the step takes the fallback.  Checked
    on dense matrices, independent of the oracle's sparse products: Omega falls without
    bound along D, the capped step lowers it monotonically over its whole length, and the
    cap is the active limit (an RMS change of L of exactly 0.01, shorter than 2 a2)."""
    cell, pS, pL, pX, pU, S, H, T, L0 = _si64_start(si64)
    lnv = O.LNV(pS, S, H, pL, 3.0 * L0, 256.0, pX, pU, max_corr=0)
    Lstart = lnv.L.copy()
    mu, _ = lnv.mu_and_g()
    rec = lnv.step()
    assert rec["fallback"]
    D, alpha = lnv.D_prev, rec["alpha"]
    Sd, Hd = O.to_dense(pS, S), O.to_dense(pS, H)

    def omega(a):
        Ld = O.to_dense(pL, Lstart + a * D)
        LS = Ld @ Sd
        K = 3.0 * LS @ Ld - 2.0 * LS @ LS @ Ld
        return 2.0 * np.trace(K @ Hd) - mu * 2.0 * np.trace(K @ Sd)

    # no minimiser: Omega keeps falling far beyond the step
    far = [omega(a) for a in (0.0, alpha, 4.0 * alpha, 16.0 * alpha, 64.0 * alpha)]
    assert all(b < a for a, b in zip(far, far[1:])), far
    # the capped step lowers Omega at every point along it
    along = [omega(t * alpha) for t in np.linspace(0.0, 1.0, 6)]
    assert all(b < a for a, b in zip(along, along[1:])), along
    # the cap, not 2 a2, fixed the length: RMS change of L = 0.01 over its stored values
    assert alpha < 2.0 * (2.0 * rec["a1"])
    assert np.sqrt(np.mean((alpha * D) ** 2)) == pytest.approx(0.01, rel=1e-12)
    assert np.allclose(lnv.L, Lstart + alpha * D, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ preconditioned LNV

def _si64_start(si64):
    cell, pS, pL, pX, pU, S, H = _lnv_setup(si64)
    T = O.hotelling_init(pS, S, pL)
    for _ in range(12):
        T, _ = O.hotelling_step(pS, S, pL, T, pX)
    L0 = O.pm_guess(pS, S, H, pL, T, pX, pL, 128.0)
    return cell, pS, pL, pX, pU, S, H, T, L0


def _steps_to(lnv, tol=1e-8, cap=80):
    k = 0
    while lnv.gnorm_rms() > tol and k < cap:
        lnv.step()
        k += 1
    return k


def test_identity_preconditioner_reproduces_plain_steps(si64):
    cell, pS, pL, pX, pU, S, H, T, L0 = _si64_start(si64)
    plain = O.LNV(pS, S, H, pL, L0, 256.0, pX, pU)
    pre = O.LNV(pS, S, H, pL, L0, 256.0, pX, pU)
    pre.set_preconditioner(pL, O.identity(pL), O.Pattern.of_cell(cell, 24.0))
    for k in range(6):
        a, b = plain.step(), pre.step()
        assert b["E"] == pytest.approx(a["E"], abs=1e-10 * 64), k
        assert b["alpha"] == pytest.approx(a["alpha"], rel=1e-8), k
        assert (b["restart"], b["fallback"], b["n_corr"]) == (a["restart"], a["fallback"],
                                                              a["n_corr"]), k


def test_inverse_overlap_preconditioner_converges_in_fewer_steps(si64):
    cell, pS, pL, pX, pU, S, H, T, L0 = _si64_start(si64)
    plain = O.LNV(pS, S, H, pL, L0, 256.0, pX, pU)
    pre = O.LNV(pS, S, H, pL, L0, 256.0, pX, pU)
    pre.set_preconditioner(pL, T, O.Pattern.of_cell(cell, 24.0))
    n_plain, n_pre = _steps_to(plain), _steps_to(pre)
    assert pre.gnorm_rms() <= 1e-8 and plain.gnorm_rms() <= 1e-8
    assert n_pre < n_plain                      # 21 against 28 on this cell
    assert pre.E == pytest.approx(plain.E, abs=1e-10 * 64)
    assert abs(pre.N - 256.0) < 1e-8


def test_preconditioned_dense_limit_is_the_band_energy(si64):
    cell, pS, pD, S, H = _dense_setup(si64)
    T = O.from_dense(pD, np.linalg.inv(O.to_dense(pS, S)))
    L0 = O.pm_guess(pS, S, H, pD, T, pD, pD, 128.0)
    lnv = O.LNV(pS, S, H, pD, L0, 256.0, pD, pD)
    lnv.set_preconditioner(pD, T, pD)
    _steps_to(lnv, 1e-9, 60)
    e = sl.eigh(O.to_dense(pS, H), O.to_dense(pS, S), eigvals_only=True)
    assert lnv.E == pytest.approx(2.0 * e[:128].sum(), abs=1e-8)


# ------------------------------------------------------------------ CG overlap inverse

def _best_sparse_inverse(pS, S, pT):
    """The exact minimiser of ||I - S T||_F over symmetric T on P_T, by a direct sparse
    least-squares solve: unknowns t_u for the scalar pairs a <= b stored in P_T, columns
    vec(S E_u) with E_u = e_a e_b^T + e_b e_a^T (e_a e_a^T on the diagonal), normal
    equations solved by scipy.sparse.linalg.spsolve."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    Sd = O.to_dense(pS, S)
    n = Sd.shape[0]
    mask = O.to_dense(pT, np.ones(pT.n_values)) != 0
    ia, ib = np.nonzero(np.triu(mask))
    rows, cols, vals = [], [], []
    for u, (a, b) in enumerate(zip(ia, ib)):
        for src, dst in ((a, b), (b, a)) if a != b else ((a, b),):
            r = np.nonzero(Sd[:, src])[0]
            rows.append(r * n + dst)           # (r, dst) of S E_u, row-major vec
            cols.append(np.full(r.size, u))
            vals.append(Sd[r, src])
    A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n * n, ia.size))
    y = np.eye(n).ravel()
    t = spl.spsolve((A.T @ A).tocsc(), A.T @ y)
    Td = np.zeros((n, n))
    Td[ia, ib] = t
    Td[ib, ia] = t
    return O.from_dense(pT, Td), float(np.linalg.norm(A @ t - y))


def test_cg_inverse_reaches_the_least_squares_minimiser_on_p_t(si64):
    cell, Spb, _ = si64
    pS, pT = O.Pattern.of_cell(cell, 10.0), O.Pattern.of_cell(cell, 5.0)  # nearest neighbours
    pV = O.Pattern.of_cell(cell, 15.0)
    S = O.scatter(pS, Spb)
    T_best, r_best = _best_sparse_inverse(pS, S, pT)
    # a symmetric start that does not commute with S (I / sigma would hide a transposed
    # S T in the first residual)
    T0 = O.hotelling_init(pS, S, pT) + 0.05 * O.scatter(pT, I.random_blocks(cell, 5.0, 31))
    assert np.array_equal(O.gather(pT, T0, pT, transpose=True), T0)
    T, resid, gnorm = O.overlap_inverse_cg(pS, S, pT, T0, pV, 200, gtol=1e-13)
    assert gnorm[-1] <= 1e-13 * gnorm[0] and len(resid) < 200
    assert np.all(np.diff(resid) <= 1e-14 * resid[0])       # exact line searches
    assert resid[-1] == pytest.approx(r_best, rel=1e-10)
    assert np.abs(T - T_best).max() <= 1e-9 * np.abs(T_best).max()
    # the residual the function reports is the one of the T it returns
    V = O.bsmm(1.0, pS, S, pT, T, 0.0, pV)
    assert O.frob_minus_identity(pV, V) == pytest.approx(resid[-1], rel=1e-10)


def test_cg_inverse_dense_limit_is_the_inverse(si64):
    cell, Spb, _ = si64
    pS, pD = O.Pattern.of_cell(cell, 10.0), O.Pattern.of_cell(cell, 22.0)
    assert pD.nnzb == cell.n_atoms ** 2
    S = O.scatter(pS, Spb)
    T, resid, _ = O.overlap_inverse_cg(pS, S, pD, O.hotelling_init(pS, S, pD), pD, 200,
                                       gtol=1e-14)
    Sinv = np.linalg.inv(O.to_dense(pS, S))
    assert np.abs(O.to_dense(pD, T) - Sinv).max() <= 1e-10 * np.abs(Sinv).max()
    assert resid[-1] <= 1e-11 * resid[0]


def test_cg_inverse_beats_the_truncated_hotelling_fixed_point(si64):
    cell, Spb, _ = si64
    pS, pT = O.Pattern.of_cell(cell, 10.0), O.Pattern.of_cell(cell, 12.0)
    pV = O.Pattern.of_cell(cell, 22.0)
    S = O.scatter(pS, Spb)
    T0 = O.hotelling_init(pS, S, pT)
    Th = T0
    for _ in range(20):
        Th, r_hot = O.hotelling_step(pS, S, pT, Th, pV)
    T, resid, _ = O.overlap_inverse_cg(pS, S, pT, T0, pV, 40)
    assert resid[-1] < r_hot                               # best T on the same pattern
    assert np.array_equal(O.gather(pT, T, pT, transpose=True), T)   # stays exactly symmetric


# ------------------------------------------------------------------ degenerate cells

def test_single_atom_cell_reduces_to_dense_algebra():
    """One atom: every pattern, whatever its range (below, near or beyond the box), is the
    self pair alone, and the product, trace and Hotelling iteration are those of one dense
    9 x 9 block."""
    pos, box, nb = np.array([[1.0, 2.0, 3.0]]), np.array([7.0, 7.0, 7.0]), np.array([9])
    rng = np.random.default_rng(5)
    for r in (0.5, 3.0, 20.0):
        p = O.Pattern(pos, box, nb, r)
        assert p.nnzb == 1 and list(p.col) == [0] and list(p.off) == [0, 81]
    A, B, C = (rng.standard_normal((9, 9)) for _ in range(3))
    got = O.bsmm(0.7, p, A.ravel(), p, B.ravel(), 1.3, p, C.ravel().copy())
    np.testing.assert_allclose(got.reshape(9, 9), 0.7 * A @ B + 1.3 * C, rtol=0, atol=1e-13)
    assert abs(O.trace_prod(p, A.ravel(), p, B.ravel()) - np.trace(A @ B)) < 1e-12
    M = rng.standard_normal((9, 9))
    S = np.eye(9) + 0.05 * (M @ M.T)
    T = O.hotelling_init(p, S.ravel(), p)
    for _ in range(40):
        R0 = np.eye(9) - S @ T.reshape(9, 9)
        T, _ = O.hotelling_step(p, S.ravel(), p, T, p)
        np.testing.assert_allclose(np.eye(9) - S @ T.reshape(9, 9), R0 @ R0, rtol=0, atol=1e-13)
    np.testing.assert_allclose(T.reshape(9, 9), sl.inv(S), rtol=0, atol=1e-12)
