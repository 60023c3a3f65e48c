"""Oracle for the block-sparse linear-scaling solver: plain CPU FP64, slow and obvious.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg may import this package.  It shares no code with the CUDA library in
paper_2205_08941_gb300/ and never imports it.

The paper states the method only in words: CONQUEST's linear-scaling ground-state solver
works on sparse, atom-blocked matrices with locality enforced everywhere (Background), by
linear-scaling optimisation of the density matrix with a linear-scaling inversion of the
overlap (Development Priorities), and a GPU matrix multiplication is its first offloaded
kernel (Meeting the Exascale Challenges).  The formulas written out here are the published
methods that solver is built from, restated from their mathematics:

* masked block product  C = mask_{P_C}(A B)               (the sparse matrix product)
* Hotelling / Schulz     T <- 2T - T S T                   (overlap inversion)
* least-squares inverse  min ||I - S T||_F over T on P_T, by linear CG (overlap inversion)
* Li-Nunes-Vanderbilt    K = 3LSL - 2LSLSL, E = 2Tr(KH), N = 2Tr(KS)  (density matrix)
* McWeeny purification   L <- 3LSL - 2LSLSL
* Palser-Manolopoulos    initial L from T ~ S^-1 and Gershgorin bounds of TH

Heavy loops live in oracle.c (compiled by build() with gcc, OpenMP over output rows);
the drivers below are plain numpy on the values of each pattern.  Every function that is
pinned names its pin in tests/test_oracle_*.py; none is unpinned.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_liboracle.so")
_LIB = None

_I64P = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_I32P = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so (plain gcc, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", _SO + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        pat = [_I64P, _I32P, _I64P]
        lib.orc_pattern_count.argtypes = [ctypes.c_int, _F64P, _F64P, ctypes.c_double, _I64P]
        lib.orc_pattern_fill.argtypes = [ctypes.c_int, _F64P, _F64P, ctypes.c_double, _I64P,
                                         _I32P]
        lib.orc_bsmm.argtypes = ([ctypes.c_int, _I32P] + pat + [_F64P] + pat + [_F64P] + pat
                                 + [_F64P, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                    ctypes.c_int])
        lib.orc_bsmm.restype = ctypes.c_int
        lib.orc_triplet_count.argtypes = [ctypes.c_int, _I32P, _I64P, _I32P, _I64P, _I32P,
                                          _I64P, _I32P, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                          ctypes.c_int]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_trace_prod.argtypes = [ctypes.c_int, _I32P] + pat + [_F64P] + pat + [_F64P]
        lib.orc_trace_prod.restype = ctypes.c_double
        lib.orc_dot.argtypes = [ctypes.c_int64, _F64P, _F64P]
        lib.orc_dot.restype = ctypes.c_double
        lib.orc_frob2_minus_identity.argtypes = [ctypes.c_int, _I32P] + pat + [_F64P]
        lib.orc_frob2_minus_identity.restype = ctypes.c_double
        lib.orc_gather.argtypes = ([ctypes.c_int, _I32P] + pat + [_F64P] + pat
                                   + [_F64P, ctypes.c_int])
        lib.orc_row_sums.argtypes = [ctypes.c_int, _I32P] + pat + [_F64P, _F64P, _F64P, _F64P]
        lib.orc_find_block.argtypes = [_I64P, _I32P, ctypes.c_int, ctypes.c_int]
        lib.orc_find_block.restype = ctypes.c_int64
        _LIB = lib
    return _LIB


class Pattern:
    """P_R = {(i, j) : minimum-image d(i, j) < R} over the atoms of a cell, CSR by atom row.

    Self pairs are always included (d = 0).  Block b = (i, col[b]) is nb[i] x nb[col[b]]
    doubles, row-major, at values[off[b]:off[b+1]].
    """

    def __init__(self, pos, box, nb, range_):
        self.pos = np.ascontiguousarray(pos, dtype=np.float64)
        self.box = np.ascontiguousarray(box, dtype=np.float64)
        self.nb = np.ascontiguousarray(nb, dtype=np.int32)
        self.range = float(range_)
        self.n = int(self.pos.shape[0])
        lib = _lib()
        cnt = np.zeros(self.n, dtype=np.int64)
        lib.orc_pattern_count(self.n, self.pos.reshape(-1), self.box, self.range, cnt)
        self.rp = np.zeros(self.n + 1, dtype=np.int64)
        np.cumsum(cnt, out=self.rp[1:])
        self.col = np.zeros(int(self.rp[-1]), dtype=np.int32)
        lib.orc_pattern_fill(self.n, self.pos.reshape(-1), self.box, self.range, self.rp,
                             self.col)
        self.row = np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.rp))
        sizes = self.nb[self.row].astype(np.int64) * self.nb[self.col].astype(np.int64)
        self.off = np.zeros(self.nnzb + 1, dtype=np.int64)
        np.cumsum(sizes, out=self.off[1:])

    @classmethod
    def of_cell(cls, cell, range_):
        return cls(cell.pos, cell.box, cell.nb, range_)

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_values(self) -> int:
        return int(self.off[-1])

    @property
    def n_orb(self) -> int:
        return int(self.nb.sum())

    def args(self):
        return (self.rp, self.col, self.off)

    def keys(self):
        return self.row.astype(np.int64) * self.n + self.col

    def zeros(self):
        return np.zeros(self.n_values)


def block_index(p: Pattern, i, j):
    """Index of block (i, j) in p for arrays i, j (-1 where not stored)."""
    keys = p.keys()
    q = np.asarray(i, dtype=np.int64) * p.n + np.asarray(j, dtype=np.int64)
    pos = np.searchsorted(keys, q)
    pos_c = np.minimum(pos, keys.shape[0] - 1)
    return np.where((pos < keys.shape[0]) & (keys[pos_c] == q), pos_c, -1)


def scatter(p: Pattern, pb) -> np.ndarray:
    """Values on p from a PairBlocks coordinate list; every pair must be stored in p."""
    out = p.zeros()
    if pb.n_pairs == 0:
        return out
    idx = block_index(p, pb.i, pb.j)
    if np.any(idx < 0):
        raise ValueError("pair list holds a block outside the pattern")
    lens = np.diff(pb.off)
    dst = np.repeat(p.off[idx] - pb.off[:-1], lens) + np.arange(int(pb.off[-1]))
    out[dst] = pb.values
    return out


def gather(p_src: Pattern, src, p_dst: Pattern, transpose: bool = False):
    """dst_ij = src_ij (or (src_ji)^T) on p_dst, zero where src does not store the block."""
    dst = p_dst.zeros()
    _lib().orc_gather(p_src.n, p_src.nb, *p_src.args(), np.ascontiguousarray(src),
                      *p_dst.args(), dst, 1 if transpose else 0)
    return dst


def bsmm(alpha, pA: Pattern, A, pB: Pattern, B, beta, pC: Pattern, C=None, rows=None):
    """C <- beta C + alpha mask_{P_C}(A B), the exact masked block product.

    rows: optional list of atom rows to compute (the others are left as they are).
    """
    if C is None:
        C = pC.zeros()
    rows_arr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    rc = _lib().orc_bsmm(pA.n, pA.nb, *pA.args(), np.ascontiguousarray(A), *pB.args(),
                         np.ascontiguousarray(B), *pC.args(), C, float(alpha), float(beta),
                         None if rows_arr is None else rows_arr.ctypes.data,
                         0 if rows_arr is None else int(rows_arr.shape[0]))
    if rc != 0:
        raise ValueError("orbital count per atom outside 1..32")
    return C


def triplets(pA: Pattern, pB: Pattern, pC: Pattern, rows=None):
    """(number of (i,k,j) triplets, useful flops = sum 2 n_i n_k n_j) of mask_{P_C}(A B),
    over all rows or the listed output rows."""
    t = ctypes.c_int64()
    f = ctypes.c_double()
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    _lib().orc_triplet_count(pA.n, pA.nb, pA.rp, pA.col, pB.rp, pB.col, pC.rp, pC.col,
                             ctypes.byref(t), ctypes.byref(f),
                             None if r is None else r.ctypes.data,
                             0 if r is None else int(r.shape[0]))
    return int(t.value), float(f.value)


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(_lib().orc_num_threads())


def trace_prod(pA: Pattern, A, pB: Pattern, B) -> float:
    """Tr(A B) = sum_{(i,j) in P_A} <A_ij, (B_ji)^T> (compensated sum)."""
    return float(_lib().orc_trace_prod(pA.n, pA.nb, *pA.args(), np.ascontiguousarray(A),
                                       *pB.args(), np.ascontiguousarray(B)))


def dot(A, B) -> float:
    """Frobenius inner product over the stored values of one pattern."""
    A = np.ascontiguousarray(A)
    return float(_lib().orc_dot(A.shape[0], A, np.ascontiguousarray(B)))


def frob_minus_identity(p: Pattern, M) -> float:
    """||M - I||_F over the stored blocks of M."""
    return math.sqrt(_lib().orc_frob2_minus_identity(p.n, p.nb, *p.args(),
                                                     np.ascontiguousarray(M)))


def row_sums(p: Pattern, M):
    """Per scalar row: (diagonal element, off-diagonal |.| sum, |.| row sum)."""
    n = p.n_orb
    c, r, a = np.zeros(n), np.zeros(n), np.zeros(n)
    _lib().orc_row_sums(p.n, p.nb, *p.args(), np.ascontiguousarray(M), c, r, a)
    return c, r, a


def identity(p: Pattern, scale: float = 1.0):
    """scale * I on the diagonal blocks of p."""
    out = p.zeros()
    for i in range(p.n):
        b = int(block_index(p, [i], [i])[0])
        n_ = int(p.nb[i])
        blk = out[p.off[b]:p.off[b + 1]].reshape(n_, n_)
        blk[np.arange(n_), np.arange(n_)] = scale
    return out


def to_dense(p: Pattern, M) -> np.ndarray:
    """Dense (n_orb, n_orb) matrix of M on p (tiny cells only)."""
    o = np.zeros(p.n + 1, dtype=np.int64)
    np.cumsum(p.nb, out=o[1:])
    d = np.zeros((int(o[-1]), int(o[-1])))
    for b in range(p.nnzb):
        i, j = int(p.row[b]), int(p.col[b])
        d[o[i]:o[i + 1], o[j]:o[j + 1]] = M[p.off[b]:p.off[b + 1]].reshape(p.nb[i], p.nb[j])
    return d


def from_dense(p: Pattern, D) -> np.ndarray:
    """mask_P(D): the blocks of a dense matrix on p (tiny cells only)."""
    o = np.zeros(p.n + 1, dtype=np.int64)
    np.cumsum(p.nb, out=o[1:])
    out = p.zeros()
    for b in range(p.nnzb):
        i, j = int(p.row[b]), int(p.col[b])
        out[p.off[b]:p.off[b + 1]] = D[o[i]:o[i + 1], o[j]:o[j + 1]].reshape(-1)
    return out


# ---------------------------------------------------------------------------------------
# Hotelling (Schulz) inversion of the overlap: T_{n+1} = 2 T_n - T_n S T_n.
# ---------------------------------------------------------------------------------------

def hotelling_init(pS: Pattern, S, pT: Pattern):
    """T_0 = I / sigma with sigma = max_a sum_b |S_ab| (largest absolute scalar row sum).

    S is symmetric positive definite with lambda_max <= sigma, so ||I - T_0 S|| < 1.
    """
    _, _, a = row_sums(pS, S)
    return identity(pT, 1.0 / float(a.max()))


def hotelling_step(pS: Pattern, S, pT: Pattern, T, pV: Pattern):
    """One step: V = mask_{P_V}(S T), r = ||V - I||_F, T' = 2T - mask_{P_T}(T V).

    P_V must reach r_S + r_T so that V is the whole product.  Returns (T', r); r belongs
    to the incoming T.
    """
    V = bsmm(1.0, pS, S, pT, T, 0.0, pV)
    r = frob_minus_identity(pV, V)
    W = bsmm(1.0, pT, T, pV, V, 0.0, pT)
    return 2.0 * T - W, r


def overlap_inverse_cg(pS: Pattern, S, pT: Pattern, T, pV: Pattern, max_iter: int,
                       gtol: float = 0.0):
    """Overlap inverse as the best T on P_T: minimise f(T) = ||I - S T||_F^2 over symmetric T
    stored on P_T, by linear conjugate gradients from the given T (another route than the
    Hotelling iteration to the overlap inverse; Development Priorities).

    R = I - S T lives on P_V (P_V must reach r_S + r_T, so R is the whole residual).  For a
    symmetric change dT on P_T, df = -2 <S R, dT>, so the gradient on P_T is
    G = -(W + W^T) with W = mask_{P_T}(S R).  Along D, f is the quadratic
    ||R||^2 - 2a<R, S D> + a^2 ||S D||^2, minimised at a = -<G, D> / (2 ||S D||^2); then
    T += a D, R -= a S D, and the next direction is -G + (<G, G> / <G_prev, G_prev>) D
    (Fletcher-Reeves, exact for a quadratic with exact line searches).
    Stops after max_iter steps, or once ||G||_F <= gtol * ||G_0||_F.

    Returns (T, resid, gnorm): resid[k] = ||I - S T_k||_F and gnorm[k] = ||G_k||_F for every
    iterate T_0 (the start) ... T_n, so n = len(resid) - 1 steps were taken.
    """
    T = np.array(T, dtype=np.float64, copy=True)
    R = identity(pV) - bsmm(1.0, pS, S, pT, T, 0.0, pV)
    D, gg_prev = None, None
    resid, gnorm = [], []
    for k in range(max_iter + 1):
        W = bsmm(1.0, pS, S, pV, R, 0.0, pT)
        G = -(W + gather(pT, W, pT, transpose=True))
        gg = dot(G, G)
        resid.append(float(np.sqrt(dot(R, R))))
        gnorm.append(float(np.sqrt(gg)))
        if k == max_iter or gnorm[-1] <= gtol * gnorm[0]:
            break
        D = -G if D is None else -G + (gg / gg_prev) * D
        SD = bsmm(1.0, pS, S, pT, D, 0.0, pV)
        a = -dot(G, D) / (2.0 * dot(SD, SD))
        T += a * D
        R -= a * SD
        gg_prev = gg
    return T, resid, gnorm


# ---------------------------------------------------------------------------------------
# Palser-Manolopoulos start and McWeeny purification (non-orthogonal forms).
# ---------------------------------------------------------------------------------------

def pm_guess(pS: Pattern, S, H, pT: Pattern, T, pX: Pattern, pL: Pattern, n_occ: float):
    """L_0 = mask_L[(lambda/N)(mu T - T H T) + (n_occ/N) T], N = number of orbitals.

    mu = Tr(T H)/N; h_min, h_max are the Gershgorin bounds of T H;
    lambda = min(n_occ/(h_max - mu), (N - n_occ)/(mu - h_min)).
    With T = S^-1 this gives Tr(L_0 S) = n_occ and spec(L_0 S) in [0, 1].
    P_X must reach r_T + r_S.
    """
    n_orb = pS.n_orb
    TH = bsmm(1.0, pT, T, pS, H, 0.0, pX)
    mu = trace_prod(pT, T, pS, H) / n_orb
    centre, radius, _ = row_sums(pX, TH)
    h_min = float((centre - radius).min())
    h_max = float((centre + radius).max())
    lam = min(n_occ / (h_max - mu), (n_orb - n_occ) / (mu - h_min))
    L0 = bsmm(-lam / n_orb, pX, TH, pT, T, 0.0, pL)
    L0 += (lam * mu / n_orb + n_occ / n_orb) * gather(pT, T, pL)
    return L0


def mcweeny_step(pS: Pattern, S, pL: Pattern, L, pX: Pattern, pU: Pattern, p2L: Pattern):
    """L' = mask_L(3 LSL - 2 LSLSL).

    X = L S on P_X (r_L + r_S), U = S X on P_U (2 r_S + r_L), M = L U on P_2L (2 r_L);
    L' = 3 mask_L(X L) - 2 mask_L(M L).  Each product is exact on its pattern.
    """
    X = bsmm(1.0, pL, L, pS, S, 0.0, pX)
    U = bsmm(1.0, pS, S, pX, X, 0.0, pU)
    M = bsmm(1.0, pL, L, pU, U, 0.0, p2L)
    out = bsmm(3.0, pX, X, pL, L, 0.0, pL)
    return bsmm(-2.0, p2L, M, pL, L, 1.0, pL, out)


# ---------------------------------------------------------------------------------------
# Li-Nunes-Vanderbilt minimisation (spin-degenerate).
# ---------------------------------------------------------------------------------------

def cubic_coeffs(f0, g, a1, f1, a2, f2):
    """(c2, c3) of f(a) = f0 + g a + c2 a^2 + c3 a^3 through (a1, f1) and (a2, f2)."""
    r1 = f1 - f0 - g * a1
    r2 = f2 - f0 - g * a2
    det = a1 * a1 * a2 * a2 * (a2 - a1)
    c2 = (r1 * a2 ** 3 - r2 * a1 ** 3) / det
    c3 = (a1 * a1 * r2 - a2 * a2 * r1) / det
    return c2, c3


def cubic_min(w1, w2, w3):
    """Smallest positive minimiser of w1 a + w2 a^2 + w3 a^3 (derivative root with positive
    curvature), or None.  The root is written as -2 w1 / (2 w2 + sqrt(disc))."""
    disc = 4.0 * w2 * w2 - 12.0 * w3 * w1
    if disc < 0.0:
        return None
    den = 2.0 * w2 + math.sqrt(disc)
    if den <= 0.0:
        return None
    a = -2.0 * w1 / den
    return a if a > 0.0 else None


def fallback_alpha(a2, n_values, dd):
    """Step when the cubic has no minimiser (it falls without bound along D): 2 a2, but at
    most the step that changes L by 0.01 RMS over its n_values stored values."""
    return min(2.0 * a2, 0.01 * math.sqrt(n_values / dd)) if dd > 0.0 else 2.0 * a2


class LNV:
    """Li-Nunes-Vanderbilt minimisation of E = 2 Tr[(3LSL - 2LSLSL) H] at fixed
    N = 2 Tr[(3LSL - 2LSLSL) S] = n_electrons, over L on the pattern P_L.

    Patterns: P_X reaches r_L + r_S, P_U reaches 2 r_S + r_L (H shares S's pattern).
    Each step: chemical potential mu = <G_E,G_N>/<G_N,G_N>, G = G_E - mu G_N, Polak-Ribiere
    conjugate direction projected orthogonal to G_N, exact cubic line search of
    Omega = E - mu N from two trial points, L += alpha* D, then at most five linear
    corrections along G_N while |N - N_e| > n_tol N_e.
    """

    def __init__(self, pS, S, H, pL, L, n_electrons, pX, pU, n_tol=1e-10, max_corr=5):
        self.pS, self.S, self.H, self.pL, self.pX, self.pU = pS, S, H, pL, pX, pU
        self.L = np.array(L, dtype=np.float64)
        self.ne = float(n_electrons)
        self.n_tol = n_tol
        self.max_corr = max_corr
        self.G_prev = None
        self.D_prev = None
        self.Z_prev = None
        self.alpha_prev = None
        self.precond = None
        self.history = []
        self.evaluate()
        self.n_corrections_initial = self.correct_n()

    def set_preconditioner(self, pT, T, pTL):
        """Search directions from Z = sym(mask_L(T G T)) in place of G, with T ~ S^-1 from
        Hotelling on P_T (the covariant gradient raised with the inverse overlap, the
        tensorially consistent steepest-descent direction in a non-orthogonal basis).  T G
        lands on pTL, which must reach r_T + r_L.  Resets the search history."""
        self.precond = (pT, np.array(T, dtype=np.float64), pTL)
        self.G_prev = self.D_prev = self.Z_prev = self.alpha_prev = None

    def direction_of(self, G):
        """G itself, or with a preconditioner Z = (mask_L(T G T) + its transpose) / 2."""
        if self.precond is None:
            return G
        pT, T, pTL = self.precond
        TG = bsmm(1.0, pT, T, self.pL, G, 0.0, pTL)
        Z = bsmm(1.0, pTL, TG, pT, T, 0.0, self.pL)
        return 0.5 * (Z + gather(self.pL, Z, self.pL, transpose=True))

    # E and N from the five products that a trial point needs
    def energy_number(self, L):
        pS, pL, pX, pU = self.pS, self.pL, self.pX, self.pU
        X = bsmm(1.0, pL, L, pS, self.S, 0.0, pX)      # L S
        Y = bsmm(1.0, pL, L, pS, self.H, 0.0, pX)      # L H
        U = bsmm(1.0, pS, self.S, pX, X, 0.0, pU)      # S L S
        R1 = bsmm(1.0, pU, U, pX, Y, 0.0, pL)          # S L S L H
        R3 = bsmm(1.0, pU, U, pX, X, 0.0, pL)          # S L S L S
        E = 2.0 * (3.0 * trace_prod(pX, X, pX, Y) - 2.0 * trace_prod(pL, L, pL, R1))
        N = 2.0 * (3.0 * trace_prod(pX, X, pX, X) - 2.0 * trace_prod(pL, L, pL, R3))
        return E, N, (X, Y, U, R1, R3)

    def evaluate(self):
        """Full evaluation at self.L: E, N and the gradients G_E, G_N on P_L."""
        pS, pL, pX, pU = self.pS, self.pL, self.pX, self.pU
        L = self.L
        E, N, (X, Y, U, R1, R3) = self.energy_number(L)
        Z = bsmm(1.0, pS, self.S, pX, Y, 0.0, pU)      # S L H
        R2 = bsmm(1.0, pU, Z, pX, X, 0.0, pL)          # S L H L S
        Zl = gather(pU, Z, pL)
        ZTl = gather(pU, Z, pL, transpose=True)
        R1T = gather(pL, R1, pL, transpose=True)
        self.GE = 2.0 * (3.0 * (Zl + ZTl) - 2.0 * (R1 + R1T + R2))
        self.GN = 12.0 * (gather(pU, U, pL) - R3)
        self.E, self.N = E, N
        return E, N

    def correct_n(self):
        k = 0
        while abs(self.N - self.ne) > self.n_tol * self.ne and k < self.max_corr:
            self.L = self.L + ((self.ne - self.N) / dot(self.GN, self.GN)) * self.GN
            self.evaluate()
            k += 1
        return k

    def mu_and_g(self):
        mu = dot(self.GE, self.GN) / dot(self.GN, self.GN)
        return mu, self.GE - mu * self.GN

    def gnorm_rms(self):
        _, G = self.mu_and_g()
        return math.sqrt(dot(G, G) / G.shape[0])

    def step(self):
        GN = self.GN
        gn2 = dot(GN, GN)
        mu, G = self.mu_and_g()
        Zg = self.direction_of(G)  # G itself unless a preconditioner is set
        restart = self.G_prev is None
        if restart:
            D = -Zg
        else:
            # Polak-Ribiere in the preconditioned form <G, Z - Z_prev> / <G_prev, Z_prev>
            beta = max(0.0, dot(G, Zg - self.Z_prev) / dot(self.G_prev, self.Z_prev))
            D = -Zg + beta * self.D_prev
        D = D - (dot(D, GN) / gn2) * GN
        if dot(G, D) >= 0.0:
            D = -Zg
            restart = True
        if self.alpha_prev is None:
            a1 = 0.1 * math.sqrt(G.shape[0]) / math.sqrt(dot(Zg, Zg))
        else:
            a1 = self.alpha_prev
        a2 = 2.0 * a1
        E0, N0 = self.E, self.N
        gE = dot(self.GE, D)
        gN = dot(GN, D)
        E1, N1, _ = self.energy_number(self.L + a1 * D)
        E2, N2, _ = self.energy_number(self.L + a2 * D)
        e2, e3 = cubic_coeffs(E0, gE, a1, E1, a2, E2)
        n2, n3 = cubic_coeffs(N0, gN, a1, N1, a2, N2)
        alpha = cubic_min(gE - mu * gN, e2 - mu * n2, e3 - mu * n3)
        fallback = alpha is None
        if fallback:
            alpha = fallback_alpha(a2, G.shape[0], dot(D, D))
        self.L = self.L + alpha * D
        self.evaluate()
        ncorr = self.correct_n()
        self.G_prev, self.D_prev, self.Z_prev, self.alpha_prev = G, D, Zg, alpha
        mu_new, G_new = self.mu_and_g()
        rec = {"E": self.E, "N": self.N, "mu": mu_new,
               "gnorm": math.sqrt(dot(G_new, G_new) / G_new.shape[0]),
               "alpha": alpha, "a1": a1, "restart": restart, "fallback": fallback,
               "n_corr": ncorr, "E1": E1, "E2": E2, "omega_pred": None}
        self.history.append(rec)
        return rec
