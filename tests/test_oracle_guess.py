"""Pins of the learned-guess oracle: frames, rotations, descriptors, network gradients."""
import numpy as np
import pytest

import oracle as O
from oracle import guess as G
from paper_2205_08941_gb300 import inputs as I


@pytest.fixture(scope="module")
def cell_and_pattern():
    cell = I.diamond_cell(2, a=10.26, sigma=0.1, seed=5, norb=9)
    return cell, O.Pattern.of_cell(cell, 7.0)


def test_frames_orthonormal_right_handed_along_bond(cell_and_pattern):
    cell, p = cell_and_pattern
    for b in G.pairs_of(p)[:200]:
        F, _ = G.frame_and_descriptor(p, b)
        assert np.allclose(F @ F.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(F) == pytest.approx(1.0, abs=1e-12)
        i, j = p.row[b], p.col[b]
        if i != j:
            d = G._mi(p.pos, p.box, i, j)
            assert np.allclose(F[2], d / np.linalg.norm(d), atol=1e-12)


def test_orbital_rotation_is_orthogonal_and_round_trips(cell_and_pattern):
    cell, p = cell_and_pattern
    rng = np.random.default_rng(1)
    for b in G.pairs_of(p)[:50]:
        F, _ = G.frame_and_descriptor(p, b)
        D = G.orbital_rotation(F, 9)
        assert np.allclose(D @ D.T, np.eye(9), atol=1e-12)
        blk = rng.normal(size=(9, 9))
        assert np.allclose(G.untarget(F, G.target(F, blk), 9), blk, atol=1e-12)


def test_rotation_matches_slater_koster_generator():
    # the d-shell rotation equals the one the input generator builds from its own frames
    rng = np.random.default_rng(2)
    u = rng.normal(size=(5, 3))
    rot = I._frames(u / np.linalg.norm(u, axis=1, keepdims=True))
    full = I.orbital_rotation(rot)
    for k in range(5):
        assert np.allclose(G.orbital_rotation(rot[k], 9), full[k], atol=1e-12)


def test_descriptors_and_targets_invariant_under_cubic_rotation():
    cell = I.diamond_cell(2, a=10.26, sigma=0.1, seed=6, norb=9)
    # 90 degree rotation about z maps the cubic box onto itself: (x, y, z) -> (-y, x, z)
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    rot = I.Cell(pos=np.mod(cell.pos @ R.T, cell.box), box=cell.box.copy(), nb=cell.nb)
    p, q = O.Pattern.of_cell(cell, 7.0), O.Pattern.of_cell(rot, 7.0)
    assert np.array_equal(p.col, q.col)
    L = O.scatter(p, I.random_blocks(cell, 7.0, 3))
    # the same operator in the rotated global frame: L' = D(R) L D(R)^T per block
    DR = G.orbital_rotation(R, 9)
    Lr = np.concatenate([(DR @ G.block(p, L, b) @ DR.T).reshape(-1) for b in range(p.nnzb)])
    for b in G.pairs_of(p)[:120]:
        F, f = G.frame_and_descriptor(p, b)
        Fr, fr = G.frame_and_descriptor(q, b)
        assert np.allclose(f, fr, atol=1e-10)
        assert np.allclose(G.target(F, G.block(p, L, b)), G.target(Fr, G.block(q, Lr, b)),
                           atol=1e-10)


def test_network_gradients_by_finite_differences():
    rng = np.random.default_rng(3)
    n_w = sum(G.DIMS[k] * G.DIMS[k + 1] for k in range(4))
    n_b = sum(G.DIMS[1:])
    w = rng.normal(size=n_w) * 0.05
    b = rng.normal(size=n_b) * 0.05
    X = rng.normal(size=(7, 64))
    T = rng.normal(size=(7, 81))
    args = (np.zeros(64), np.ones(64), np.zeros(81), np.ones(81))
    loss, gw, gb = G.loss_and_grads(w, b, X, T, *args)
    h = 1e-6
    for idx in rng.choice(n_w, size=12, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (G.loss_and_grads(wp, b, X, T, *args)[0] - G.loss_and_grads(wm, b, X, T, *args)[0]) / (2 * h)
        assert gw[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    for idx in rng.choice(n_b, size=8, replace=False):
        bp, bm = b.copy(), b.copy()
        bp[idx] += h
        bm[idx] -= h
        fd = (G.loss_and_grads(w, bp, X, T, *args)[0] - G.loss_and_grads(w, bm, X, T, *args)[0]) / (2 * h)
        assert gb[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_descriptor_values_of_a_hand_computed_four_atom_case():
    """Descriptor of pair (0, 1) in a four-atom cluster whose values are fixed by hand.

    Atoms (box 60 bohr, so no periodic image is within the 10-bohr pattern): 0 at the
    origin, 1 at 4 along z, 2 at (3.2, 0, 2) and 3 at (0, 4.8 s, 2 + 4.8 s), s = 1/sqrt(2).
    Bond midpoint m = (0, 0, 2): atom 2 sits 3.2 from m along +x (it fixes e1 = x), atom 3
    sits 4.8 from m along (0, s, s).  So the frame is the identity and the neighbour terms
    need only exact values: the cosine cut at 8 bohr is (1 + cos(0.4 pi))/2 = (3 + sqrt5)/8
    at 3.2 and (5 - sqrt5)/8 at 4.8; the radial Gaussians (width 1.2, centres 1.6 n) take
    the values 1, exp(-8/9), exp(-32/9), exp(-8) at 0, 1, 2, 3 centre spacings; the harmonics
    (1, z, x, y, (3z^2-1)/2, xz, yz, (x^2-y^2)/2, xy) are (1, 0, 1, 0, -1/2, 0, 0, 1/2, 0)
    along x and (1, s, 0, s, 1/4, 0, 1/2, -1/4, 0) along (0, s, s).  The pair part: ten
    Gaussians of r = 4 (width 1.6, centres 1.6 q): exp(-t^2/2) with t = 2.5, 1.5, 0.5,
    -0.5, ..., -5.5."""
    s = 1.0 / np.sqrt(2.0)
    o = np.array([20.0, 20.0, 20.0])
    pos = np.array([[0, 0, 0], [0, 0, 4.0], [3.2, 0, 2.0], [0, 4.8 * s, 2.0 + 4.8 * s]]) + o
    cell = I.Cell(pos=pos, box=np.array([60.0, 60.0, 60.0]), nb=np.full(4, 9, np.int32))
    p = O.Pattern.of_cell(cell, 10.0)
    b = int(O.block_index(p, 0, 1))
    F, f = G.frame_and_descriptor(p, b)
    assert np.allclose(F, np.eye(3), atol=1e-12)
    expect = np.zeros(64)
    for q in range(10):
        expect[q] = np.exp(-0.5 * (2.5 - q) ** 2)
    g = {0: 1.0, 1: np.exp(-8.0 / 9.0), 2: np.exp(-32.0 / 9.0), 3: np.exp(-8.0)}
    fc2, fc3 = (3.0 + np.sqrt(5.0)) / 8.0, (5.0 - np.sqrt(5.0)) / 8.0
    ang2 = np.array([1, 0, 1, 0, -0.5, 0, 0, 0.5, 0])
    ang3 = np.array([1, s, 0, s, 0.25, 0, 0.5, -0.25, 0])
    for n in range(6):
        h2 = g[abs(n - 2)] * fc2      # atom 2 sits at centre n = 2
        h3 = g[abs(n - 3)] * fc3      # atom 3 sits at centre n = 3
        expect[10 + 9 * n:19 + 9 * n] = h2 * ang2 + h3 * ang3
    assert np.allclose(f, expect, rtol=0, atol=1e-13), np.nonzero(~np.isclose(f, expect))
