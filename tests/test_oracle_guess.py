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
