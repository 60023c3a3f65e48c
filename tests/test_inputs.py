"""Checks of the synthetic input generator: Slater-Koster angular forms, symmetry, gap."""
import math

import numpy as np
import pytest
import scipy.linalg as sl

from paper_2205_08941_gb300 import inputs as I


def _params():
    keys = ["sss", "sps", "pps", "ppp", "sds", "pds", "pdp", "dds", "ddp", "ddd"]
    rng = np.random.default_rng(3)
    return dict(zip(keys, rng.normal(size=len(keys))))


def test_sk_rotation_reproduces_textbook_table():
    v = _params()
    model = I.SKModel(onsite={}, v=v, s=v, r_nn=1.0, decay=1e30, r_cut=1e9)
    rng = np.random.default_rng(4)
    d = rng.normal(size=(20, 3))
    _, h = I.sk_blocks(model, d, 9)
    r = np.linalg.norm(d, axis=1)
    l, m, n = (d / r[:, None]).T
    s3 = math.sqrt(3.0)
    # Slater & Koster (1954) two-centre table, a few representative entries
    assert np.allclose(h[:, 0, 0], v["sss"])
    assert np.allclose(h[:, 0, 1], l * v["sps"])
    assert np.allclose(h[:, 1, 0], -l * v["sps"])
    assert np.allclose(h[:, 1, 1], l * l * v["pps"] + (1 - l * l) * v["ppp"])
    assert np.allclose(h[:, 1, 2], l * m * (v["pps"] - v["ppp"]))
    assert np.allclose(h[:, 0, 4], s3 * l * m * v["sds"])
    assert np.allclose(h[:, 0, 8], (n * n - 0.5 * (l * l + m * m)) * v["sds"])
    assert np.allclose(h[:, 1, 4], s3 * l * l * m * v["pds"] + m * (1 - 2 * l * l) * v["pdp"])
    assert np.allclose(h[:, 3, 8], n * (n * n - 0.5 * (l * l + m * m)) * v["pds"]
                       + s3 * n * (l * l + m * m) * v["pdp"])
    assert np.allclose(h[:, 4, 4], 3 * l * l * m * m * v["dds"]
                       + (l * l + m * m - 4 * l * l * m * m) * v["ddp"]
                       + (n * n + l * l * m * m) * v["ddd"])
    assert np.allclose(h[:, 8, 8], (n * n - 0.5 * (l * l + m * m)) ** 2 * v["dds"]
                       + 3 * n * n * (l * l + m * m) * v["ddp"]
                       + 0.75 * (l * l + m * m) ** 2 * v["ddd"])
    # reversing the bond transposes the block
    _, hr = I.sk_blocks(model, -d, 9)
    assert np.allclose(hr, np.transpose(h, (0, 2, 1)))


@pytest.mark.parametrize("norb,rc", [(4, 10.0), (9, 14.0)])
def test_model_is_symmetric_gapped_and_well_conditioned(norb, rc):
    cell = I.diamond_cell(2, a=10.26, sigma=0.1, seed=1, norb=norb)
    S, H = I.overlap_hamiltonian(cell, I.silicon_model(rc))
    Sd, Hd = I.dense_from_pairs(cell, S), I.dense_from_pairs(cell, H)
    assert np.abs(Sd - Sd.T).max() < 1e-15 and np.abs(Hd - Hd.T).max() < 1e-15
    e = sl.eigh(Hd, Sd, eigvals_only=True)
    n_occ = 2 * cell.n_atoms
    assert e[n_occ] - e[n_occ - 1] > 0.1
    assert np.linalg.eigvalsh(Sd)[0] > 0.3


def test_random_blocks_symmetric_and_seeded():
    cell = I.diamond_cell(1, a=10.26, sigma=0.1, seed=1, norb=4)
    a = I.random_blocks(cell, 6.0, 9)
    b = I.random_blocks(cell, 6.0, 9)
    assert np.array_equal(a.values, b.values)
    d = I.dense_from_pairs(cell, a)
    assert np.array_equal(d, d.T)


@pytest.mark.parametrize("ncell,sigma,seed,ranges", [
    (2, 0.05, 1, (10.0, 12.0, 22.0, 32.0)),          # the 64-atom cell
    (8, 0.10, 2, (14.0, 16.0, 30.0, 44.0)),          # the 4096-atom benchmark cell
])
def test_no_pair_sits_on_a_cutoff(ncell, sigma, seed, ranges):
    """Pattern membership d^2 < R^2 must not hinge on rounding: no minimum-image pair
    distance of the seeded cells lies within 1e-9 bohr of a cutoff they are used with."""
    from scipy.spatial import cKDTree
    cell = I.diamond_cell(ncell, a=10.26, sigma=sigma, seed=seed, norb=9)
    tree = cKDTree(cell.pos % cell.box, boxsize=cell.box)
    d = tree.sparse_distance_matrix(tree, max(ranges) + 1.0, output_type="ndarray")["v"]
    for R in ranges:
        assert np.abs(d - R).min() > 1e-9, R
