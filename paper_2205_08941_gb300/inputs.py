"""Seeded synthetic inputs: diamond-silicon cells and a two-centre tight-binding model.

This module generates the *inputs* of the linear-scaling solver and nothing else: atomic
positions, the orbital count per atom, and the Gamma-point overlap S and Hamiltonian H of a
Slater-Koster two-centre model, as coordinate lists of atom-pair blocks.  It performs none of
the solver's arithmetic (no sparsity pattern, no block product, no trace); both the CUDA path
and the CPU oracle take its output and scatter it into their own pattern storage.

The paper's workloads are bulk silicon (Background; Fig. 2c).  Neither the paper nor the
solver fixes the integrals, so the model here is a synthetic stand-in chosen to be gapped
(the linear-scaling solver is unsuitable for metals, Development Priorities):

* diamond lattice, conventional cubic cell of side ``a`` with 8 sites, atoms ordered by cell
  (ix, iy, iz) row-major, then by site; each coordinate displaced by a seeded normal deviate;
* orbitals per atom: 4 (s, p) or 9 (s, p, d: "SZP"); real orbitals in the order
  s, px, py, pz, dxy, dyz, dzx, dx2-y2, d3z2-r2;
* bond integrals V(r) = V0 * exp(-(r - r_nn)/2) * f(r) with a cosine cut f over the last
  2 bohr before r_c; overlaps of the same angular form;
* Gamma folding: each (i, j) block is the sum over the periodic images of j closer than r_c.

Units: bohr and hartree.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

EV = 1.0 / 27.211386245988  # hartree per eV

# Diamond conventional cell: FCC sites plus the same shifted by (1/4, 1/4, 1/4).
_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
DIAMOND_SITES = np.concatenate([_FCC, _FCC + 0.25], axis=0)


@dataclasses.dataclass
class Cell:
    """Atoms in an orthorhombic periodic box (bohr)."""

    pos: np.ndarray   # (N, 3) float64, wrapped into [0, box)
    box: np.ndarray   # (3,) float64
    nb: np.ndarray    # (N,) int32 orbitals per atom

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_orb(self) -> int:
        return int(self.nb.sum())


def diamond_cell(ncell, a: float = 10.26, sigma: float = 0.0, seed: int = 0,
                 norb: int = 4) -> Cell:
    """ncell^3 (or ncell = (nx, ny, nz)) conventional diamond cells, seeded N(0, sigma) jitter."""
    if np.isscalar(ncell):
        ncell = (int(ncell),) * 3
    nx, ny, nz = ncell
    idx = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"),
                   axis=-1).reshape(-1, 3).astype(np.float64)
    frac = (idx[:, None, :] + DIAMOND_SITES[None, :, :]).reshape(-1, 3)
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    pos = frac * a
    rng = np.random.default_rng(seed)
    if sigma > 0.0:
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    pos = np.mod(pos, box)
    nb = np.full(pos.shape[0], norb, dtype=np.int32)
    return Cell(pos=pos, box=box, nb=nb)


@dataclasses.dataclass
class SKModel:
    """Two-centre Slater-Koster parameters (hartree); overlap integrals are dimensionless."""

    onsite: dict            # {"s": E_s, "p": E_p, "d": E_d}
    v: dict                 # bond integrals at r_nn, e.g. {"sss": ..., "sps": ..., ...}
    s: dict                 # overlap integrals at r_nn, same keys
    r_nn: float = 4.443
    decay: float = 2.0
    r_cut: float = 10.0
    cut_width: float = 2.0


def silicon_model(r_cut: float = 10.0) -> SKModel:
    """The gapped synthetic Si model (sp part from Harrison-like ratios, d shell well above)."""
    v = {
        "sss": 2 * -1.93 * EV, "sps": 2 * 2.54 * EV, "pps": 2 * 4.47 * EV, "ppp": 2 * -1.12 * EV,
        "sds": 2 * -1.20 * EV, "pds": 2 * -1.40 * EV, "pdp": 2 * 0.70 * EV,
        "dds": 2 * -1.00 * EV, "ddp": 2 * 0.60 * EV, "ddd": 2 * -0.15 * EV,
    }
    s = {k: -0.1 * val / v["pps"] for k, val in v.items()}
    onsite = {"s": -8.0 * EV, "p": -8.0 * EV, "d": 6.0 * EV}
    return SKModel(onsite=onsite, v=v, s=s, r_cut=r_cut)


def _cutoff(r, r_cut, width):
    x = (r - (r_cut - width)) / width
    f = 0.5 * (1.0 + np.cos(np.pi * np.clip(x, 0.0, 1.0)))
    return np.where(r < r_cut, f, 0.0)


def _frames(u):
    """Rows e1, e2, e3 of a rotation with e3 = u (unit vectors, shape (P, 3))."""
    helper = np.where(np.abs(u[:, 0:1]) < 0.9, np.array([[1.0, 0.0, 0.0]]),
                      np.array([[0.0, 1.0, 0.0]]))
    e1 = np.cross(helper, u)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(u, e1)
    return np.stack([e1, e2, u], axis=1)  # (P, 3, 3)


# Real d orbitals as unit-Frobenius quadratic forms, order xy, yz, zx, x2-y2, 3z2-r2.
def _dforms():
    q = np.zeros((5, 3, 3))
    r2 = 1.0 / math.sqrt(2.0)
    q[0, 0, 1] = q[0, 1, 0] = r2
    q[1, 1, 2] = q[1, 2, 1] = r2
    q[2, 2, 0] = q[2, 0, 2] = r2
    q[3, 0, 0], q[3, 1, 1] = r2, -r2
    q[4, 0, 0] = q[4, 1, 1] = -1.0 / math.sqrt(6.0)
    q[4, 2, 2] = 2.0 / math.sqrt(6.0)
    return q


_DQ = _dforms()


def orbital_rotation(rot):
    """Block-diagonal map local->global orbitals, (P, 9, 9): D[a, b] = <local a | global b>."""
    p = rot.shape[0]
    d = np.zeros((p, 9, 9))
    d[:, 0, 0] = 1.0
    d[:, 1:4, 1:4] = rot
    # local quadratic form Q_a expressed in global coordinates is R^T Q_a R
    qg = np.einsum("pji,ajk,pkl->pail", rot, _DQ, rot)
    d[:, 4:9, 4:9] = np.einsum("pail,bil->pab", qg, _DQ)
    return d


def _bond_frame_matrix(par, scale):
    """Two-centre matrix in the bond frame (bond along +z from atom i to atom j), (P, 9, 9).

    Local order s, px, py, pz, dxy, dyz, dzx, dx2-y2, dz2; only equal |m| couple.  Parity:
    element (a, b) for the reversed bond is (-1)^(l_a + l_b) times the forward one, so
    the (p, s) and (d, p) elements carry the opposite sign of (s, p) and (p, d).
    """
    p = scale.shape[0]
    m = np.zeros((p, 9, 9))
    s, px, py, pz, dxy, dyz, dzx, dx2, dz2 = range(9)
    m[:, s, s] = par["sss"]
    m[:, s, pz] = par["sps"]
    m[:, pz, s] = -par["sps"]
    m[:, s, dz2] = par["sds"]
    m[:, dz2, s] = par["sds"]
    m[:, pz, pz] = par["pps"]
    m[:, px, px] = par["ppp"]
    m[:, py, py] = par["ppp"]
    m[:, pz, dz2] = par["pds"]
    m[:, dz2, pz] = -par["pds"]
    m[:, px, dzx] = par["pdp"]
    m[:, dzx, px] = -par["pdp"]
    m[:, py, dyz] = par["pdp"]
    m[:, dyz, py] = -par["pdp"]
    m[:, dz2, dz2] = par["dds"]
    m[:, dzx, dzx] = par["ddp"]
    m[:, dyz, dyz] = par["ddp"]
    m[:, dxy, dxy] = par["ddd"]
    m[:, dx2, dx2] = par["ddd"]
    return m * scale[:, None, None]


def sk_blocks(model: SKModel, disp: np.ndarray, norb: int = 9):
    """S and H blocks (P, norb, norb) for displacement vectors disp = r_j - r_i (P, 3), r > 0."""
    r = np.linalg.norm(disp, axis=1)
    u = disp / r[:, None]
    radial = np.exp(-(r - model.r_nn) / model.decay) * _cutoff(r, model.r_cut, model.cut_width)
    d = orbital_rotation(_frames(u))
    hb = np.einsum("pab,pac,pcd->pbd", d, _bond_frame_matrix(model.v, radial), d)
    sb = np.einsum("pab,pac,pcd->pbd", d, _bond_frame_matrix(model.s, radial), d)
    return sb[:, :norb, :norb], hb[:, :norb, :norb]


@dataclasses.dataclass
class PairBlocks:
    """Coordinate list of atom-pair blocks, sorted by (i, j); block b is
    values[off[b] : off[b] + nb[i]*nb[j]] in row-major (nb[i], nb[j]) order."""

    i: np.ndarray       # (P,) int32
    j: np.ndarray       # (P,) int32
    off: np.ndarray     # (P + 1,) int64
    values: np.ndarray  # (off[-1],) float64

    @property
    def n_pairs(self) -> int:
        return int(self.i.shape[0])


def _min_image(d, box):
    return d - box * np.rint(d / box)


def neighbour_pairs(cell: Cell, r: float, chunk: int = 256):
    """Ordered pairs (i, j), i == j included, whose minimum-image distance is below r.

    Returns (i, j, disp) sorted by (i, j); disp = minimum-image r_j - r_i.
    """
    pos, box = cell.pos, cell.box
    n = pos.shape[0]
    ii, jj, dd = [], [], []
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d = _min_image(pos[None, :, :] - pos[s:e, None, :], box)
        d2 = (d * d).sum(axis=2)
        a, b = np.nonzero(d2 < r * r)
        ii.append(a + s)
        jj.append(b)
        dd.append(d[a, b])
    return (np.concatenate(ii).astype(np.int32), np.concatenate(jj).astype(np.int32),
            np.concatenate(dd))


def _pack(i, j, nb, blocks_of_pair):
    sizes = nb[i].astype(np.int64) * nb[j].astype(np.int64)
    off = np.zeros(i.shape[0] + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return PairBlocks(i=i, j=j, off=off, values=blocks_of_pair)


def overlap_hamiltonian(cell: Cell, model: SKModel):
    """Gamma-folded S and H of the two-centre model as PairBlocks over pairs closer than r_c.

    All atoms must carry the same orbital count (4 or 9).
    """
    nb = cell.nb
    norb = int(nb[0])
    if not np.all(nb == norb) or norb not in (4, 9):
        raise ValueError("overlap_hamiltonian supports a uniform 4- or 9-orbital basis")
    i, j, d0 = neighbour_pairs(cell, model.r_cut)
    p = i.shape[0]
    s_blk = np.zeros((p, norb, norb))
    h_blk = np.zeros((p, norb, norb))
    n_img = [int(math.ceil(model.r_cut / b)) for b in cell.box]
    for sx in range(-n_img[0], n_img[0] + 1):
        for sy in range(-n_img[1], n_img[1] + 1):
            for sz in range(-n_img[2], n_img[2] + 1):
                shift = np.array([sx, sy, sz], dtype=np.float64) * cell.box
                disp = d0 + shift
                r = np.linalg.norm(disp, axis=1)
                sel = np.nonzero((r < model.r_cut) & (r > 1e-12))[0]
                if sel.size == 0:
                    continue
                sb, hb = sk_blocks(model, disp[sel], norb)
                s_blk[sel] += sb
                h_blk[sel] += hb
    diag = np.nonzero(i == j)[0]
    e = np.array([model.onsite["s"]] + [model.onsite["p"]] * 3 + [model.onsite["d"]] * 5)[:norb]
    s_blk[diag] += np.eye(norb)
    h_blk[diag] += np.diag(e)
    return (_pack(i, j, nb, s_blk.reshape(-1)), _pack(i, j, nb, h_blk.reshape(-1)))


def random_blocks(cell: Cell, r: float, seed: int, decay: float = 4.0,
                  symmetric: bool = True) -> PairBlocks:
    """Seeded N(0,1) * exp(-r_ij/decay) blocks on all pairs closer than r.

    symmetric=True makes block (j, i) the transpose of block (i, j).
    """
    i, j, d = neighbour_pairs(cell, r)
    nb = cell.nb
    rng = np.random.default_rng(seed)
    sizes = nb[i].astype(np.int64) * nb[j].astype(np.int64)
    off = np.zeros(i.shape[0] + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    vals = rng.standard_normal(int(off[-1]))
    w = np.exp(-np.linalg.norm(d, axis=1) / decay)
    vals *= np.repeat(w, sizes)
    if symmetric:
        key = i.astype(np.int64) * cell.n_atoms + j
        tkey = j.astype(np.int64) * cell.n_atoms + i
        tpos = np.searchsorted(key, tkey)
        for b in np.nonzero(i > j)[0]:
            t = tpos[b]
            ni, nj = int(nb[i[b]]), int(nb[j[b]])
            vals[off[b]:off[b + 1]] = vals[off[t]:off[t + 1]].reshape(nj, ni).T.reshape(-1)
        for b in np.nonzero(i == j)[0]:
            n_ = int(nb[i[b]])
            blk = vals[off[b]:off[b + 1]].reshape(n_, n_)
            vals[off[b]:off[b + 1]] = (0.5 * (blk + blk.T)).reshape(-1)
    return PairBlocks(i=i, j=j, off=off, values=vals)


def dense_from_pairs(cell: Cell, pb: PairBlocks) -> np.ndarray:
    """Scatter PairBlocks into a dense (n_orb, n_orb) matrix (tests and tiny cells only)."""
    nb = cell.nb.astype(np.int64)
    o = np.zeros(nb.shape[0] + 1, dtype=np.int64)
    np.cumsum(nb, out=o[1:])
    m = np.zeros((int(o[-1]), int(o[-1])))
    for b in range(pb.n_pairs):
        i, j = int(pb.i[b]), int(pb.j[b])
        m[o[i]:o[i + 1], o[j]:o[j + 1]] = pb.values[pb.off[b]:pb.off[b + 1]].reshape(
            nb[i], nb[j])
    return m


def write_fixture(path: str, cell: Cell, **pair_lists: PairBlocks) -> None:
    """Save a cell and its pair lists to a .npz file that both paths can read."""
    arrays = {"pos": cell.pos, "box": cell.box, "nb": cell.nb}
    for name, pb in pair_lists.items():
        arrays[f"{name}_i"] = pb.i
        arrays[f"{name}_j"] = pb.j
        arrays[f"{name}_off"] = pb.off
        arrays[f"{name}_values"] = pb.values
    np.savez(path, **arrays)


# ---------------------------------------------------------------------------------------
# Mixed species (batched heterogeneous cells): 5-orbital sp3s*, 9-orbital spd and
# 13-orbital s p s* p* d atoms, all with four valence electrons.
# ---------------------------------------------------------------------------------------

# shells of each species: (label, l); orbitals follow shell order, m order as above
SPECIES = {
    5: [("s", 0), ("p", 1), ("s*", 0)],
    9: [("s", 0), ("p", 1), ("d", 2)],
    13: [("s", 0), ("p", 1), ("s*", 0), ("p*", 1), ("d", 2)],
}
SHELL_ONSITE_EV = {"s": -8.0, "p": -8.0, "d": 6.0, "s*": 4.0, "p*": 6.0}
SHELL_SCALE = {"s": 1.0, "p": 1.0, "d": 1.0, "s*": 0.6, "p*": 0.5}
_LKEY = {(0, 0): "ss", (0, 1): "sp", (1, 1): "pp", (0, 2): "sd", (1, 2): "pd", (2, 2): "dd"}
_MSYM = {0: "s", 1: "p", 2: "d"}
# local bond-frame orbitals of a shell: symmetry (|m|, partner tag) per component
_LOCAL = {0: [(0, "z")], 1: [(1, "x"), (1, "y"), (0, "z")],
          2: [(2, "xy"), (1, "y"), (1, "x"), (2, "x2"), (0, "z")]}


def _shell_rotation(l, rot):
    if l == 0:
        return np.ones((rot.shape[0], 1, 1))
    if l == 1:
        return rot
    qg = np.einsum("pji,ajk,pkl->pail", rot, _DQ, rot)
    return np.einsum("pail,bil->pab", qg, _DQ)


def species_blocks(model: SKModel, disp: np.ndarray, sa: int, sb: int, which: str):
    """Two-centre blocks (P, nb_a, nb_b) between species sa (at the origin) and sb (at disp),
    `which` = "v" (hamiltonian) or "s" (overlap).  Shell pairs couple through the bond
    integral of their l pair scaled by both shells' factors; the (l_a > l_b) element carries
    the parity sign (-1)^(l_a + l_b)."""
    par = model.v if which == "v" else model.s
    r = np.linalg.norm(disp, axis=1)
    rot = _frames(disp / r[:, None])
    radial = np.exp(-(r - model.r_nn) / model.decay) * _cutoff(r, model.r_cut, model.cut_width)
    p = disp.shape[0]
    out = np.zeros((p, sa, sb))
    oa = 0
    for la_name, la in SPECIES[sa]:
        da = _shell_rotation(la, rot)
        ob = 0
        for lb_name, lb in SPECIES[sb]:
            db = _shell_rotation(lb, rot)
            lo, hi = min(la, lb), max(la, lb)
            key = _LKEY[(lo, hi)]
            sign = (-1.0) ** (la + lb) if la > lb else 1.0
            scale = SHELL_SCALE[la_name] * SHELL_SCALE[lb_name] * sign
            m0 = np.zeros((2 * la + 1, 2 * lb + 1))
            for ia, (ma, ta) in enumerate(_LOCAL[la]):
                for ib, (mb, tb) in enumerate(_LOCAL[lb]):
                    # only components of equal |m| and equal orientation couple
                    if ma != mb or ta != tb:
                        continue
                    m0[ia, ib] = par[key + "spd"[ma]] * scale
            blk = np.einsum("pab,ac,pcd->pbd", da, m0, db) * radial[:, None, None]
            out[:, oa:oa + 2 * la + 1, ob:ob + 2 * lb + 1] = blk
            ob += 2 * lb + 1
        oa += 2 * la + 1
    return out


def species_onsite(nb: int) -> np.ndarray:
    e = []
    for name, l in SPECIES[nb]:
        e += [SHELL_ONSITE_EV[name] * EV] * (2 * l + 1)
    return np.array(e)


def overlap_hamiltonian_species(cell: Cell, model: SKModel):
    """Gamma-folded S and H for cells whose atoms carry 5, 9 or 13 orbitals (PairBlocks).

    Blocks (i, j) with i <= j are computed; (j, i) is their transpose."""
    i, j, d0 = neighbour_pairs(cell, model.r_cut)
    nb = cell.nb
    sizes = nb[i].astype(np.int64) * nb[j].astype(np.int64)
    off = np.zeros(i.shape[0] + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    s_val, h_val = np.zeros(int(off[-1])), np.zeros(int(off[-1]))
    n_img = [int(math.ceil(model.r_cut / b)) for b in cell.box]
    upper = np.nonzero(i <= j)[0]
    blocks_s, blocks_h = {}, {}
    for sa in SPECIES:
        for sb in SPECIES:
            sel = upper[(nb[i[upper]] == sa) & (nb[j[upper]] == sb)]
            if sel.size == 0:
                continue
            bs = np.zeros((sel.size, sa, sb))
            bh = np.zeros((sel.size, sa, sb))
            for sx in range(-n_img[0], n_img[0] + 1):
                for sy in range(-n_img[1], n_img[1] + 1):
                    for sz in range(-n_img[2], n_img[2] + 1):
                        disp = d0[sel] + np.array([sx, sy, sz], dtype=np.float64) * cell.box
                        r = np.linalg.norm(disp, axis=1)
                        m = np.nonzero((r < model.r_cut) & (r > 1e-12))[0]
                        if m.size == 0:
                            continue
                        bs[m] += species_blocks(model, disp[m], sa, sb, "s")
                        bh[m] += species_blocks(model, disp[m], sa, sb, "v")
            diag = np.nonzero(i[sel] == j[sel])[0]
            if diag.size:
                bs[diag] += np.eye(sa)
                bh[diag] += np.diag(species_onsite(sa))
            for q, b in enumerate(sel):
                blocks_s[b] = bs[q]
                blocks_h[b] = bh[q]
    key = i.astype(np.int64) * cell.n_atoms + j
    tpos = np.searchsorted(key, j.astype(np.int64) * cell.n_atoms + i)
    for b in range(i.shape[0]):
        if i[b] <= j[b]:
            s_blk, h_blk = blocks_s[b], blocks_h[b]
        else:
            s_blk, h_blk = blocks_s[tpos[b]].T, blocks_h[tpos[b]].T
        s_val[off[b]:off[b + 1]] = s_blk.reshape(-1)
        h_val[off[b]:off[b + 1]] = h_blk.reshape(-1)
    return PairBlocks(i=i, j=j, off=off, values=s_val), PairBlocks(i=i, j=j, off=off, values=h_val)


def mixed_cell(ncell, density_per_A3: float, sigma: float, seed: int,
               species=(5, 9, 13)) -> Cell:
    """Diamond lattice scaled to a density (atoms per cubic angstrom) with species drawn per
    atom from `species` (seeded)."""
    a = (8.0 / (density_per_A3 / 1.8897261254578281 ** 3)) ** (1.0 / 3.0)
    cell = diamond_cell(ncell, a=a, sigma=sigma, seed=seed, norb=9)
    rng = np.random.default_rng(seed + 7919)
    cell.nb = rng.choice(np.array(species, dtype=np.int32), size=cell.n_atoms)
    return cell


def concat_cells(cells):
    """Atoms of several cells back to back: positions, nb, atom prefix, boxes (per cell)."""
    pos = np.concatenate([c.pos for c in cells])
    nb = np.concatenate([c.nb for c in cells]).astype(np.int32)
    start = np.zeros(len(cells) + 1, dtype=np.int32)
    np.cumsum([c.n_atoms for c in cells], out=start[1:])
    boxes = np.stack([c.box for c in cells])
    return pos, nb, start, boxes
