"""Oracle of the learned initial guess: pair frames, descriptors, frame rotations of L blocks
and the MLP (forward and backward) in plain numpy FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The definitions follow the library's
stated design (pair frame, 64-number descriptor, 64-256-256-256-81 SiLU network, MSE on
normalised targets); they are restated here from that definition, not shared.  Pinned by
tests/test_oracle_guess.py: frame orthonormality, exact round trip of the frame rotation,
invariance of descriptors and targets under a cubic rotation of the cell, and
finite-difference gradients of the network.
"""
from __future__ import annotations

import math

import numpy as np

DIMS = (64, 256, 256, 256, 81)


def pairs_of(p):
    """Block indices b = (i, j) of the oracle pattern p with i <= j, in block order."""
    return np.nonzero(p.row <= p.col)[0]


def _mi(pos, box, i, j):
    d = pos[j] - pos[i]
    return d - box * np.rint(d / box)


def frame_and_descriptor(p, b):
    """(3x3 frame rows e1, e2, e3; 64 descriptor values) of pair block b of pattern p."""
    pos, box = p.pos, p.box
    i, j = int(p.row[b]), int(p.col[b])
    row = p.col[p.rp[i]:p.rp[i + 1]]
    if i != j:
        dij = _mi(pos, box, i, j)
        e3 = dij / np.linalg.norm(dij)
        m = 0.5 * dij
    else:
        dij = np.zeros(3)
        best, kb, e3 = None, None, np.array([0.0, 0.0, 1.0])
        for k in row:
            if k == i:
                continue
            d = _mi(pos, box, i, k)
            r2 = float(d @ d)
            if best is None or r2 < best or (r2 == best and k < kb):
                best, kb, e3 = r2, k, d
        e3 = e3 / np.linalg.norm(e3)
        m = np.zeros(3)
    best, kb, e1 = None, None, None
    for k in row:
        if k == i or k == j:
            continue
        w = _mi(pos, box, i, k) - m
        perp = w - (w @ e3) * e3
        pn = np.linalg.norm(perp)
        if pn < 1e-6:
            continue
        r2 = float(w @ w)
        if best is None or r2 < best or (r2 == best and k < kb):
            best, kb, e1 = r2, k, perp / pn
    if e1 is None:
        h = np.array([1.0, 0.0, 0.0]) if abs(e3[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        e1 = h - (h @ e3) * e3
        e1 /= np.linalg.norm(e1)
    e2 = np.cross(e3, e1)
    frame = np.stack([e1, e2, e3])
    f = np.zeros(64)
    rij = float(np.linalg.norm(dij))
    for q in range(10):
        f[q] = math.exp(-0.5 * ((rij - 1.6 * q) / 1.6) ** 2)
    for k in row:
        if k == i or k == j:
            continue
        w = _mi(pos, box, i, k) - m
        rho = float(np.linalg.norm(w))
        if rho >= 8.0 or rho < 1e-6:
            continue
        x, y, z = frame @ w / rho
        ang = [1.0, z, x, y, 0.5 * (3 * z * z - 1), x * z, y * z, 0.5 * (x * x - y * y), x * y]
        fc = 0.5 * (1.0 + math.cos(math.pi * rho / 8.0))
        for n in range(6):
            h = math.exp(-0.5 * ((rho - 1.6 * n) / 1.2) ** 2) * fc
            for a in range(9):
                f[10 + 9 * n + a] += h * ang[a]
    return frame, f


def d_shell_rotation(frame):
    """5x5 rotation of the real d orbitals (xy, yz, zx, x2-y2, 3z2-r2) for frame rows R:
    entry (a, b) = <Q_b, R^T Q_a R> with Q the unit-norm quadratic forms of the orbitals."""
    s = 1.0 / math.sqrt(2.0)
    Q = np.zeros((5, 3, 3))
    Q[0][0, 1] = Q[0][1, 0] = s
    Q[1][1, 2] = Q[1][2, 1] = s
    Q[2][0, 2] = Q[2][2, 0] = s
    Q[3][0, 0], Q[3][1, 1] = s, -s
    Q[4][0, 0] = Q[4][1, 1] = -1.0 / math.sqrt(6.0)
    Q[4][2, 2] = 2.0 / math.sqrt(6.0)
    out = np.zeros((5, 5))
    for a in range(5):
        t = frame.T @ Q[a] @ frame
        for b in range(5):
            out[a, b] = float(np.sum(Q[b] * t))
    return out


def orbital_rotation(frame, nb):
    D = np.zeros((nb, nb))
    D[0, 0] = 1.0
    D[1:4, 1:4] = frame
    if nb == 9:
        D[4:9, 4:9] = d_shell_rotation(frame)
    return D


def block(p, vals, b):
    n = int(p.nb[p.row[b]])
    return vals[p.off[b]:p.off[b + 1]].reshape(n, n)


def target(frame, blk):
    """81 numbers: the block in the pair frame, D L D^T, zero-padded to 9 x 9."""
    nb = blk.shape[0]
    D = orbital_rotation(frame, nb)
    out = np.zeros((9, 9))
    out[:nb, :nb] = D @ blk @ D.T
    return out.reshape(-1)


def untarget(frame, t81, nb):
    """Inverse of target(): the global block D^T L_loc D."""
    D = orbital_rotation(frame, nb)
    return D.T @ t81.reshape(9, 9)[:nb, :nb] @ D


# ------------------------------------------------------------------ network (FP64)

def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def unpack(w, b):
    """Weights (in x out, row-major) and biases of each layer from the packed arrays."""
    Ws, bs, ow, ob = [], [], 0, 0
    for k in range(len(DIMS) - 1):
        n_in, n_out = DIMS[k], DIMS[k + 1]
        Ws.append(np.asarray(w[ow:ow + n_in * n_out], dtype=np.float64).reshape(n_in, n_out))
        bs.append(np.asarray(b[ob:ob + n_out], dtype=np.float64))
        ow += n_in * n_out
        ob += n_out
    return Ws, bs


def forward(w, b, X, in_mean, in_scale):
    """Normalised outputs and the per-layer (Z, H) of the network on raw descriptors X."""
    Ws, bs = unpack(w, b)
    H = (np.asarray(X, dtype=np.float64) - in_mean) / in_scale
    cache = [(None, H)]
    for k, (W, bb) in enumerate(zip(Ws, bs)):
        Z = H @ W + bb
        H = silu(Z) if k + 1 < len(Ws) else Z
        cache.append((Z, H))
    return H, cache


def loss_and_grads(w, b, X, T, in_mean, in_scale, out_mean, out_scale):
    """Mean-square error on normalised targets and its gradients (packed like w, b)."""
    Y, cache = forward(w, b, X, in_mean, in_scale)
    Tn = (np.asarray(T, dtype=np.float64) - out_mean) / out_scale
    diff = Y - Tn
    loss = float(np.mean(diff ** 2))
    Ws, _ = unpack(w, b)
    dZ = 2.0 * diff / diff.size
    gws, gbs = [None] * len(Ws), [None] * len(Ws)
    for k in range(len(Ws) - 1, -1, -1):
        H_prev = cache[k][1]
        gws[k] = H_prev.T @ dZ
        gbs[k] = dZ.sum(axis=0)
        if k > 0:
            dZ = (dZ @ Ws[k].T) * silu_grad(cache[k][0])
    return loss, np.concatenate([g.reshape(-1) for g in gws]), np.concatenate(gbs)
