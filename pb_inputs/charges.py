"""Seeded synthetic solutes: point-charge sets and protein-like atom chains.

A charge set is an (Nc, 4) float64 array of rows (x, y, z, Q) with positions in
Angstrom and Q in units of the elementary charge e_c (Section 1: the solute is a
set of Nc point charges Q_i at positions x_i).
"""
from __future__ import annotations

import numpy as np


def ball_charges(n: int, radius: float, seed: int, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """``n`` charges uniform in the ball of the given radius, Q ~ U[-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    q = rng.uniform(-1.0, 1.0, size=n)
    out = np.empty((n, 4))
    out[:, :3] = d * r[:, None] + np.asarray(center, dtype=np.float64)
    out[:, 3] = q
    return out


def helix_charges(step: float = np.pi / 4, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """The nine-charge helix of the spherical-cavity test (Section 3.2):
    positions r(t) = ((3/(4 pi)) cos t, (3/(4 pi)) sin t, t/pi) for t = 0, step, ..., 2 pi,
    charges 0.1, 0.2, ..., 0.9 e_c.  Nine points need step = pi/4."""
    t = np.arange(0.0, 2 * np.pi + 1e-12, step)
    out = np.empty((t.size, 4))
    out[:, 0] = 3.0 / (4.0 * np.pi) * np.cos(t)
    out[:, 1] = 3.0 / (4.0 * np.pi) * np.sin(t)
    out[:, 2] = t / np.pi
    out[:, :3] += np.asarray(center, dtype=np.float64)
    out[:, 3] = 0.1 * np.arange(1, t.size + 1)
    return out


def compact_chain(n_atoms: int, seed: int, step: float = 3.8, min_sep: float = 3.0,
                  bias: float = 0.35, max_tries: int = 200):
    """A seeded compact random chain standing in for a protein backbone.

    Consecutive atoms are ``step`` apart; a move is rejected if it comes closer
    than ``min_sep`` to any earlier atom; each direction is drawn uniformly on the
    sphere and pulled toward the running centre of mass with weight ``bias``.
    Radii ~ U[1.5, 2.0]; partial charges ~ N(0, 0.3) shifted so that the net
    charge is an integer.  Returns (positions (n,3), radii (n,), charges (n,)).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = np.zeros((n_atoms, 3))
    k = 1
    while k < n_atoms:
        com = pos[:k].mean(0)
        placed = False
        for _ in range(max_tries):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            to_c = com - pos[k - 1]
            nc = np.linalg.norm(to_c)
            if nc > 1e-9:
                d = d + bias * to_c / nc
                d /= np.linalg.norm(d)
            cand = pos[k - 1] + step * d
            d2 = np.sum((pos[:k] - cand) ** 2, axis=1)
            if np.all(d2 >= min_sep * min_sep):
                pos[k] = cand
                placed = True
                break
        if placed:
            k += 1
        else:
            k = max(1, k - 1)   # dead end: back up one atom
    radii = rng.uniform(1.5, 2.0, size=n_atoms)
    q = rng.normal(0.0, 0.3, size=n_atoms)
    q -= (q.sum() - np.round(q.sum())) / n_atoms
    return pos, radii, q


def charge_variants(charges: np.ndarray, n_variants: int, seed: int, frac: float = 0.05,
                    delta: float = 0.5) -> np.ndarray:
    """Right-hand-side variants of one charge set: each variant changes the charge
    of a seeded ``frac`` of the atoms by +delta or -delta.  Returns (R, Nc, 4);
    variant 0 is the unmodified set."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = charges.shape[0]
    out = np.repeat(charges[None, :, :], n_variants, axis=0).copy()
    m = max(1, int(round(frac * nc)))
    for r in range(1, n_variants):
        idx = rng.choice(nc, size=m, replace=False)
        out[r, idx, 3] += rng.choice([-delta, delta], size=m)
    return out
