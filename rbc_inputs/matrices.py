"""Seeded synthetic matrices A, B (Section 3: the paper uses only synthetic inputs).

All generators return float64 numpy arrays drawn from numpy's PCG64 with the
given seed, so the oracle (CPU) and the CUDA side (which copies them to the
device) see identical inputs.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(n: int, seed: int) -> np.ndarray:
    """i.i.d. standard normal entries ("Gaussian matrix", Section 3)."""
    return _rng(seed).standard_normal((n, n))


def uniform(n: int, seed: int) -> np.ndarray:
    """i.i.d. Uniform(0,1) entries ("uniform matrix", Section 3)."""
    return _rng(seed).random((n, n))


def scaled_hard(n: int, seed: int, which: str) -> np.ndarray:
    """Uniform[0,1] entries with rows (which='A') or columns (which='B') scaled by
    10^Uniform(-3, 3): the badly scaled case of the at-scale workloads."""
    g = _rng(seed)
    X = g.random((n, n))
    s = 10.0 ** g.uniform(-3.0, 3.0, size=n)
    return X * s[:, None] if which == "A" else X * s[None, :]


def adversarial(n: int, seed: int, kind: int):
    """Type 1/2/3 adversarial pairs (Section 3, Def. "Adversarial matrices"), with
    the 1-based index comparisons taken literally."""
    g = _rng(seed)
    i = np.arange(1, n + 1)[:, None] * np.ones((1, n))
    j = np.ones((n, 1)) * np.arange(1, n + 1)[None, :]
    ua, ub = g.random((n, n)), g.random((n, n))
    small, big = 1.0 / n**2, float(n) ** 2
    if kind == 1:
        A = np.where(j > n / 2, ua * small, ua)
        B = np.where(i < n / 2, ub * small, ub)
    elif kind == 2:
        A = np.where((i < n / 2) & (j > n / 2), ua * big, ua)
        B = np.where(j < n / 2, ub * small, ub)
    elif kind == 3:
        mask = ((i < n / 2) & (j > n / 2)) | ((i >= n / 2) & (j <= n / 2))
        A = np.where(mask, ua * small, ua)
        B = np.where(mask, ub * small, ub)
    else:
        raise ValueError(kind)
    return A, B


def hilbert(n: int) -> np.ndarray:
    """h_ij = 1/(i+j-1), 1-based (Section 3)."""
    i = np.arange(1, n + 1)
    return 1.0 / (i[:, None] + i[None, :] - 1.0)


def matrix_pair(dist: str, n: int, seed: int):
    """(A, B) for a named distribution: 'normal' | 'uniform' | 'hard' |
    'adv1' | 'adv2' | 'adv3' | 'hilbert'.  A uses `seed`, B uses `seed + 1`."""
    if dist == "normal":
        return gaussian(n, seed), gaussian(n, seed + 1)
    if dist == "uniform":
        return uniform(n, seed), uniform(n, seed + 1)
    if dist == "hard":
        return scaled_hard(n, seed, "A"), scaled_hard(n, seed + 1, "B")
    if dist in ("adv1", "adv2", "adv3"):
        return adversarial(n, seed, int(dist[-1]))
    if dist == "hilbert":
        H = hilbert(n)
        return H, H.copy()
    raise ValueError(f"unknown distribution {dist!r}")
