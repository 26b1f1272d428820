"""Coefficient tensors (U, V, W) of bilinear formulas for n0 x n0 block products.

Every tensor is a float64 array of shape (n0, n0, R), indexed [k, l, r] for U
(coefficient of A_kl in product r), [k', l', r] for V (coefficient of B_k'l')
and [i, j, r] for W (coefficient of product r in C_ij), all 0-based.  This is
the layout of the bilinear computation of Section 1, Eq. (1).

Strassen (1969, R = 7) and Laderman (1976, R = 23) are entered from the
original publications' well-known product lists; whether a tensor triple is an
exact bilinear computation is *not* asserted here -- the oracle checks Eq. (3)
by brute force.
"""
from __future__ import annotations

import re

import numpy as np


def _parse_terms(expr: str, letter: str, n0: int) -> np.ndarray:
    """'a11+a22-a12' -> n0 x n0 coefficient matrix (1-based indices in text)."""
    out = np.zeros((n0, n0))
    for sign, i, j in re.findall(r"([+-]?)\s*%s(\d)(\d)" % letter, expr.replace(" ", "")):
        out[int(i) - 1, int(j) - 1] += -1.0 if sign == "-" else 1.0
    return out


def _from_lists(n0: int, products: list[tuple[str, str]], outputs: dict[str, str]):
    R = len(products)
    U = np.zeros((n0, n0, R))
    V = np.zeros((n0, n0, R))
    W = np.zeros((n0, n0, R))
    for r, (ua, vb) in enumerate(products):
        U[:, :, r] = _parse_terms(ua, "a", n0)
        V[:, :, r] = _parse_terms(vb, "b", n0)
    for cij, expr in outputs.items():
        i, j = int(cij[1]) - 1, int(cij[2]) - 1
        for sign, r in re.findall(r"([+-]?)\s*m(\d+)", expr.replace(" ", "")):
            W[i, j, int(r) - 1] += -1.0 if sign == "-" else 1.0
    return U, V, W


def strassen():
    """Strassen's 2x2 formula with 7 products (Section 1 names it; textbook form)."""
    products = [
        ("a11+a22", "b11+b22"),
        ("a21+a22", "b11"),
        ("a11", "b12-b22"),
        ("a22", "b21-b11"),
        ("a11+a12", "b22"),
        ("a21-a11", "b11+b12"),
        ("a12-a22", "b21+b22"),
    ]
    outputs = {
        "c11": "m1+m4-m5+m7",
        "c12": "m3+m5",
        "c21": "m2+m4",
        "c22": "m1-m2+m3+m6",
    }
    return _from_lists(2, products, outputs)


def laderman():
    """Laderman's 3x3 formula with 23 products (Section 1 names it)."""
    products = [
        ("a11+a12+a13-a21-a22-a32-a33", "b22"),
        ("a11-a21", "-b12+b22"),
        ("a22", "-b11+b12+b21-b22-b23-b31+b33"),
        ("-a11+a21+a22", "b11-b12+b22"),
        ("a21+a22", "-b11+b12"),
        ("a11", "b11"),
        ("-a11+a31+a32", "b11-b13+b23"),
        ("-a11+a31", "b13-b23"),
        ("a31+a32", "-b11+b13"),
        ("a11+a12+a13-a22-a23-a31-a32", "b23"),
        ("a32", "-b11+b13+b21-b22-b23-b31+b32"),
        ("-a13+a32+a33", "b22+b31-b32"),
        ("a13-a33", "b22-b32"),
        ("a13", "b31"),
        ("a32+a33", "-b31+b32"),
        ("-a13+a22+a23", "b23+b31-b33"),
        ("a13-a23", "b23-b33"),
        ("a22+a23", "-b31+b33"),
        ("a12", "b21"),
        ("a23", "b32"),
        ("a21", "b13"),
        ("a31", "b12"),
        ("a33", "b33"),
    ]
    outputs = {
        "c11": "m6+m14+m19",
        "c12": "m1+m4+m5+m6+m12+m14+m15",
        "c13": "m6+m7+m9+m10+m14+m16+m18",
        "c21": "m2+m3+m4+m6+m14+m16+m17",
        "c22": "m2+m4+m5+m6+m20",
        "c23": "m14+m16+m17+m18+m21",
        "c31": "m6+m7+m8+m11+m12+m13+m14",
        "c32": "m12+m13+m14+m15+m22",
        "c33": "m6+m7+m8+m9+m23",
    }
    return _from_lists(3, products, outputs)


def classical_formula(n0: int):
    """The standard n0^3-product formula: product r = (i, l, j) is a_il * b_lj into c_ij."""
    R = n0 ** 3
    U = np.zeros((n0, n0, R))
    V = np.zeros((n0, n0, R))
    W = np.zeros((n0, n0, R))
    r = 0
    for i in range(n0):
        for l in range(n0):
            for j in range(n0):
                U[i, l, r] = 1.0
                V[l, j, r] = 1.0
                W[i, j, r] = 1.0
                r += 1
    return U, V, W


def perturbed(U, V, W, seed: int, std: float = 1e-3, n_zero: int = 5):
    """Approximate formula of Section 3.1: for each tensor, add i.i.d. N(0, std^2)
    noise to every entry equal to 1 and to `n_zero` entries equal to 0 chosen
    uniformly without replacement.  Seeded with numpy's PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for X in (U, V, W):
        Y = np.array(X, dtype=np.float64, copy=True)
        flat = Y.reshape(-1)
        ones = np.flatnonzero(flat == 1.0)
        zeros = np.flatnonzero(flat == 0.0)
        pick = rng.choice(zeros, size=min(n_zero, zeros.size), replace=False)
        idx = np.concatenate([ones, np.sort(pick)])
        flat[idx] += rng.normal(0.0, std, size=idx.size)
        out.append(Y)
    return tuple(out)


def ones_rank1(n0: int):
    """R = 1 with every coefficient equal to 1 (the remark after Prop. 5: kappa = 0
    yet a very poor formula)."""
    return (np.ones((n0, n0, 1)), np.ones((n0, n0, 1)), np.ones((n0, n0, 1)))


def gaussian_formula(n0: int, R: int, seed: int):
    """Dense random tensors with i.i.d. N(0,1) entries (an arbitrary ABC)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(rng.standard_normal((n0, n0, R)) for _ in range(3))


def formula_by_name(name: str, seed: int = 0):
    """'strassen' | 'laderman' | 'noisy-strassen' (Section 3.1 recipe, given seed)."""
    if name == "strassen":
        return strassen()
    if name == "laderman":
        return laderman()
    if name == "noisy-strassen":
        return perturbed(*strassen(), seed=seed)
    raise ValueError(f"unknown formula {name!r}")
