"""Pins of the oracle's formula quantities (Section 1 Eq. (3); Section 2.1
Eq. epsilon-def; Props. 4-5; Eq. square-root-of-sum) against exact identities,
closed forms and the paper's printed values."""
import json
import math
import os

import numpy as np
import pytest

from oracle import rbc_oracle as o
from rbc_inputs import (classical_formula, gaussian_formula, laderman, ones_rank1,
                        perturbed, strassen)

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("name,fn", [("strassen", strassen), ("laderman", laderman)])
def test_eq3_exact_by_brute_force(name, fn):
    U, V, W = fn()
    n0, R = GOLDEN["section1"][name]["n0"], GOLDEN["section1"][name]["R"]
    assert U.shape == (n0, n0, R)
    assert o.exactness_violations(U, V, W) == []
    assert o.tau(U, V, W) == 0.0
    assert o.kappa(U, V, W) == 0.0


def test_eq3_catches_planted_errors():
    # A mistake in any tensor entry must show up as a violated identity.
    for t in range(3):
        for idx in [(0, 0, 0), (1, 1, 6), (0, 1, 3)]:
            UVW = [x.copy() for x in strassen()]
            UVW[t][idx] = 1.0 - UVW[t][idx] if UVW[t][idx] == 0 else -UVW[t][idx]
            assert o.exactness_violations(*UVW)
            assert o.tau(*UVW) > 0.0


def test_eq3_classical_formula_and_tensor_X():
    U, V, W = classical_formula(2)
    assert o.exactness_violations(U, V, W) == []
    X = o.tensor_X(3)
    # X has exactly n^3 ones (one per (i, j, l)), ||X|| = n^{3/2} (Eq. Ye-bound).
    assert X.sum() == 27 and math.isclose(np.linalg.norm(X), 27 ** 0.5)


def test_gamma_closed_forms_and_example13():
    # Classical formula: every slice has one nonzero in each tensor -> Gamma = sqrt(n^3).
    assert math.isclose(o.gamma(*classical_formula(2)), math.sqrt(8))
    assert math.isclose(o.gamma(*classical_formula(3)), math.sqrt(27))
    g = o.gamma(*strassen())
    assert math.isclose(g, math.sqrt(32))
    # Example 13 prints "approximately 6".
    assert abs(g - GOLDEN["example13"]["strassen_gamma_approx"]) < 0.5


def test_example13_second_term_value():
    e = GOLDEN["example13"]
    n, R, m, eps, gb = e["n"], e["R"], e["m"], e["eps_machine"], e["gamma_bound"]
    coeff = gb * 1.01 * (4 * n + m + R - 2) * math.sqrt(R) / 2 ** 2.5 * eps
    assert abs(coeff - e["second_term_coefficient"]) < 5e-5


def test_kappa_closed_form_under_scaling():
    # Scaling W of an exact formula by c multiplies every sum_r u v w on the
    # "diagonal" (i, j, l) by c, so kappa = 1 - c exactly.
    U, V, W = strassen()
    for c in (1.1, 0.5, -2.0):
        assert math.isclose(o.kappa(U, V, c * W), 1.0 - c, rel_tol=1e-14)
    # R = 1, all ones: kappa = 0 (remark after Prop. 5), yet tau is large.
    U1, V1, W1 = ones_rank1(2)
    assert o.kappa(U1, V1, W1) == 0.0
    assert o.tau(U1, V1, W1) > 1.0


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_prop5_kappa_bound_on_perturbed_strassen(seed):
    U, V, W = perturbed(*strassen(), seed=seed)
    n = 2
    t = o.tau(U, V, W)
    k = o.kappa(U, V, W)
    assert t > 0
    assert abs(k) <= n ** -2.5 * t + 1e-15          # Eq. epsilon-bound
    eta = 1.0 / (1.0 - k) - 1.0
    Ynorm = np.linalg.norm(o.tensor_Y(U, V, W))
    assert Ynorm <= t + n ** 1.5 + 1e-12              # Eq. Ye-bound
    assert abs(eta) * Ynorm <= 2 * (n ** -2.5 * t + 1.0 / n) * t + 1e-15  # Prop. 5


def test_perturbed_recipe_section31():
    U0, V0, W0 = strassen()
    U, V, W = perturbed(U0, V0, W0, seed=7)
    for X0, X in ((U0, U), (V0, V), (W0, W)):
        changed = X != X0
        # every +1 entry is perturbed, exactly five zeros are perturbed, -1 untouched
        assert changed[X0 == 1.0].all()
        assert changed[X0 == 0.0].sum() == 5
        assert not changed[X0 == -1.0].any()
        assert np.abs(X - X0).max() < 1e-2


def test_tensor_Y_matches_eq2_bilinear_form():
    # Eq. (2): c_ij = sum a_kl b_k'l' Y_{klk'l'ij}; compare with Eq. (1) evaluated directly.
    U, V, W = gaussian_formula(2, 5, seed=3)
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((2, 2)), rng.standard_normal((2, 2))
    Y = o.tensor_Y(U, V, W)
    c2 = np.einsum("kl,pq,klpqij->ij", a, b, Y)
    c1 = np.zeros((2, 2))
    for r in range(5):
        c1 += W[:, :, r] * np.sum(U[:, :, r] * a) * np.sum(V[:, :, r] * b)
    assert np.allclose(c1, c2, rtol=1e-13, atol=1e-13)
