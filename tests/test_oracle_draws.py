"""Pins of the oracle's random draws (Section 2.1: i.i.d. Rademacher signs,
uniform independent permutations) and of the counter-based generator."""
from collections import Counter
from itertools import permutations

import numpy as np
import pytest

from oracle import rbc_oracle as o


def test_splitmix64_published_sequence():
    # SplitMix64 with state 0: the first outputs of the published generator.
    assert o.draw_word(0, 0, 0) == 0xE220A8397B1DCDAF
    assert o.mix64(2 * 0x9E3779B97F4A7C15 & (2**64 - 1)) == 0x6E789E6AA1B965F4
    assert o.mix64(3 * 0x9E3779B97F4A7C15 & (2**64 - 1)) == 0x06C45D188009454F


@pytest.mark.parametrize("n0", [2, 3, 4])
def test_permutations_are_uniform(n0):
    # Chi-square goodness of fit over all n0! permutations, many nodes.
    trials = 600 * len(list(permutations(range(n0))))
    cnt = Counter()
    for node in range(trials):
        p = o.perm_from_word(o.draw_word(12345, node, node % 3), n0)
        assert sorted(p) == list(range(n0))
        cnt[tuple(p)] += 1
    k = len(list(permutations(range(n0))))
    assert len(cnt) == k
    exp = trials / k
    chi2 = sum((c - exp) ** 2 / exp for c in cnt.values())
    # 99.9% quantile of chi2 with k-1 dof is < 3*(k-1)+15 for k <= 24
    assert chi2 < 3 * (k - 1) + 15
    # marginal P[pi(j) = k] = 1/n0 (Section 2.1)
    for j in range(n0):
        col = Counter()
        for p, c in cnt.items():
            col[p[j]] += c
        for v in range(n0):
            q = 1.0 / n0
            assert abs(col[v] / trials - q) < 4 * (q * (1 - q) / trials) ** 0.5


def test_signs_are_rademacher_and_independent():
    n = 20000
    s = np.array([o.signs_from_word(o.draw_word(99, node, 3), 4) for node in range(n)])
    assert set(np.unique(s)) == {-1, 1}
    assert np.all(np.abs(s.mean(axis=0)) < 0.03)
    # pairwise independence across positions and across streams c
    t = np.array([o.signs_from_word(o.draw_word(99, node, 4), 4) for node in range(n)])
    for a in range(4):
        for b in range(4):
            assert abs(np.mean(s[:, a] * t[:, b])) < 0.03
            if a != b:
                assert abs(np.mean(s[:, a] * s[:, b])) < 0.03


def test_node_draw_modes():
    d_full = o.node_draw(5, 3, 3, o.RAND_FULL)
    d_sign = o.node_draw(5, 3, 3, o.RAND_SIGN)
    d_perm = o.node_draw(5, 3, 3, o.RAND_PERM)
    d_none = o.node_draw(5, 3, 3, o.RAND_NONE)
    assert d_sign.pi == ((0, 1, 2),) * 3 and d_sign.s == d_full.s
    assert d_perm.s == ((1, 1, 1),) * 3 and d_perm.pi == d_full.pi
    assert d_none.pi == ((0, 1, 2),) * 3 and d_none.s == ((1, 1, 1),) * 3


def test_tree_numbering_and_scope():
    R = 7
    assert [o.child_node(0, r, R) for r in range(R)] == list(range(1, 8))
    assert o.child_node(3, 0, R) == 22
    # heap numbering: depth-d nodes occupy a contiguous range starting at (R^d - 1)/(R - 1)
    ids = [o.child_node(o.child_node(0, r1, R), r2, R) for r1 in range(R) for r2 in range(R)]
    assert ids == list(range((R**2 - 1) // (R - 1), (R**2 - 1) // (R - 1) + R**2))
    from rbc_inputs import strassen
    p_node = o.Plan(*strassen(), levels=2, seed=11, scope=o.DRAW_PER_NODE)
    p_lvl = o.Plan(*strassen(), levels=2, seed=11, scope=o.DRAW_PER_LEVEL)
    assert p_lvl.draw(5, 1) == p_lvl.draw(2, 1) == o.node_draw(11, 1, 2, o.RAND_FULL)
    assert p_node.draw(5, 1) == o.node_draw(11, 5, 2, o.RAND_FULL)
    assert p_node.node_count() == 8


def test_enumeration_counts_example7():
    # Example 7: 64 sign functions x 8 permutation functions for n = 2.
    draws = o.all_node_draws(2)
    assert len(draws) == 512
    assert len({d.s for d in draws}) == 64
    assert len({d.pi for d in draws}) == 8
    assert len(o.all_node_draws(3)) == 2**9 * 6**3
