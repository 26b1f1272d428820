"""The bound behind the f16x3 leaf scales, checked on the oracle's own recursion (CPU).

Row i of every left leaf operand S_rho is a signed sum, over the recursion's block path, of rows
of A congruent to i mod m (m = N / n0^L), with one coefficient u^ per level (Section 2.1.1,
Eq. recursive-random-formula; the randomized tables of Prop. 10 permute and sign the entries of
U without changing their magnitudes).  So

    |S_rho[i][k]| <= gamma_U^L * max_{i' == i mod m} max_k' |A[i'][k']|,
    gamma_U = max_r sum_{k,l} |u_klr|,

and likewise every column j of the right operands T_rho with V and the columns of B congruent
to j mod m.  The f16x3 leaf mode chooses a power of two per class from this bound, so that the
scaled entries (and hence both fp16 pieces) stay below 2^15.  The leaf operands here are the
oracle's (its leaf callback receives S_rho and T_rho), with random signed permutations."""
import numpy as np
import pytest

from oracle import rbc_oracle as o
from rbc_inputs import matrix_pair

from ._helpers import formula

CASES = [("strassen", 3, 6, "hard"), ("strassen", 2, 7, "normal"), ("laderman", 2, 5, "hard"),
         ("laderman", 1, 9, "normal"), ("noisy-strassen", 2, 8, "hard")]


def _class_max(absmax, n_blocks, m):
    """max over the n_blocks entries congruent mod m (entry index = block * m + i)."""
    return absmax.reshape(n_blocks, m).max(axis=0)


@pytest.mark.parametrize("name,L,m,dist", CASES)
def test_leaf_operands_within_the_class_bound(name, L, m, dist):
    U, V, W = formula(name, seed=3)
    n0, R = U.shape[0], U.shape[2]
    N = n0**L * m
    A, B = matrix_pair(dist, N, seed=31 + m)
    plan = o.Plan(U, V, W, levels=L, seed=17 + L)
    leaves = []

    def record(X, Y):
        leaves.append((X.copy(), Y.copy()))
        return X @ Y

    o.rbc(A, B, plan, leaf=record)
    assert len(leaves) == R**L
    gU = np.abs(U).sum(axis=(0, 1)).max()
    gV = np.abs(V).sum(axis=(0, 1)).max()
    rows = _class_max(np.abs(A).max(axis=1), n0**L, m)   # per leaf row i
    cols = _class_max(np.abs(B).max(axis=0), n0**L, m)   # per leaf column j
    worst_s = worst_t = 0.0
    for S, T in leaves:
        worst_s = max(worst_s, float((np.abs(S) / (gU**L * rows[:, None])).max()))
        worst_t = max(worst_t, float((np.abs(T) / (gV**L * cols[None, :])).max()))
    assert worst_s <= 1.0 + 1e-12 and worst_t <= 1.0 + 1e-12, (worst_s, worst_t)
    # the bound is attained up to the inputs' cancellation: not vacuous
    assert worst_s > 1e-3 and worst_t > 1e-3, (worst_s, worst_t)


def test_bound_is_tight_for_one_nonzero_path():
    """With A = all ones, the rank-one rule u = v = w = 1 (n0 = 2, R = 1) and no randomization
    (random signs would cancel the equal blocks), every leaf entry is exactly gamma^L times the
    class maximum: the bound cannot be lowered."""
    U = np.ones((2, 2, 1))
    V = np.ones((2, 2, 1))
    W = np.ones((2, 2, 1))
    L, m = 3, 4
    N = 2**L * m
    A = np.ones((N, N))
    plan = o.Plan(U, V, W, levels=L, seed=1, mode=o.RAND_NONE)
    leaves = []

    def record(X, Y):
        leaves.append(X.copy())
        return X @ Y

    o.rbc(A, A, plan, leaf=record)
    assert len(leaves) == 1
    assert np.all(np.abs(leaves[0]) == 4.0**L)   # gamma = 4 (four unit coefficients), max |A| = 1
