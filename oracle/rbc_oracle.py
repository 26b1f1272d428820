"""FP64 CPU oracle of the randomized bilinear computation (RBC).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module.  It shares no code with the CUDA library and
imports nothing from it: the random draws, the expanded coefficient tables, the
recursion and the error norms are all written here a second time, from the
paper's definitions, in plain numpy float64.

Notation follows the paper: an (n, tau)-ABC with tensors U, V, W of shape
(n, n, R) (Section 1, Eq. (1)); the randomization with signed permutations
M_i = P_i S_i and the rescaling (1 - kappa)^{-1} (Section 2.1, Def. RandABC);
the recursive algorithm F^(Q) (Section 2.1.1); the table form
u^_klr, v^_k'l'r, w^_ijr of Prop. 10.  The paper's n is called n0 here, Q is
called L (levels), and the leaf block size is m = N / n0^L.

Readings of points the paper leaves open (each also listed in the design notes):
  * random draws: the paper asks for i.i.d. Rademacher signs and uniform
    permutations (Section 2.1) without fixing a generator.  Both sides
    implement the counter-based SplitMix64 scheme of `draw_word` below.
  * scope: one draw set per recursion level (Section 2.1.1, literal) or one
    per tree node (independent draws per call; unbiasedness holds for both).
  * deterministic variant (s = 1, pi = id, Section 3) carries no rescaling
    unless asked; the randomized variants rescale by (1 - kappa)^{-1} at every
    level (Eq. recursive-random-formula).
  * summation order: sequential, l inner and k outer, as in the proof of
    Prop. 8; decoding sums r = 1..R sequentially.

Parity status: every function here is pinned by a test in tests/test_oracle_*.py
against closed forms, exact identities, enumeration or the paper's printed
values, except the exact digits of Example 7 (see `strassen_two_digit`), which
are only loosely pinned ("parity unpinned" for those digits).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from decimal import Decimal, Context, ROUND_HALF_EVEN
from typing import Callable, Optional

import numpy as np

# ----------------------------------------------------------------------------
# Formula quantities (Section 1, Eq. (3), Eqs. def-x / def-y; Section 2.1,
# Eq. epsilon-def; Eq. square-root-of-sum)
# ----------------------------------------------------------------------------


def tensor_Y(U, V, W) -> np.ndarray:
    """Y_{k l k' l' i j} = sum_r u_klr v_k'l'r w_ijr (Eq. def-y), by explicit loops over r."""
    n0, _, R = U.shape
    Y = np.zeros((n0,) * 6)
    for r in range(R):
        Y += np.multiply.outer(np.multiply.outer(U[:, :, r], V[:, :, r]), W[:, :, r])
    return Y


def tensor_X(n0: int) -> np.ndarray:
    """X_{k l k' l' i j} = delta_ki delta_l'j delta_lk' (Eq. def-x)."""
    X = np.zeros((n0,) * 6)
    for k in range(n0):
        for l in range(n0):
            for kp in range(n0):
                for lp in range(n0):
                    for i in range(n0):
                        for j in range(n0):
                            X[k, l, kp, lp, i, j] = float(k == i and lp == j and l == kp)
    return X


def exactness_violations(U, V, W) -> list:
    """Brute force over all (k,l,k',l',i,j) in [n]^6 of Eq. (3) in exact integer
    arithmetic (the tensors must hold integers); returns the violating tuples."""
    n0, _, R = U.shape
    Ui = U.astype(np.int64)
    Vi = V.astype(np.int64)
    Wi = W.astype(np.int64)
    if not (np.array_equal(Ui, U) and np.array_equal(Vi, V) and np.array_equal(Wi, W)):
        raise ValueError("exact check needs integer coefficients")
    bad = []
    rng = range(n0)
    for k in rng:
        for l in rng:
            for kp in rng:
                for lp in rng:
                    for i in rng:
                        for j in rng:
                            s = 0
                            for r in range(R):
                                s += int(Ui[k, l, r]) * int(Vi[kp, lp, r]) * int(Wi[i, j, r])
                            want = int(k == i and lp == j and l == kp)
                            if s != want:
                                bad.append((k, l, kp, lp, i, j, s, want))
    return bad


def tau(U, V, W) -> float:
    """||Y - X|| (Frobenius), the tau of Def. ABC."""
    return float(np.sqrt(np.sum((tensor_Y(U, V, W) - tensor_X(U.shape[0])) ** 2)))


def kappa(U, V, W) -> float:
    """kappa = n^-3 sum_{(i,j,l) in [n]^3} (1 - sum_r u_ilr v_ljr w_ijr)
    (Eq. epsilon-def), a sequential fp64 loop in (i, j, l, r) order."""
    n0, _, R = U.shape
    acc = 0.0
    for i in range(n0):
        for j in range(n0):
            for l in range(n0):
                s = 0.0
                for r in range(R):
                    s += U[i, l, r] * V[l, j, r] * W[i, j, r]
                acc += 1.0 - s
    return acc / n0**3


def gamma(U, V, W) -> float:
    """sqrt(sum_r ||U_::r||^2 ||V_::r||^2 ||W_::r||^2) (Eq. square-root-of-sum)."""
    R = U.shape[2]
    s = 0.0
    for r in range(R):
        s += np.sum(U[:, :, r] ** 2) * np.sum(V[:, :, r] ** 2) * np.sum(W[:, :, r] ** 2)
    return float(np.sqrt(s))


# ----------------------------------------------------------------------------
# Random draws (Section 2.1: Rademacher s_i(j), uniform permutations pi_i)
# ----------------------------------------------------------------------------

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15  # SplitMix64 increment (Steele, Lea, Flood 2014)

RAND_FULL, RAND_SIGN, RAND_PERM, RAND_NONE = 0, 1, 2, 3
DRAW_PER_NODE, DRAW_PER_LEVEL = 0, 1


def mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood 2014), exact on Python ints."""
    z &= _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def draw_word(seed: int, node: int, c: int) -> int:
    """64-bit word for stream c of a node: mix64(seed + golden * (1 + 8*node + c)) mod 2^64.
    c = 0, 1, 2 feed pi_1, pi_2, pi_3; c = 3, 4, 5 feed s_1, s_2, s_3."""
    return mix64((seed + _GOLDEN * (1 + 8 * node + c)) & _MASK)


def perm_from_word(word: int, n0: int) -> list:
    """Uniform permutation by Fisher-Yates, i = n0-1 down to 1, swapping p[i] with
    p[j], j = floor(x_i * (i+1) / 2^64), x_i = mix64(word + i).  pi(j) = p[j]."""
    p = list(range(n0))
    for i in range(n0 - 1, 0, -1):
        x = mix64((word + i) & _MASK)
        j = (x * (i + 1)) >> 64
        p[i], p[j] = p[j], p[i]
    return p


def signs_from_word(word: int, n0: int) -> list:
    """s(j) = -1 if bit j of the word is set, else +1 (i.i.d. Rademacher)."""
    return [-1 if (word >> j) & 1 else 1 for j in range(n0)]


@dataclass(frozen=True)
class NodeDraw:
    """pi_1, pi_2, pi_3 (as lists p with pi(j) = p[j]) and s_1, s_2, s_3."""
    pi: tuple
    s: tuple


def node_draw(seed: int, node: int, n0: int, mode: int) -> NodeDraw:
    ident = list(range(n0))
    ones = [1] * n0
    pis, ss = [], []
    for c in range(3):
        pis.append(tuple(perm_from_word(draw_word(seed, node, c), n0)
                         if mode in (RAND_FULL, RAND_PERM) else ident))
    for c in range(3):
        ss.append(tuple(signs_from_word(draw_word(seed, node, 3 + c), n0)
                        if mode in (RAND_FULL, RAND_SIGN) else ones))
    return NodeDraw(tuple(pis), tuple(ss))


def child_node(parent: int, r: int, R: int) -> int:
    """Heap numbering of the recursion tree: root 0, child r of p is p*R + r + 1."""
    return parent * R + r + 1


# ----------------------------------------------------------------------------
# Expanded tables (Prop. 10, Eq. randomized-algorithm)
# ----------------------------------------------------------------------------


def expand_tables(U, V, W, d: NodeDraw, scale: float):
    """u^_klr = u_{pi1(k) pi2(l) r} s1(k) s2(l);
       v^_k'l'r = v_{pi2(k') pi3(l') r} s2(k') s3(l');
       w^_ijr = scale * s1(i) s3(j) w_{pi1(i) pi3(j) r}  with scale = (1-kappa)^{-1}."""
    n0, _, R = U.shape
    (p1, p2, p3), (s1, s2, s3) = d.pi, d.s
    Uh = np.zeros_like(U)
    Vh = np.zeros_like(V)
    Wh = np.zeros_like(W)
    for a in range(n0):
        for b in range(n0):
            for r in range(R):
                Uh[a, b, r] = U[p1[a], p2[b], r] * s1[a] * s2[b]
                Vh[a, b, r] = V[p2[a], p3[b], r] * s2[a] * s3[b]
                Wh[a, b, r] = scale * s1[a] * s3[b] * W[p1[a], p3[b], r]
    return Uh, Vh, Wh


def signed_perm_matrix(pi, s, m: int) -> np.ndarray:
    """M = P S (Section 2.1): S = blockdiag(s(j) I_m), P has I_m at block (pi(j), j)."""
    n0 = len(pi)
    P = np.zeros((n0 * m, n0 * m))
    for j in range(n0):
        P[pi[j] * m:(pi[j] + 1) * m, j * m:(j + 1) * m] = s[j] * np.eye(m)
    return P


# ----------------------------------------------------------------------------
# Plan (all the per-call constants of one randomized computation)
# ----------------------------------------------------------------------------


@dataclass
class Plan:
    U: np.ndarray
    V: np.ndarray
    W: np.ndarray
    levels: int
    seed: int = 0
    mode: int = RAND_FULL
    scope: int = DRAW_PER_NODE
    rescale: Optional[bool] = None  # None: rescale iff randomized
    kappa: float = field(init=False)
    scale: float = field(init=False)

    def __post_init__(self):
        self.U = np.asarray(self.U, dtype=np.float64)
        self.V = np.asarray(self.V, dtype=np.float64)
        self.W = np.asarray(self.W, dtype=np.float64)
        self.kappa = kappa(self.U, self.V, self.W)
        if self.kappa == 1.0:
            raise ValueError("kappa = 1: RandABC undefined (Def. RandABC)")
        do = (self.mode != RAND_NONE) if self.rescale is None else bool(self.rescale)
        self.scale = 1.0 / (1.0 - self.kappa) if do else 1.0

    @property
    def n0(self):
        return self.U.shape[0]

    @property
    def R(self):
        return self.U.shape[2]

    def node_count(self) -> int:
        return sum(self.R ** d for d in range(self.levels))

    def draw(self, node: int, depth: int) -> NodeDraw:
        key = node if self.scope == DRAW_PER_NODE else depth
        return node_draw(self.seed, key, self.n0, self.mode)

    def tables(self, node: int, depth: int):
        return expand_tables(self.U, self.V, self.W, self.draw(node, depth), self.scale)


# ----------------------------------------------------------------------------
# The recursive algorithm (Section 2.1.1, Eq. recursive-random-formula)
# ----------------------------------------------------------------------------


def _blk(X, a, b, nb):
    return X[a * nb:(a + 1) * nb, b * nb:(b + 1) * nb]


def rbc(A, B, plan: Plan, leaf: Optional[Callable] = None) -> np.ndarray:
    """F^(L)(A, B) in fp64.  At each node: S_r = sum_{k,l} u^_klr A_kl and
    T_r = sum_{k',l'} v^_k'l'r B_k'l' (l inner, k outer), M_r = F^(q-1)(S_r, T_r),
    C_ij = sum_r w^_ijr M_r (r sequential).  F^(0) is the standard product."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    N = A.shape[0]
    if A.shape != (N, N) or B.shape != (N, N):
        raise ValueError("square inputs required")
    if N % plan.n0 ** plan.levels:
        raise ValueError("N must be a multiple of n0^L (pad first, Section 2.1.1)")
    mult = leaf if leaf is not None else (lambda X, Y: X @ Y)
    n0, R = plan.n0, plan.R

    def node_eval(X, Y, depth, node):
        if depth == plan.levels:
            return mult(X, Y)
        n = X.shape[0]
        nb = n // n0
        Uh, Vh, Wh = plan.tables(node, depth)
        M = []
        for r in range(R):
            S = np.zeros((nb, nb))
            T = np.zeros((nb, nb))
            for k in range(n0):
                for l in range(n0):
                    S = S + Uh[k, l, r] * _blk(X, k, l, nb)
            for k in range(n0):
                for l in range(n0):
                    T = T + Vh[k, l, r] * _blk(Y, k, l, nb)
            M.append(node_eval(S, T, depth + 1, child_node(node, r, R)))
        C = np.zeros((n, n))
        for i in range(n0):
            for j in range(n0):
                acc = np.zeros((nb, nb))
                for r in range(R):
                    acc = acc + Wh[i, j, r] * M[r]
                C[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = acc
        return C

    return node_eval(A, B, 0, 0)


def rbc_matrix_form(A, B, plan: Plan) -> np.ndarray:
    """One level (L = 1) through the matrix definition (Eq. f-hat-def):
    f^ = (1-kappa)^{-1} M1^T f(M1 A M2^T, M2 B M3^T) M3, with f the plain
    blockwise formula (Eq. bilinear-computation-block)."""
    if plan.levels != 1:
        raise ValueError("matrix form is written for one level")
    n0, R = plan.n0, plan.R
    N = A.shape[0]
    m = N // n0
    d = plan.draw(0, 0)
    M1, M2, M3 = (signed_perm_matrix(d.pi[c], d.s[c], m) for c in range(3))
    At = M1 @ A @ M2.T
    Bt = M2 @ B @ M3.T
    F = np.zeros((N, N))
    for r in range(R):
        S = sum(plan.U[k, l, r] * _blk(At, k, l, m) for k in range(n0) for l in range(n0))
        T = sum(plan.V[k, l, r] * _blk(Bt, k, l, m) for k in range(n0) for l in range(n0))
        P = S @ T
        for i in range(n0):
            for j in range(n0):
                F[i * m:(i + 1) * m, j * m:(j + 1) * m] += plan.W[i, j, r] * P
    return plan.scale * (M1.T @ F @ M3)


def rbc_entries(A, B, plan: Plan, rows, cols) -> np.ndarray:
    """Selected entries C[rows[t], cols[t]] of F^(L)(A, B) without forming C.

    Entry (alpha, beta) of a node's output lies in block (i, j) and only needs
    row (alpha mod nb) of every S_r and column (beta mod nb) of every T_r, which
    in turn need the rows {k*nb + .} of the node's left operand, k in [n0]; at
    the leaves this is a single row and column.  The recursion, tables and
    summation order are those of `rbc`; all requested entries are carried
    together as a leading batch axis."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    n0, R, L = plan.n0, plan.R, plan.levels
    N = A.shape[0]
    m = N // n0 ** L
    nb_count = n0 ** L
    # Rows of A needed for entry alpha: leaf-level block row K at intra-block row
    # alpha mod m, ordered with the root-level digit most significant.
    K = np.arange(nb_count)
    Xs = A[(K[None, :] * m + (rows % m)[:, None]), :]          # (b, n0^L, N)
    Ys = B[:, (K[None, :] * m + (cols % m)[:, None])]          # (N, b, n0^L)
    Ys = np.transpose(Ys, (1, 0, 2))                           # (b, N, n0^L)

    def node_eval(X, Y, alpha, beta, depth, node):
        # X: (b, c*n0, n) rows of the left operand; Y: (b, n, c*n0) its columns.
        if depth == L:
            return np.einsum("bk,bk->b", X[:, 0, :], Y[:, :, 0])
        n = X.shape[2]
        nb = n // n0
        c = X.shape[1] // n0
        Uh, Vh, Wh = plan.tables(node, depth)
        i = alpha // nb
        j = beta // nb
        acc = np.zeros(X.shape[0])
        for r in range(R):
            S = np.zeros((X.shape[0], c, nb))
            T = np.zeros((X.shape[0], nb, c))
            for k in range(n0):
                for l in range(n0):
                    S = S + Uh[k, l, r] * X[:, k * c:(k + 1) * c, l * nb:(l + 1) * nb]
            for k in range(n0):
                for l in range(n0):
                    T = T + Vh[k, l, r] * Y[:, k * nb:(k + 1) * nb, l * c:(l + 1) * c]
            Mr = node_eval(S, T, alpha % nb, beta % nb, depth + 1, child_node(node, r, R))
            acc = acc + Wh[i, j, r] * Mr
        return acc

    return node_eval(Xs, Ys, rows, cols, 0, 0)


def classical(A, B) -> np.ndarray:
    """The standard O(n^3) product in fp64, the truth of Section 3.2."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64)


# ----------------------------------------------------------------------------
# Enumeration of all draws (Props. 3 and 6; Example 7 counts 64 x 8 = 512)
# ----------------------------------------------------------------------------


def all_node_draws(n0: int, mode: int = RAND_FULL) -> list:
    """Every (pi_1, pi_2, pi_3, s_1, s_2, s_3) combination, each equally likely."""
    from itertools import permutations, product
    perms = list(permutations(range(n0))) if mode in (RAND_FULL, RAND_PERM) else [tuple(range(n0))]
    signs = list(product((1, -1), repeat=n0)) if mode in (RAND_FULL, RAND_SIGN) else [(1,) * n0]
    out = []
    for p1, p2, p3 in product(perms, repeat=3):
        for s1, s2, s3 in product(signs, repeat=3):
            out.append(NodeDraw((p1, p2, p3), (s1, s2, s3)))
    return out


def one_level(A, B, U, V, W, d: NodeDraw, scale: float, mult=None) -> np.ndarray:
    """f^(A, B) for one given draw, Eq. randomized-algorithm."""
    n0, _, R = U.shape
    mult = mult if mult is not None else (lambda X, Y: X @ Y)
    N = A.shape[0]
    nb = N // n0
    Uh, Vh, Wh = expand_tables(U, V, W, d, scale)
    M = []
    for r in range(R):
        S = np.zeros((nb, nb))
        T = np.zeros((nb, nb))
        for k in range(n0):
            for l in range(n0):
                S = S + Uh[k, l, r] * _blk(A, k, l, nb)
        for k in range(n0):
            for l in range(n0):
                T = T + Vh[k, l, r] * _blk(B, k, l, nb)
        M.append(mult(S, T))
    C = np.zeros((N, N))
    for i in range(n0):
        for j in range(n0):
            acc = np.zeros((nb, nb))
            for r in range(R):
                acc = acc + Wh[i, j, r] * M[r]
            C[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = acc
    return C


def expected_one_level(A, B, U, V, W, scale: float, mode: int = RAND_FULL) -> np.ndarray:
    """E[f^(A, B)] as the exact average over all equally likely draws."""
    draws = all_node_draws(U.shape[0], mode)
    acc = np.zeros((A.shape[0], A.shape[0]))
    for d in draws:
        acc = acc + one_level(A, B, U, V, W, d, scale)
    return acc / len(draws)


# ----------------------------------------------------------------------------
# Emulated low precision (Section 2.2 floating point model; Example 7)
# ----------------------------------------------------------------------------


def round_fp32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(x):
    """Round-to-nearest-even to bfloat16 (8 exponent bits, 8 significand bits),
    written from the IEEE-754 definition on the float32 bit pattern."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def round_tf32(x):
    """Round-to-nearest-even to 10 explicit significand bits (tf32) on float32."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 13) & 1
    b = (b + 0xFFF + lsb) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def round_fp16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def rbc_emulated(A, B, plan: Plan, rnd: Callable) -> np.ndarray:
    """F^(L) with every scalar operation rounded by `rnd` (fl(x op y) =
    (x op y)(1 + Delta), Section 2.2), sums sequential as in Prop. 8: encode
    products u*a rounded, partial sums rounded after each add; the leaf is the
    standard product with sequential rounded inner products; decode rounds
    each w*M and each add.  Inputs and coefficients are first rounded to the
    target format."""
    A = rnd(np.asarray(A, dtype=np.float64))
    B = rnd(np.asarray(B, dtype=np.float64))
    n0, R = plan.n0, plan.R

    def leaf(X, Y):
        n = X.shape[0]
        out = np.zeros((n, n))
        for z in range(n):  # sequential inner product, rounded after every op
            out = rnd(out + rnd(np.multiply.outer(X[:, z], Y[z, :])))
        return out

    def node_eval(X, Y, depth, node):
        if depth == plan.levels:
            return leaf(X, Y)
        n = X.shape[0]
        nb = n // n0
        Uh, Vh, Wh = (rnd(t) for t in plan.tables(node, depth))
        M = []
        for r in range(R):
            S = np.zeros((nb, nb))
            T = np.zeros((nb, nb))
            for k in range(n0):
                for l in range(n0):
                    S = rnd(S + rnd(Uh[k, l, r] * _blk(X, k, l, nb)))
            for k in range(n0):
                for l in range(n0):
                    T = rnd(T + rnd(Vh[k, l, r] * _blk(Y, k, l, nb)))
            M.append(node_eval(S, T, depth + 1, child_node(node, r, R)))
        C = np.zeros((n, n))
        for i in range(n0):
            for j in range(n0):
                acc = np.zeros((nb, nb))
                for r in range(R):
                    acc = rnd(acc + rnd(Wh[i, j, r] * M[r]))
                C[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = acc
        return C

    return node_eval(A, B, 0, 0)


def strassen_two_digit(A, B, U, V, W, d: Optional[NodeDraw] = None) -> np.ndarray:
    """Example 7: one level of a 2x2 formula on a machine with 2-digit decimal
    floating point (round half to even after every operation), scalar blocks.
    With d given, the randomized tables of Prop. 10 are used (kappa = 0)."""
    ctx = Context(prec=2, rounding=ROUND_HALF_EVEN)
    n0, _, R = U.shape

    def q(x):
        return ctx.create_decimal(repr(float(x))) if not isinstance(x, Decimal) else ctx.plus(x)

    if d is not None:
        U, V, W = expand_tables(U, V, W, d, 1.0)
    a = [[q(A[i][j]) for j in range(n0)] for i in range(n0)]
    b = [[q(B[i][j]) for j in range(n0)] for i in range(n0)]
    M = []
    for r in range(R):
        s = None
        for k in range(n0):
            for l in range(n0):
                if U[k, l, r] != 0:
                    t = ctx.multiply(q(U[k, l, r]), a[k][l])
                    s = t if s is None else ctx.add(s, t)
        t_ = None
        for k in range(n0):
            for l in range(n0):
                if V[k, l, r] != 0:
                    t = ctx.multiply(q(V[k, l, r]), b[k][l])
                    t_ = t if t_ is None else ctx.add(t_, t)
        M.append(ctx.multiply(s, t_))
    C = np.zeros((n0, n0))
    for i in range(n0):
        for j in range(n0):
            acc = None
            for r in range(R):
                if W[i, j, r] != 0:
                    t = ctx.multiply(q(W[i, j, r]), M[r])
                    acc = t if acc is None else ctx.add(acc, t)
            C[i, j] = float(acc) if acc is not None else 0.0
    return C


# ----------------------------------------------------------------------------
# Error norms (Section 3: relative Frobenius error, Eqs. error-of-average and
# average-of-error)
# ----------------------------------------------------------------------------


def fro(X) -> float:
    return float(np.sqrt(np.sum(np.asarray(X, dtype=np.float64) ** 2)))


def rel_fro(C, Cref) -> float:
    """||C - Cref||_F / ||Cref||_F."""
    return fro(np.asarray(C, dtype=np.float64) - Cref) / fro(Cref)
