"""Parity at the measured sizes, in the configuration bench.py times: each product of the fp32
sweep (Strassen n = 8192, L = 1..4; Laderman n = 6561, L = 1..3; perturbed Strassen n = 4096,
L = 1..3; f16x3 leaves, the default, and bf16x6 leaves; per-node draws, automatic decode) and of
the precision sweep
(Strassen n = 16384, every leaf mode), compared with the oracle's randomized recursion with the
same draws on sampled entries (the oracle evaluates single entries of the full-size product).

Samples: 1024 entries per product.  Beside uniformly drawn ones they hold every pairing of
special rows and columns: the first and last, both sides of leaf-block boundaries
(k m - 1, k m) and the tile edges of the leaf kernels inside a leaf (offsets 127, 128, 255,
256), so that a wrong tile edge, padding column or leaf boundary is sampled.

Gates (t per leaf mode, g = 2 per level for n0 = 2, 3 for n0 = 3):
  * normwise ||C - C_oracle||_F / (||A||_F ||B||_F) <= t g^L / sqrt(N), with ||C - C_oracle||_F
    estimated from the sampled entries as N times their root mean square;
  * entrywise |C - C_oracle|_ij <= t g^L bound_ij on every sampled entry (bound as in
    tests/_helpers.entrywise_bound: (|A||B|)_ij on zero-mean inputs, the block-mixed form on the
    badly scaled ones).
The two-piece 3xbf16 split keeps 16 significant bits of each leaf operand; on the entrywise
positive scaled inputs its error (about 1e-5 relative to ||AB||, which there is about
||A|| ||B||) does not cancel, and it is gated in the relative form ||C - C_oracle|| / ||AB|| <= t g^L
only."""
import numpy as np
import pytest
import torch

from rbc_inputs import formula_by_name

from ._helpers import egate, entrywise_bound, gate
from ._oracle_pool import oracle_entries

pytestmark = pytest.mark.gpu

SAMPLES = 1024


def sample_entries(n, m, seed, count=SAMPLES):
    """count (row, col) pairs: every pairing of the special indices (first, last, both sides of
    leaf boundaries, tile edges inside the first and last leaf block), then uniform ones."""
    q = n // m
    special = {0, n - 1}
    for k in sorted({1, q // 2, q - 1}):
        if 0 < k < q:
            special |= {k * m - 1, k * m}
    for base in (0, (q - 1) * m):
        for t in (127, 128, 255, 256):
            if t < m:
                special.add(base + t)
    sp = np.array(sorted(special))
    rows, cols = np.meshgrid(sp, sp, indexing="ij")
    rows, cols = rows.ravel()[:count], cols.ravel()[:count]
    rng = np.random.default_rng(seed)
    extra = count - rows.size
    rows = np.concatenate([rows, rng.integers(0, n, extra)])
    cols = np.concatenate([cols, rng.integers(0, n, extra)])
    return rows, cols


@pytest.fixture(scope="module")
def rbc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_07439_gb300 import build as b
    b.build()
    import paper_1905_07439_gb300 as pkg
    return pkg


def _bench_inputs(n):
    """The sweep's inputs: a seeded N(0,1) fp32 pair per size (torch CPU generator)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(1000 + n)
    A = torch.randn((n, n), generator=g, dtype=torch.float32)
    B = torch.randn((n, n), generator=g, dtype=torch.float32)
    return A, B


_ORACLE_CACHE = {}


def _sampled_normwise(rbc, name, n, L, seed, A, B, leaf, fseed=7, mixed=False, count=SAMPLES):
    """(normwise estimate, n0, relative rms error, max entrywise ratio |dC| / bound) over the
    sampled entries."""
    U, V, W = formula_by_name(name, seed=fseed)
    n0 = U.shape[0]
    plan = rbc.Plan(U, V, W, levels=L, seed=seed)
    Ad, Bd = A.cuda(), B.cuda()
    C = rbc.matmul(plan, Ad, Bd, leaf=rbc.LEAF_NAMES[leaf])
    rows, cols = sample_entries(n, n // n0**L, n + 31 * L, count)
    got = C[torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")].double().cpu().numpy()
    del C, Ad, Bd
    torch.cuda.empty_cache()
    An, Bn = A.double().numpy(), B.double().numpy()
    key = (name, n, L, seed, fseed, len(rows), int(rows[-1]), int(cols[-1]))
    if key not in _ORACLE_CACHE:  # the same entries for every leaf mode of a product
        _ORACLE_CACHE.clear()
        _ORACLE_CACHE[key] = oracle_entries(An, Bn, U, V, W, L, seed, rows, cols)
    want = _ORACLE_CACHE[key]
    bound = entrywise_bound(An, Bn, n0, L, mixed, rows, cols)
    est = n * np.sqrt(np.mean((got - want) ** 2))
    rel = float(np.sqrt(np.mean((got - want) ** 2) / np.mean(want**2)))
    ent = float(np.max(np.abs(got - want) / bound))
    return est / (np.linalg.norm(An) * np.linalg.norm(Bn)), n0, rel, ent


SWEEP = [("strassen", 8192, L) for L in (1, 2, 3, 4)] + [("laderman", 6561, L) for L in (1, 2, 3)] + \
        [("noisy-strassen", 4096, L) for L in (1, 2, 3)]


@pytest.mark.parametrize("leaf", ["f16x3", "bf16x6"])
@pytest.mark.parametrize("name,n,L", SWEEP)
def test_sweep_sampled_parity(rbc, name, n, L, leaf):
    A, B = _bench_inputs(n)
    err, n0, _, ent = _sampled_normwise(rbc, name, n, L, 2024 + L, A, B, leaf)
    assert err <= gate(leaf, n0, L, n), (name, n, L, err)
    assert ent <= egate(leaf, n0, L), (name, n, L, ent)


# Deeper plans than the sweep's: Laderman L = 4 (two two-level passes, the second over the 529
# depth-2 blocks), Strassen L = 5 (a one-level pass, then four-level passes over the 7 depth-1
# blocks) and perturbed Strassen L = 4 (one four-level pass, dense coefficients); 128 sampled
# entries each (the oracle's recursion per entry grows as R^L).
@pytest.mark.parametrize("name,n,L", [("laderman", 2592, 4), ("strassen", 8192, 5), ("noisy-strassen", 4096, 4)])
def test_deep_plans_sampled_parity(rbc, name, n, L):
    A, B = _bench_inputs(n)
    err, n0, _, ent = _sampled_normwise(rbc, name, n, L, 77 + L, A, B, "f16x3", count=128)
    assert err <= gate("f16x3", n0, L, n), (name, n, L, err)
    assert ent <= egate("f16x3", n0, L), (name, n, L, ent)


@pytest.mark.parametrize("leaf", ["tf32", "bf16", "f16", "3xbf16", "3xtf32", "bf16x6", "f16x3", "f32"])
def test_precision_sweep_sampled_parity(rbc, leaf):
    n, L = 16384, 2
    g = torch.Generator(device="cpu")
    g.manual_seed(16384)
    A = torch.randn((n, n), generator=g, dtype=torch.float32)
    B = torch.randn((n, n), generator=g, dtype=torch.float32)
    err, n0, _, ent = _sampled_normwise(rbc, "strassen", n, L, 2024 + L, A, B, leaf)
    assert err <= gate(leaf, n0, L, n), (leaf, err)
    assert ent <= egate(leaf, n0, L), (leaf, ent)


@pytest.mark.parametrize("name,L,leaf", [("strassen", 2, "bf16x6"), ("laderman", 2, "bf16x6"), ("strassen", 2, "f16x3"),
                                         ("laderman", 2, "f16x3"),
                                         ("strassen", 2, "3xbf16")])
def test_hard_inputs_sampled_parity(rbc, name, L, leaf):
    """The badly scaled case: Uniform[0,1] with rows of A and columns of B scaled by
    10^U(-3,3)."""
    from rbc_inputs.matrices import matrix_pair
    n = 8192 if name == "strassen" else 6561
    Ah, Bh = matrix_pair("hard", n, 9)
    A = torch.tensor(Ah, dtype=torch.float32)
    B = torch.tensor(Bh, dtype=torch.float32)
    err, n0, rel, ent = _sampled_normwise(rbc, name, n, L, 77, A, B, leaf, mixed=True)
    assert ent <= egate(leaf, n0, L), (leaf, ent)
    if leaf == "3xbf16":
        assert rel <= gate(leaf, n0, L, n) * np.sqrt(n), rel   # = t g^L relative to ||AB||
    else:
        assert err <= gate(leaf, n0, L, n), err


@pytest.mark.parametrize("n,L,decode", [(46400, 1, 2), (46400, 1, 1), (47104, 2, 2)])
def test_more_than_2_31_elements(rbc, n, L, decode):
    """n^2 > 2^31: element offsets into A, B, C and the workspace need 64 bits, in the passes,
    the leaf epilogue (staged, decode 2, and fused into C, decode 1) and the decode.  Exact
    Strassen with bf16 leaves; the RBC of an exact formula equals AB up to rounding (Section 2,
    orthogonality of the signed permutations), so sampled entries, the last row and column
    among them, are compared with fp64 dot products of the same rows and columns under the
    bf16 gate."""
    g = torch.Generator(device="cuda")
    g.manual_seed(n + L)
    A = torch.randn((n, n), generator=g, device="cuda")
    B = torch.randn((n, n), generator=g, device="cuda")
    plan = rbc.Plan(*formula_by_name("strassen"), levels=L, seed=2024 + L)
    C = rbc.matmul(plan, A, B, leaf=rbc.LEAF_BF16, decode=decode)
    rng = np.random.default_rng(n + L)
    rows, cols = rng.integers(0, n, SAMPLES), rng.integers(0, n, SAMPLES)
    rows[0], cols[0] = n - 1, n - 1
    rt, ct = torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")
    got = C[rt, ct].double().cpu().numpy()
    want = np.einsum("sk,ks->s", A[rt].double().cpu().numpy(), B[:, ct].double().cpu().numpy())
    nA = float(np.sqrt(rbc.norms(A).cpu().numpy()[0]))
    nB = float(np.sqrt(rbc.norms(B).cpu().numpy()[0]))
    del A, B, C
    torch.cuda.empty_cache()
    err = n * np.sqrt(np.mean((got - want) ** 2)) / (nA * nB)
    assert err <= gate("bf16", 2, L, n), (n, L, decode, err)
