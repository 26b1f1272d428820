"""Parity at the measured sizes, in the configuration bench.py times: each product of the fp32
sweep (Strassen n = 8192, L = 1..4; Laderman n = 6561, L = 1..3; perturbed Strassen n = 4096,
L = 1..3; 3xbf16 leaves, per-node draws, automatic decode) and of the precision sweep
(Strassen n = 16384, every leaf mode), compared with the oracle's randomized recursion with the
same draws on sampled entries (the oracle evaluates single entries of the full-size product).

The gate is t g^L relative to ||AB|| (t per leaf mode, g = 2 per level for n0 = 2, 3 for n0 = 3).
For the zero-mean N(0,1) inputs it is checked in its normwise form
||C - C_oracle||_F / (||A||_F ||B||_F) <= t g^L / sqrt(N) (there ||AB||_F ~ ||A||_F ||B||_F / sqrt(N)),
with ||C - C_oracle||_F estimated from the sampled entries as N times their root mean square.
For the entrywise-positive scaled inputs ||AB||_F ~ ||A||_F ||B||_F and the relative form is
checked directly on the sampled entries."""
import numpy as np
import pytest
import torch

from oracle import rbc_oracle as o
from rbc_inputs import formula_by_name

from ._helpers import gate

pytestmark = pytest.mark.gpu

SAMPLES = 32


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


def _sampled_normwise(rbc, name, n, L, seed, A, B, leaf, fseed=7):
    U, V, W = formula_by_name(name, seed=fseed)
    plan = rbc.Plan(U, V, W, levels=L, seed=seed)
    Ad, Bd = A.cuda(), B.cuda()
    C = rbc.matmul(plan, Ad, Bd, leaf=rbc.LEAF_NAMES[leaf])
    rng = np.random.default_rng(n + 31 * L)
    rows, cols = rng.integers(0, n, SAMPLES), rng.integers(0, n, SAMPLES)
    got = C[torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")].double().cpu().numpy()
    del C, Ad, Bd
    torch.cuda.empty_cache()
    An, Bn = A.double().numpy(), B.double().numpy()
    want = o.rbc_entries(An, Bn, o.Plan(U, V, W, levels=L, seed=seed), rows, cols)
    est = n * np.sqrt(np.mean((got - want) ** 2))
    rel = float(np.sqrt(np.mean((got - want) ** 2) / np.mean(want**2)))
    return est / (np.linalg.norm(An) * np.linalg.norm(Bn)), U.shape[0], rel


SWEEP = [("strassen", 8192, L) for L in (1, 2, 3, 4)] + [("laderman", 6561, L) for L in (1, 2, 3)] + \
        [("noisy-strassen", 4096, L) for L in (1, 2, 3)]


@pytest.mark.parametrize("name,n,L", SWEEP)
def test_sweep_sampled_parity(rbc, name, n, L):
    A, B = _bench_inputs(n)
    err, n0, _ = _sampled_normwise(rbc, name, n, L, 2024 + L, A, B, "3xbf16")
    assert err <= gate("3xbf16", n0, L, n), (name, n, L, err)


@pytest.mark.parametrize("leaf", ["tf32", "bf16", "f16", "3xbf16", "3xtf32", "f32"])
def test_precision_sweep_sampled_parity(rbc, leaf):
    n, L = 16384, 2
    g = torch.Generator(device="cpu")
    g.manual_seed(16384)
    A = torch.randn((n, n), generator=g, dtype=torch.float32)
    B = torch.randn((n, n), generator=g, dtype=torch.float32)
    err, n0, _ = _sampled_normwise(rbc, "strassen", n, L, 2024 + L, A, B, leaf)
    assert err <= gate(leaf, n0, L, n), (leaf, err)


def test_hard_inputs_sampled_parity(rbc):
    """The badly scaled case: Uniform[0,1] with rows of A and columns of B scaled by
    10^U(-3,3)."""
    from rbc_inputs.matrices import matrix_pair
    n, L = 8192, 2
    Ah, Bh = matrix_pair("hard", n, 9)
    A = torch.tensor(Ah, dtype=torch.float32)
    B = torch.tensor(Bh, dtype=torch.float32)
    _, n0, rel = _sampled_normwise(rbc, "strassen", n, L, 77, A, B, "3xbf16")
    assert rel <= gate("3xbf16", n0, L, n) * np.sqrt(n), rel   # = t g^L relative to ||AB||


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
