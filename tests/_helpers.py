"""Shared helpers of the GPU tests: run the library and the oracle on the same inputs."""
import numpy as np

from oracle import rbc_oracle as o
from rbc_inputs import formula_by_name, laderman, perturbed, strassen

# Normwise gate ||C - C_oracle||_F / (||A||_F ||B||_F) <= t * g^L / sqrt(N) per leaf mode
# (t at L = 0; g = 2 per level for n0 = 2 formulas, 3 for n0 = 3).
GATE_T = {"f32": 2e-5, "bf16x6": 2e-5, "f16x3": 2e-5, "3xtf32": 2e-5, "3xbf16": 4e-5, "tf32": 1e-3, "f16": 1e-3, "bf16": 8e-3}


def formula(name, seed=0):
    if name == "noisy-laderman":
        return perturbed(*laderman(), seed=seed)
    return formula_by_name(name, seed=seed)


def gate(leaf: str, n0: int, L: int, N: int) -> float:
    g = 2.0 if n0 == 2 else 3.0
    return GATE_T[leaf] * g**L / np.sqrt(N)


def entrywise_bound(A, B, n0: int, L: int, mixed: bool = False, rows=None, cols=None):
    """Entrywise scale of the rounding error of C = F^(L)(A, B), in fp64.

    Plain: (|A||B|)_ij, the scale of the standard product's error.  Mixed: the recursion adds
    the n0^L x n0^L grid of m x m blocks of A (and of B) into the leaf operands, so an entry
    of C also carries rounding error of every block row and column it is mixed with; the scale
    is (Abar Bbar)_{i mod m, j mod m} with Abar = sum of |A| over the blocks (m x m).  The
    mixed form is the one that holds for badly scaled rows and columns.  With rows/cols the
    bound of those entries only."""
    A = np.abs(np.asarray(A, dtype=np.float64))
    B = np.abs(np.asarray(B, dtype=np.float64))
    N = A.shape[0]
    if not mixed:
        if rows is None:
            return A @ B
        return np.einsum("sk,ks->s", A[rows], B[:, cols])
    q = n0**L
    m = N // q
    Ab = A.reshape(q, m, q, m).sum(axis=(0, 2))
    Bb = B.reshape(q, m, q, m).sum(axis=(0, 2))
    if rows is None:
        P = Ab @ Bb
        return np.tile(P, (q, q))
    rows, cols = np.asarray(rows) % m, np.asarray(cols) % m
    return np.einsum("sk,ks->s", Ab[rows], Bb[:, cols])


def entrywise(C, Cref, A, B, n0: int, L: int, mixed: bool = False) -> float:
    """max_ij |C - C_ref|_ij / bound_ij (entrywise_bound); compared with the gate's t g^L."""
    return float(np.max(np.abs(C - Cref) / entrywise_bound(A, B, n0, L, mixed)))


def egate(leaf: str, n0: int, L: int) -> float:
    """Entrywise gate t g^L (t and g of the normwise gate)."""
    g = 2.0 if n0 == 2 else 3.0
    return GATE_T[leaf] * g**L


def normwise(C, Cref, A, B) -> float:
    return float(np.linalg.norm(C - Cref) / (np.linalg.norm(A) * np.linalg.norm(B)))


def rel(C, Cref) -> float:
    return float(np.linalg.norm(C - Cref) / np.linalg.norm(Cref))


def gpu_rbc(rbc, plan, A, B, io_dtype, leaf, decode=0):
    import torch
    At = torch.tensor(A, dtype=io_dtype, device="cuda")
    Bt = torch.tensor(B, dtype=io_dtype, device="cuda")
    C = rbc.matmul(plan, At, Bt, leaf=leaf, decode=decode)
    torch.cuda.synchronize()
    return C.double().cpu().numpy()


def oracle_plan(U, V, W, L, seed, mode=o.RAND_FULL, scope=o.DRAW_PER_NODE):
    return o.Plan(U, V, W, levels=L, seed=seed, mode=mode, scope=scope)
