"""Shared helpers of the GPU tests: run the library and the oracle on the same inputs."""
import numpy as np

from oracle import rbc_oracle as o
from rbc_inputs import formula_by_name, laderman, perturbed, strassen

# Normwise gate ||C - C_oracle||_F / (||A||_F ||B||_F) <= t * g^L / sqrt(N) per leaf mode
# (t at L = 0; g = 2 per level for n0 = 2 formulas, 3 for n0 = 3).
GATE_T = {"f32": 2e-5, "bf16x6": 2e-5, "3xtf32": 2e-5, "3xbf16": 4e-5, "tf32": 1e-3, "f16": 1e-3, "bf16": 8e-3}


def formula(name, seed=0):
    if name == "noisy-laderman":
        return perturbed(*laderman(), seed=seed)
    return formula_by_name(name, seed=seed)


def gate(leaf: str, n0: int, L: int, N: int) -> float:
    g = 2.0 if n0 == 2 else 3.0
    return GATE_T[leaf] * g**L / np.sqrt(N)


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
