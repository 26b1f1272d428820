"""Sampled entries of the oracle's full-size recursion, computed by a pool of host processes.

The oracle (oracle.rbc_oracle.rbc_entries) evaluates selected entries of F^(L)(A, B) without
forming C; at the benchmarked sizes a thousand entries of a deep recursion take minutes on
one core, so the entries are split into chunks evaluated in parallel.  The pool starts its
workers with `spawn` (never forked from a process that holds a CUDA context), and the
operands reach them through memory-mapped .npy files."""
from __future__ import annotations

import multiprocessing
import os
import tempfile
from concurrent.futures import ProcessPoolExecutor

import numpy as np

CHUNK = 64


def _entries(path_a, path_b, U, V, W, L, seed, rows, cols):
    from oracle import rbc_oracle as o
    A = np.load(path_a, mmap_mode="r")
    B = np.load(path_b, mmap_mode="r")
    return o.rbc_entries(A, B, o.Plan(U, V, W, levels=L, seed=seed), rows, cols)


def oracle_entries(A, B, U, V, W, L, seed, rows, cols, workers=None):
    """o.rbc_entries(A, B, Plan(U, V, W, L, seed), rows, cols) over a spawn process pool."""
    workers = workers or max(1, min(8, os.cpu_count() or 1))
    with tempfile.TemporaryDirectory() as d:
        pa, pb = os.path.join(d, "A.npy"), os.path.join(d, "B.npy")
        np.save(pa, np.asarray(A, dtype=np.float64))
        np.save(pb, np.asarray(B, dtype=np.float64))
        ctx = multiprocessing.get_context("spawn")
        with ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
            futs = [ex.submit(_entries, pa, pb, U, V, W, L, seed, rows[i:i + CHUNK], cols[i:i + CHUNK])
                    for i in range(0, len(rows), CHUNK)]
            return np.concatenate([f.result() for f in futs])
