"""The synthetic error experiments of Section 3, run on the GPU through librbc.

Section 3 measures two quantities for a fixed pair (A, B), both against the standard
product computed in double precision:

  * the error of the average of n realizations, ||(1/n) sum_{i<=n} F_i(A, B) - AB|| / ||AB||
    for n = 1 .. K (Eq. error-of-average; Figures 2 and 4: N = 80, K = 10^4, Q = 1..3);
  * the error of single realizations, ||F_i(A, B) - AB|| / ||AB|| for i = 1 .. 100
    (Eq. average-of-error; Figures 3 and 5: N = 320, Q = 1..5), beside the deterministic
    recursion F^(Q) (s = 1, pi = id) and, in floating point, the standard algorithm.

Section 3.1 uses a perturbed Strassen formula (noise of standard deviation 1e-3 on every
entry equal to 1 and on five zero entries per tensor) in double precision; Section 3.2 uses
the exact Strassen formula in single precision, with the fully randomized, random-sign,
random-permutation and deterministic variants, on Gaussian, uniform, adversarial (types 1-3)
and Hilbert inputs.  Draws are per level, as the paper defines them (one draw set per
recursion level shared by its nodes); realization i draws from seed base + i.

Every realization, reference product and error norm is computed by the library's kernels:
all realizations of one configuration in batched launches (rbc_matmul_realizations), the
errors by one reduction over all of them (rbc_realization_errors).  The rescaling method of
Section 3.2's comparison is not reproduced here (its twice-applied variant is only cited).

Run:  python -m paper_1905_07439_gb300.experiments --exp fig2,fig5 --out results.json
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import rbc

VARIANTS = {"full": rbc.RAND_FULL, "sign": rbc.RAND_SIGN, "perm": rbc.RAND_PERM,
            "deterministic": rbc.RAND_NONE}
DISTS = ("normal", "uniform", "adv1", "adv2", "adv3", "hilbert")

# name -> (kind, formula, io, N, levels, dists, variants)
#   kind "average": error of the average of K realizations; "trials": single realizations
EXPERIMENTS = {
    "fig2": ("average", "noisy-strassen", "f64", 80, (1, 2, 3), ("normal",), ("full",)),
    "fig3": ("trials", "noisy-strassen", "f64", 320, (1, 2, 3, 4, 5), ("normal",), ("full",)),
    "fig3h": ("trials", "noisy-strassen", "f64", 320, (1, 2, 3, 4, 5), ("hilbert",), ("full",)),
    "fig3s": ("trials", "noisy-strassen", "f64", 320, (1, 2, 3, 4, 5), DISTS, ("full",)),
    "fig4": ("average", "strassen", "f32", 80, (1, 2, 3), ("normal",), ("full",)),
    "fig4h": ("average", "strassen", "f32", 80, (1, 2, 3), ("hilbert",), ("full",)),
    "fig4s": ("average", "strassen", "f32", 80, (1, 2, 3), DISTS, ("full",)),
    "fig5": ("trials", "strassen", "f32", 320, (1, 2, 3, 4, 5), DISTS, ("full", "sign", "perm")),
}


def _formula(name: str, seed: int):
    from rbc_inputs.formulas import formula_by_name
    return formula_by_name(name, seed=seed)


def _inputs(dist: str, n: int, seed: int):
    from rbc_inputs.matrices import matrix_pair
    return matrix_pair(dist, n, seed)


class Runner:
    """Device state of one experiment: inputs, the fp64 standard product and scratch."""

    def __init__(self, U, V, W, A, B, io: str, device: str = "cuda"):
        import torch
        self.torch = torch
        self.U, self.V, self.W = U, V, W
        self.dtype = torch.float64 if io == "f64" else torch.float32
        self.io = rbc.IO_F64 if io == "f64" else rbc.IO_F32
        self.leaf = rbc.LEAF_F64 if io == "f64" else rbc.LEAF_F32
        self.N = A.shape[0]
        self.A64 = torch.tensor(A, dtype=torch.float64, device=device)
        self.B64 = torch.tensor(B, dtype=torch.float64, device=device)
        self.A = self.A64.to(self.dtype)
        self.B = self.B64.to(self.dtype)
        # the true product: the standard algorithm in double precision (F^(0), fp64 leaves)
        p0 = rbc.Plan(U, V, W, levels=0, seed=0, rand_mode=rbc.RAND_NONE)
        self.ref = rbc.matmul(p0, self.A64, self.B64, leaf=rbc.LEAF_F64)

    def plan(self, levels: int, mode: int, scope: int):
        return rbc.Plan(self.U, self.V, self.W, levels=levels, seed=0, rand_mode=mode, draw_scope=scope)

    def realize(self, plan, seeds, leaf=None, max_ws_bytes: int = 8 << 30):
        """Realizations of `plan` with draws from each seed, batched as far as `max_ws_bytes`
        of workspace allows."""
        torch = self.torch
        leaf = self.leaf if leaf is None else leaf
        one = int(rbc.lib().rbc_realizations_workspace_size(plan.handle, self.N, self.io, leaf, 1))
        if one == 0:
            raise rbc.RbcError(rbc.RBC_EINVAL, "no layout for this configuration")
        batch = max(1, min(len(seeds), max_ws_bytes // one))
        need = int(rbc.lib().rbc_realizations_workspace_size(plan.handle, self.N, self.io, leaf, batch))
        ws = torch.empty(need, dtype=torch.uint8, device=self.A.device)
        return rbc.realizations(plan, seeds, self.A, self.B, leaf=leaf, workspace=ws)

    def errors(self, Cs, mode: int):
        return rbc.realization_errors(Cs, self.ref, mode).cpu().numpy()

    def standard_error(self, leaf=None) -> float:
        """Error of the standard algorithm in the experiment's precision."""
        p0 = rbc.Plan(self.U, self.V, self.W, levels=0, seed=0, rand_mode=rbc.RAND_NONE)
        C0 = rbc.matmul(p0, self.A, self.B, leaf=self.leaf if leaf is None else leaf)
        return float(self.errors(C0[None], rbc.ERR_EACH)[0])


def _log_grid(K: int):
    pts, x = [], 1
    while x <= K:
        for m in (1, 2, 5):
            if m * x <= K:
                pts.append(m * x)
        x *= 10
    if pts[-1] != K:
        pts.append(K)
    return pts


def _quantiles(e: np.ndarray) -> dict:
    q = np.quantile(e, [0.0, 0.25, 0.5, 0.75, 1.0])
    return {"min": float(q[0]), "q1": float(q[1]), "median": float(q[2]), "q3": float(q[3]), "max": float(q[4])}


def run_experiment(name: str, K: int = 10_000, trials: int = 100, seed: int = 0, scope: int = rbc.DRAW_PER_LEVEL,
                   leaf: str | None = None, dists=None, levels=None, full: bool = False) -> dict:
    """One experiment of Section 3; returns a JSON-ready summary (and the raw error arrays
    when `full`)."""
    import torch
    kind, fname, io, N, lv, ds, variants = EXPERIMENTS[name]
    ds = tuple(dists) if dists else ds
    lv = tuple(levels) if levels else lv
    U, V, W = _formula(fname, seed)
    out = {"experiment": name, "kind": kind, "formula": fname, "io": io, "N": N,
           "leaf": leaf or io, "scope": "level" if scope == rbc.DRAW_PER_LEVEL else "node", "results": []}
    leaf_id = rbc.LEAF_NAMES[leaf] if leaf else None
    realizations = 0
    t0 = time.perf_counter()
    for dist in ds:
        A, B = _inputs(dist, N, seed + 1000)
        run = Runner(U, V, W, A, B, io)
        row = {"dist": dist, "standard": run.standard_error(leaf_id) if io == "f32" or leaf else None}
        for Q in lv:
            if N % (2 ** Q):
                continue
            det = run.realize(run.plan(Q, rbc.RAND_NONE, scope), [0], leaf_id)
            e_det = float(run.errors(det, rbc.ERR_EACH)[0])
            entry = {"Q": Q, "deterministic": e_det}
            for var in variants:
                mode = VARIANTS[var]
                count = K if kind == "average" else trials
                base = (seed << 32) + (Q << 24)
                Cs = run.realize(run.plan(Q, mode, scope), np.arange(base, base + count, dtype=np.uint64), leaf_id)
                realizations += count
                if kind == "average":
                    e = run.errors(Cs, rbc.ERR_AVERAGE)
                    grid = _log_grid(count)
                    entry[var] = {"n": grid, "error_of_average": [float(e[n - 1]) for n in grid]}
                else:
                    e = run.errors(Cs, rbc.ERR_EACH)
                    entry[var] = _quantiles(e)
                if full:
                    entry[var]["all"] = e.tolist()
                del Cs
            row.setdefault("levels", []).append(entry)
        out["results"].append(row)
        del run
    torch.cuda.synchronize()
    out["seconds"] = time.perf_counter() - t0
    out["realizations"] = realizations
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--exp", default="fig2,fig3,fig3h,fig4,fig4h,fig5",
                    help="comma list of " + ", ".join(EXPERIMENTS))
    ap.add_argument("--K", type=int, default=10_000, help="realizations averaged (error-of-average experiments)")
    ap.add_argument("--trials", type=int, default=100, help="single realizations (trial experiments)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--scope", choices=("level", "node"), default="level")
    ap.add_argument("--leaf", choices=sorted(rbc.LEAF_NAMES), default=None,
                    help="leaf arithmetic instead of the paper's (f32 experiments only)")
    ap.add_argument("--out", default=None, help="write the JSON summaries here (default: stdout)")
    args = ap.parse_args(argv)
    scope = rbc.DRAW_PER_LEVEL if args.scope == "level" else rbc.DRAW_PER_NODE
    res = []
    for name in args.exp.split(","):
        r = run_experiment(name.strip(), K=args.K, trials=args.trials, seed=args.seed, scope=scope, leaf=args.leaf)
        print(f"{name}: {r['realizations']} realizations in {r['seconds']:.2f} s", file=sys.stderr)
        res.append(r)
    text = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    else:
        print(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
