"""The synthetic input recipes of the batched and serving workloads (host only): the
properties their generators promise, checked on the generated lists."""
import math

import numpy as np

import bench


def test_batch_recipe():
    specs = bench.batch_specs(512)
    assert len(specs) == 512
    names = [s[0] for s in specs]
    assert set(names) == {"strassen", "laderman"}
    frac = names.count("strassen") / len(names)
    assert 0.42 < frac < 0.58                      # equal odds
    for name, L, n, seed in specs:
        n0 = 2 if name == "strassen" else 3
        q = n0**L * 64
        assert L in (1, 2)
        assert n % q == 0 and n // n0**L >= 64      # divisible into 64-multiple leaves
        assert 256 <= n < 4096 + q                  # log-uniform draw in [256, 4096], rounded up
    assert [s[3] for s in specs] == list(range(7000, 7512))   # per-instance seeds
    # log-uniform: about half of the draws fall below the geometric midpoint 1024
    below = sum(n <= 1024 + 9 * 64 for _, _, n, _ in specs) / len(specs)
    assert 0.35 < below < 0.7
    assert bench.batch_specs(512) == specs          # seeded


def test_serve_recipe():
    rate = 2000.0
    reqs = bench.serve_specs(10_000, rate)
    t = np.array([r["t"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() * rate - 1.0) < 0.05     # Poisson arrivals at the rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05   # exponential: coefficient of variation 1
    for r in reqs:
        n0 = 3 if r["formula"] == "laderman" else 2
        assert r["formula"] in ("strassen", "laderman", "noisy-strassen")
        assert r["dtype"] in ("fp32", "bf16-leaf", "3xbf16-leaf")
        assert 1 <= r["L"] <= 3
        assert r["n"] % (n0 ** r["L"] * 64) == 0
        assert 128 <= r["n"] < 8192 + n0**3 * 64
        if r["L"] > 1:                              # small n keep shallow recursions
            assert r["n"] >= 64 * n0 ** r["L"]
    for key, vals in (("formula", 3), ("dtype", 3), ("L", 3)):
        counts = np.unique([r[key] for r in reqs], return_counts=True)[1]
        assert len(counts) == vals and counts.min() > 0.15 * len(reqs)
    assert bench.serve_specs(10_000, rate) == reqs
