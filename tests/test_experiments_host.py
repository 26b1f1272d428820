"""Host-side pieces of the Section 3 harness (no GPU): the experiment table follows the
paper's sizes, and the summary grid covers 1..K."""
import pytest

ex = pytest.importorskip("paper_1905_07439_gb300.experiments")


def test_experiment_table_matches_section_3():
    for name, (kind, formula, io, N, levels, dists, variants) in ex.EXPERIMENTS.items():
        assert kind in ("average", "trials")
        # Section 3: 80 x 80 for the averages (Q <= 3), 320 x 320 for the trials (Q <= 5)
        assert (N, max(levels)) == ((80, 3) if kind == "average" else (320, 5)), name
        assert all(N % 2**Q == 0 for Q in levels)
        # Section 3.1: perturbed Strassen in double precision; Section 3.2: exact Strassen in single
        assert (formula, io) in (("noisy-strassen", "f64"), ("strassen", "f32")), name
        assert set(dists) <= set(ex.DISTS) and set(variants) <= set(ex.VARIANTS)
    assert set(ex.EXPERIMENTS["fig5"][6]) == {"full", "sign", "perm"}
    assert ex.EXPERIMENTS["fig5"][5] == ex.DISTS


@pytest.mark.parametrize("K", [1, 7, 64, 100, 10_000])
def test_log_grid(K):
    g = ex._log_grid(K)
    assert g[0] == 1 and g[-1] == K and g == sorted(set(g))
