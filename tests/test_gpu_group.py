"""Grouped batches (rbc_group_*): every instance of a batch of uneven products equals the same
product computed alone by rbc_matmul, and the oracle within the leaf mode's gate; CUDA-graph
replay and autotuned configurations give the same results as eager execution."""
import numpy as np
import pytest
import torch

from oracle import rbc_oracle as o

from ._helpers import formula, gate, normwise, oracle_plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_07439_gb300 import build as b
    b.build()
    import paper_1905_07439_gb300 as pkg
    return pkg


# (formula, levels, N): leaf sizes all multiples of 256 (first batch) or ragged (second)
ALIGNED = [("strassen", 1, 512), ("strassen", 2, 1024), ("laderman", 1, 3 * 256), ("laderman", 2, 9 * 256),
           ("noisy-strassen", 1, 512), ("strassen", 0, 256)]
RAGGED = [("strassen", 1, 2 * 64), ("strassen", 2, 4 * 192), ("laderman", 1, 3 * 64), ("laderman", 2, 9 * 64),
          ("noisy-strassen", 2, 4 * 320), ("strassen", 0, 192), ("strassen", 1, 2 * 448)]


def _batch(rbc, specs, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    plans, As, Bs, Cs = [], [], [], []
    for i, (name, L, N) in enumerate(specs):
        U, V, W = formula(name, seed=i)
        plans.append(rbc.Plan(U, V, W, levels=L, seed=seed * 100 + i))
        As.append(torch.randn((N, N), generator=g, device="cuda"))
        Bs.append(torch.randn((N, N), generator=g, device="cuda"))
        Cs.append(torch.full((N, N), float("nan"), device="cuda"))
    return plans, As, Bs, Cs


@pytest.mark.parametrize("leaf", ["bf16", "3xbf16", "tf32", "bf16x6", "f16x3"])
@pytest.mark.parametrize("specs", [ALIGNED, RAGGED], ids=["aligned", "ragged"])
def test_group_equals_individual_products(rbc, specs, leaf):
    plans, As, Bs, Cs = _batch(rbc, specs, seed=3)
    grp = rbc.Group(plans, As, Bs, Cs, rbc.LEAF_NAMES[leaf])
    ws = torch.empty(grp.workspace_size(), dtype=torch.uint8, device="cuda")
    grp.run(ws)
    torch.cuda.synchronize()
    for i, (name, L, N) in enumerate(specs):
        ref = rbc.matmul(plans[i], As[i], Bs[i], leaf=rbc.LEAF_NAMES[leaf], decode=2)
        torch.cuda.synchronize()
        got = Cs[i].double().cpu().numpy()
        assert np.isfinite(got).all(), i
        A, B = As[i].double().cpu().numpy(), Bs[i].double().cpu().numpy()
        assert normwise(got, ref.double().cpu().numpy(), A, B) <= 1e-7, i
    # two instances against the oracle (same draws)
    for i in (1, 3):
        name, L, N = specs[i]
        U, V, W = formula(name, seed=i)
        A, B = As[i].double().cpu().numpy(), Bs[i].double().cpu().numpy()
        ref = o.rbc(A, B, oracle_plan(U, V, W, L, 3 * 100 + i))
        assert normwise(Cs[i].double().cpu().numpy(), ref, A, B) <= gate(leaf, U.shape[0], L, N)


def test_graph_replay_and_tuning_keep_results(rbc):
    plans, As, Bs, Cs = _batch(rbc, ALIGNED, seed=5)
    grp = rbc.Group(plans, As, Bs, Cs, rbc.LEAF_BF16)
    ws = torch.empty(grp.workspace_size(), dtype=torch.uint8, device="cuda")
    grp.run(ws)
    torch.cuda.synchronize()
    eager = [c.clone() for c in Cs]
    for c in Cs:
        c.fill_(float("nan"))
    grp.run(ws, graph=True)   # captures
    grp.run(ws, graph=True)   # replays
    torch.cuda.synchronize()
    for a, b in zip(eager, Cs):
        assert torch.equal(a, b)
    t = grp.tune(ws)
    # bn 128 with one or two CTAs per SM and bn 256 with one, each in three tile orders
    assert t["candidates"] == 9 and t["bn"] in (128, 256) and t["best_ms"] > 0
    assert t["ctas_per_sm"] in (1, 2) and (t["ctas_per_sm"] == 1 or t["bn"] == 128)
    for c in Cs:
        c.fill_(float("nan"))
    grp.run(ws, graph=True)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(eager, Cs)):
        A, B = As[i].double().cpu().numpy(), Bs[i].double().cpu().numpy()
        assert normwise(b.double().cpu().numpy(), a.double().cpu().numpy(), A, B) <= 1e-7


CONFIGS = [(128, 0, 1), (128, 1, 2), (128, 8, 2), (128, 16, 1), (256, 2, 1)]


@pytest.mark.parametrize("leaf", ["bf16", "tf32", "bf16x6", "f16x3"])
@pytest.mark.parametrize("specs", [ALIGNED, RAGGED], ids=["aligned", "ragged"])
def test_every_configuration_gives_the_same_products(rbc, specs, leaf):
    """Tile width, tile order and CTAs per SM (rbc_group_configure) change the speed only:
    each tile runs the same instruction sequence, so for one tile width every configuration
    gives bit-identical products; the two tile widths agree to rounding."""
    plans, As, Bs, Cs = _batch(rbc, specs, seed=7)
    grp = rbc.Group(plans, As, Bs, Cs, rbc.LEAF_NAMES[leaf])
    ws = torch.empty(grp.workspace_size(), dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    first = {}
    for bn, group, ctas in CONFIGS:
        if (bn == 256 and specs is RAGGED) or (leaf in ("bf16x6", "f16x3") and (bn == 256 or ctas == 2)):
            # 256-wide tiles need padded leaves divisible by 256; bf16x6 and f16x3 take
            # 128-wide tiles, one CTA per SM
            with pytest.raises(rbc.RbcError) as e:
                grp.configure(bn, group, ctas)
            assert e.value.status == 1
            continue
        grp.configure(bn, group, ctas)
        for c in Cs:
            c.fill_(float("nan"))
        grp.run(ws, stream=side, graph=(ctas == 2))
        torch.cuda.synchronize()
        got = [c.clone() for c in Cs]
        if bn not in first:
            first[bn] = got
        for i, (a, b) in enumerate(zip(first[bn], got)):
            assert torch.equal(a, b), (bn, group, ctas, i)
    if 256 in first:
        for i, (a, b) in enumerate(zip(first[128], first[256])):
            A, B = As[i].double().cpu().numpy(), Bs[i].double().cpu().numpy()
            assert normwise(b.double().cpu().numpy(), a.double().cpu().numpy(), A, B) <= 1e-7, i


def test_configuration_arguments(rbc):
    plans, As, Bs, Cs = _batch(rbc, ALIGNED[:2], seed=9)
    split = rbc.Group(plans, As, Bs, Cs, rbc.LEAF_3XBF16)
    for bn, group, ctas in [(64, 0, 1), (128, 3, 1), (128, 0, 3), (256, 0, 2)]:
        with pytest.raises(rbc.RbcError) as e:
            split.configure(bn, group, ctas)
        assert e.value.status == 1, (bn, group, ctas)
    with pytest.raises(rbc.RbcError):
        split.configure(128, 0, 2)        # two CTAs per SM: plain leaf modes only
    split.configure(256, 8, 1)
