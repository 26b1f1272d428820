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


@pytest.mark.parametrize("leaf", ["bf16", "3xbf16", "tf32"])
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
    assert t["candidates"] == 6 and t["bn"] in (128, 256) and t["best_ms"] > 0
    for c in Cs:
        c.fill_(float("nan"))
    grp.run(ws, graph=True)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(eager, Cs)):
        A, B = As[i].double().cpu().numpy(), Bs[i].double().cpu().numpy()
        assert normwise(b.double().cpu().numpy(), a.double().cpu().numpy(), A, B) <= 1e-7
