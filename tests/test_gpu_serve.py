"""Serving queue (rbc_queue_* / rbc_batch_submit / rbc_batch_poll): every request's result in
the mix (concurrent admission, overlapping streams, grouped leaf launches) matches the FP64
oracle's recursion with the same draws within its leaf mode's gates, and is the same as the
request computed alone; admission never exceeds the workspace cap; failures are reported per
ticket without disturbing the other requests."""
import time

import numpy as np
import pytest
import torch

from oracle import rbc_oracle as o

from ._helpers import egate, entrywise, formula, gate, normwise, oracle_plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_07439_gb300 import build as b
    b.build()
    import paper_1905_07439_gb300 as pkg
    return pkg


MIX = [("strassen", 1, 512, "bf16"), ("laderman", 1, 3 * 128, "3xbf16"), ("noisy-strassen", 2, 1024, "3xbf16"),
       ("strassen", 3, 8 * 96, "bf16"), ("laderman", 2, 9 * 64, "bf16"), ("strassen", 2, 4 * 200, "f32"),
       ("strassen", 1, 2048, "3xbf16"), ("noisy-strassen", 1, 2 * 300, "tf32"), ("laderman", 1, 3 * 200, "f16"),
       ("strassen", 2, 1536, "bf16"), ("strassen", 1, 256, "f32"), ("laderman", 2, 9 * 128, "3xbf16"),
       ("strassen", 2, 4 * 256, "bf16x6"), ("laderman", 1, 3 * 256, "bf16x6"), ("strassen", 1, 512, "bf16"),
       ("strassen", 1, 512, "bf16"), ("noisy-strassen", 2, 4 * 128, "bf16x6"), ("strassen", 1, 2 * 384, "bf16x6"),
       ("strassen", 2, 4 * 128, "f16x3"), ("laderman", 1, 3 * 256, "f16x3")]


def _requests(rbc, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    out = []
    for i, (name, L, N, leaf) in enumerate(MIX):
        U, V, W = formula(name, seed=i)
        plan = rbc.Plan(U, V, W, levels=L, seed=seed + i)
        A = torch.randn((N, N), generator=g, device="cuda")
        B = torch.randn((N, N), generator=g, device="cuda")
        out.append((plan, A, B, rbc.LEAF_NAMES[leaf], leaf, U.shape[0], L, N))
    return out


def _wait(q, tickets, timeout=60.0):
    t0 = time.time()
    pending = set(tickets)
    while pending:
        for t in list(pending):
            if q.poll(t):
                pending.discard(t)
        assert time.time() - t0 < timeout, "queue did not finish"
        time.sleep(0.0005)


def test_same_alone_and_in_the_mix(rbc):
    reqs = _requests(rbc, seed=21)
    alone = []
    for plan, A, B, leaf, *_ in reqs:
        alone.append(rbc.matmul(plan, A, B, leaf=leaf))
    torch.cuda.synchronize()
    q = rbc.Queue(workspace_cap=8 << 30, streams=8)
    outs = [torch.full_like(A, float("nan")) for _, A, *_ in reqs]
    tickets = [q.submit(plan, A, B, Co, leaf) for (plan, A, B, leaf, *_), Co in zip(reqs, outs)]
    _wait(q, tickets)
    torch.cuda.synchronize()
    st = q.stats()
    assert st["completed"] == len(reqs) and st["peak_running"] >= 2
    for i, ((plan, A, B, leaf, lname, n0, L, N), a, m) in enumerate(zip(reqs, alone, outs)):
        An, Bn = A.double().cpu().numpy(), B.double().cpu().numpy()
        mix = m.double().cpu().numpy()
        # against the oracle's recursion with the request's own draws
        U, V, W = formula(MIX[i][0], seed=i)
        ref = o.rbc(An, Bn, oracle_plan(U, V, W, L, 21 + i))
        assert normwise(mix, ref, An, Bn) <= gate(lname, n0, L, N), (i, lname)
        assert entrywise(mix, ref, An, Bn, n0, L) <= egate(lname, n0, L), (i, lname)
        # and the same as alone
        err = normwise(mix, a.double().cpu().numpy(), An, Bn)
        assert err <= gate(lname, n0, L, N), (lname, L, N, err)
    q.close()


def test_admission_respects_the_workspace_cap(rbc):
    reqs = _requests(rbc, seed=33)
    need = [p.workspace_size(A.shape[0], rbc.IO_F32, leaf) for p, A, _, leaf, *_ in reqs]
    cap = 2 * max(need) + (1 << 20)
    q = rbc.Queue(workspace_cap=cap, streams=16)
    outs = [torch.empty_like(A) for _, A, *_ in reqs]
    tickets = [q.submit(p, A, B, Co, leaf) for (p, A, B, leaf, *_), Co in zip(reqs, outs)]
    _wait(q, tickets)
    st = q.stats()
    assert st["completed"] == len(reqs)
    assert 0 < st["workspace_peak"] <= cap
    assert st["workspace_used"] == 0
    q.close()


def test_failures_are_reported_per_ticket(rbc):
    U, V, W = formula("strassen")
    plan = rbc.Plan(U, V, W, levels=2, seed=1)
    good = torch.randn((512, 512), device="cuda")
    bad = torch.randn((130, 130), device="cuda")       # not a multiple of 4: invalid request
    q = rbc.Queue(workspace_cap=1 << 28, streams=4)
    t_bad = q.submit(plan, bad, bad, torch.empty_like(bad), rbc.LEAF_BF16)
    t_good = q.submit(plan, good, good, torch.empty_like(good), rbc.LEAF_BF16)
    with pytest.raises(rbc.RbcError) as e:
        _wait(q, [t_bad])
    assert e.value.status == 1
    _wait(q, [t_good])
    with pytest.raises(rbc.RbcError):
        q.poll(t_good)            # already collected
    huge = torch.empty((1, 1), device="cuda")
    big = rbc.Plan(U, V, W, levels=1, seed=1)
    with pytest.raises(rbc.RbcError) as e:   # workspace beyond the whole pool: refused at submit
        A = torch.empty((8192, 8192), device="cuda")
        q.submit(big, A, A, A, rbc.LEAF_BF16)
    assert e.value.status == 2
    del huge
    q.close()
