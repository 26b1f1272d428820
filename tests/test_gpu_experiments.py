"""Realization batches (rbc_matmul_realizations), their error reductions
(rbc_realization_errors) and the Section 3 harness built on them.

  * every realization of a batch is bit-identical to the same plan run alone by rbc_matmul
    (staged decode), whatever the batch split, draw scope and table chunking;
  * realizations equal the oracle's with the same draws (fp64 gate; fp32 leaf gate);
  * the error reductions equal their definitions (Eqs. error-of-average, average-of-error)
    evaluated in numpy on the same outputs;
  * unbiasedness seen through the harness: the error of the average of K realizations of a
    perturbed Strassen formula (Section 3.1) falls like the per-realization spread / sqrt(K)
    (Props. 3 and 6), while the deterministic recursion keeps its error."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import rbc_oracle as o

from ._helpers import formula, gate, normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_07439_gb300 import build as b
    b.build()
    import paper_1905_07439_gb300 as pkg
    return pkg


def _inputs(N, seed, dtype):
    g = np.random.default_rng(seed)
    A, B = g.standard_normal((N, N)), g.standard_normal((N, N))
    return A, B, torch.tensor(A, dtype=dtype, device="cuda"), torch.tensor(B, dtype=dtype, device="cuda")


# (formula, levels, N, scope, rand mode)
CASES = [("noisy-strassen", 3, 80, "level", "full"), ("strassen", 2, 4 * 37, "node", "full"),
         ("laderman", 2, 9 * 11, "node", "sign"), ("noisy-strassen", 5, 320, "node", "perm"),
         ("laderman", 1, 3 * 40, "level", "full"), ("strassen", 4, 16 * 9, "level", "none"),
         # leaves of 33 and 40: fp32 encodes of Laderman's formula run two-level passes
         ("laderman", 2, 9 * 40, "level", "full"), ("laderman", 3, 27 * 33, "node", "full")]
MODES = {"full": 0, "sign": 1, "perm": 2, "none": 3}


@pytest.mark.parametrize("io", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-L{c[1]}-N{c[2]}-{c[3]}-{c[4]}")
def test_batch_equals_single_calls(rbc, case, io):
    name, L, N, scope, mode = case
    U, V, W = formula(name, seed=4)
    dt = torch.float64 if io == "f64" else torch.float32
    leaf = rbc.LEAF_F64 if io == "f64" else rbc.LEAF_F32
    sc = rbc.DRAW_PER_LEVEL if scope == "level" else rbc.DRAW_PER_NODE
    K = 7
    seeds = [100 + k for k in range(K)]
    plan = rbc.Plan(U, V, W, levels=L, seed=seeds[3], rand_mode=MODES[mode], draw_scope=sc)
    _, _, A, B = _inputs(N, 11, dt)
    ioc = rbc.IO_F64 if io == "f64" else rbc.IO_F32
    # a workspace for 3 realizations: batches of 3, 3, 1
    need3 = int(rbc.lib().rbc_realizations_workspace_size(plan.handle, N, ioc, leaf, 3))
    ws = torch.empty(need3, dtype=torch.uint8, device="cuda")
    Cs = torch.full((K, N, N), float("nan"), dtype=dt, device="cuda")
    rbc.realizations(plan, seeds, A, B, Cs, leaf=leaf, workspace=ws)
    whole = rbc.realizations(plan, seeds, A, B, leaf=leaf)  # everything in one batch
    torch.cuda.synchronize()
    assert torch.equal(Cs, whole)
    for k in (0, 3, 6):
        # a plan created with seed k computes realization k alone
        pk = rbc.Plan(U, V, W, levels=L, seed=seeds[k], rand_mode=MODES[mode], draw_scope=sc)
        one = rbc.matmul(pk, A, B, leaf=leaf, decode=2)
        torch.cuda.synchronize()
        assert torch.equal(Cs[k], one), k
    if L > 0 and mode != "none":
        assert not torch.equal(Cs[0], Cs[1])  # different draws give different realizations


@pytest.mark.parametrize("leaf", ["bf16", "3xbf16", "tf32", "f16x3"])
def test_batch_equals_single_calls_tensor_core_leaves(rbc, leaf):
    U, V, W = formula("laderman")
    N, L, K = 9 * 40, 2, 5   # leaves of 40: two-level encode passes
    plan = rbc.Plan(U, V, W, levels=L, seed=0)
    _, _, A, B = _inputs(N, 3, torch.float32)
    lf = rbc.LEAF_NAMES[leaf]
    need2 = int(rbc.lib().rbc_realizations_workspace_size(plan.handle, N, rbc.IO_F32, lf, 2))
    ws = torch.empty(need2, dtype=torch.uint8, device="cuda")
    Cs = rbc.realizations(plan, [7 + k for k in range(K)], A, B, leaf=lf, workspace=ws)
    torch.cuda.synchronize()
    for k in range(K):
        one = rbc.matmul(rbc.Plan(U, V, W, levels=L, seed=7 + k), A, B, leaf=lf, decode=2)
        torch.cuda.synchronize()
        assert torch.equal(Cs[k], one), k


@pytest.mark.parametrize("io", ["f64", "f32"])
def test_realizations_match_the_oracle(rbc, io):
    U, V, W = formula("noisy-strassen", seed=2)
    N, L = 80, 3
    dt = torch.float64 if io == "f64" else torch.float32
    leaf = rbc.LEAF_F64 if io == "f64" else rbc.LEAF_F32
    An, Bn, A, B = _inputs(N, 5, dt)
    for scope, osc in ((rbc.DRAW_PER_LEVEL, o.DRAW_PER_LEVEL), (rbc.DRAW_PER_NODE, o.DRAW_PER_NODE)):
        plan = rbc.Plan(U, V, W, levels=L, seed=0, draw_scope=scope)
        Cs = rbc.realizations(plan, [40 + k for k in range(5)], A, B, leaf=leaf).double().cpu().numpy()
        if io == "f32":
            An32, Bn32 = A.double().cpu().numpy(), B.double().cpu().numpy()
        for k in range(5):
            op = o.Plan(U, V, W, levels=L, seed=40 + k, mode=o.RAND_FULL, scope=osc)
            if io == "f64":
                ref = o.rbc(An, Bn, op)
                assert normwise(Cs[k], ref, An, Bn) <= 1e-12, (scope, k)
            else:
                ref = o.rbc(An32, Bn32, op)
                assert normwise(Cs[k], ref, An32, Bn32) <= gate("f32", 2, L, N), (scope, k)


@pytest.mark.parametrize("io", ["f64", "f32"])
@pytest.mark.parametrize("N", [80, 37, 130])
def test_error_reductions_equal_their_definitions(rbc, io, N):
    dt = torch.float64 if io == "f64" else torch.float32
    K = 301
    g = torch.Generator(device="cuda")
    g.manual_seed(N)
    Ref = torch.randn((N, N), generator=g, device="cuda", dtype=torch.float64)
    Cs = (Ref[None] + 0.1 * torch.randn((K, N, N), generator=g, device="cuda", dtype=torch.float64)).to(dt)
    each = rbc.realization_errors(Cs, Ref, rbc.ERR_EACH).cpu().numpy()
    avg = rbc.realization_errors(Cs, Ref, rbc.ERR_AVERAGE).cpu().numpy()
    again = rbc.realization_errors(Cs, Ref, rbc.ERR_AVERAGE).cpu().numpy()
    assert np.array_equal(avg, again)  # fixed summation order
    C = Cs.double().cpu().numpy()
    R = Ref.cpu().numpy()
    rn = np.linalg.norm(R)
    want_each = np.array([np.linalg.norm(C[k] - R) for k in range(K)]) / rn
    prefix = np.cumsum(C, axis=0) / np.arange(1, K + 1)[:, None, None]
    want_avg = np.array([np.linalg.norm(prefix[k] - R) for k in range(K)]) / rn
    np.testing.assert_allclose(each, want_each, rtol=1e-12)
    np.testing.assert_allclose(avg, want_avg, rtol=1e-10)


def test_error_reduction_arguments(rbc):
    Ref = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    Cs = torch.zeros((2, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        rbc.realization_errors(Cs, Ref.float())
    with pytest.raises(rbc.RbcError) as e:
        rbc.realization_errors(Cs, Ref, mode=5)
    assert e.value.status == 1
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(rbc.RbcError) as e:
        rbc.realization_errors(Cs, Ref, work=small)
    assert e.value.status == 2


def test_batch_arguments(rbc):
    U, V, W = formula("strassen")
    _, _, A, B = _inputs(64, 1, torch.float64)
    p1 = rbc.Plan(U, V, W, levels=2, seed=1)
    tiny = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(rbc.RbcError) as e:
        rbc.realizations(p1, [1, 2], A, B, leaf=rbc.LEAF_F64, workspace=tiny)
    assert e.value.status == 2
    Cs = torch.empty((2, 64, 64), dtype=torch.float64, device="cuda")
    st = rbc.lib().rbc_matmul_realizations(p1.handle, (ctypes.c_uint64 * 2)(1, 2), 2, A.data_ptr(), B.data_ptr(),
                                           Cs.data_ptr(), 64, 64, 64, 64, 64 * 63, rbc.IO_F64, rbc.LEAF_F64,
                                           tiny.data_ptr(), tiny.numel(), None)
    assert st == 1  # strideC < ldc * N: the outputs would overlap
    # L = 0: K copies of the standard product
    p0 = rbc.Plan(U, V, W, levels=0, seed=0)
    Cs = rbc.realizations(p0, [0, 1, 2], A, B, leaf=rbc.LEAF_F64)
    torch.cuda.synchronize()
    assert torch.equal(Cs[0], Cs[2])
    np.testing.assert_allclose(Cs[1].cpu().numpy(), (A @ B).cpu().numpy(), rtol=0, atol=1e-11)


def test_harness_unbiasedness(rbc):
    """Section 3.1 with a perturbed Strassen formula in fp64: the average of K realizations
    approaches AB (Props. 3 and 6) at the Monte-Carlo rate, the deterministic recursion does
    not move."""
    from paper_1905_07439_gb300 import experiments as ex
    U, V, W = formula("noisy-strassen", seed=0)
    from rbc_inputs.matrices import matrix_pair
    A, B = matrix_pair("normal", 80, 1000)
    run = ex.Runner(U, V, W, A, B, "f64")
    np.testing.assert_allclose(run.ref.cpu().numpy(), A @ B, rtol=0, atol=1e-11)
    K = 2048
    for Q in (1, 2, 3):
        Cs = run.realize(run.plan(Q, rbc.RAND_FULL, rbc.DRAW_PER_LEVEL), np.arange(K) + (7 << 20))
        each = run.errors(Cs, rbc.ERR_EACH)
        avg = run.errors(Cs, rbc.ERR_AVERAGE)
        rms = float(np.sqrt(np.mean(each**2)))
        assert avg[0] == pytest.approx(each[0], rel=1e-12)
        # E ||avg_K - AB||^2 = E ||F - AB||^2 / K for an unbiased estimator
        assert 0.3 * rms / np.sqrt(K) <= avg[-1] <= 3.0 * rms / np.sqrt(K), (Q, avg[-1], rms)
        det = run.realize(run.plan(Q, rbc.RAND_NONE, rbc.DRAW_PER_LEVEL), [0, 1])
        e_det = run.errors(det, rbc.ERR_AVERAGE)
        assert e_det[1] == pytest.approx(e_det[0], rel=1e-12)
        assert avg[-1] < 0.2 * e_det[0]


def test_harness_summary(rbc):
    from paper_1905_07439_gb300 import experiments as ex
    r = ex.run_experiment("fig4", K=64, levels=(1, 2))
    assert r["kind"] == "average" and r["realizations"] == 128
    (row,) = r["results"]
    assert row["standard"] > 0
    for entry in row["levels"]:
        ea = entry["full"]["error_of_average"]
        assert entry["full"]["n"][-1] == 64 and len(ea) == len(entry["full"]["n"])
        assert all(np.isfinite(ea)) and entry["deterministic"] > 0
    r = ex.run_experiment("fig5", trials=16, levels=(2,), dists=("adv1",))
    (row,) = r["results"]
    e = row["levels"][0]
    for var in ("full", "sign", "perm"):
        assert e[var]["min"] <= e[var]["median"] <= e[var]["max"]
