"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded
inputs and the same draws (Section 2.1.1 recursion, Prop. 10 tables).

Gates: fp64 leaves (fp64 I/O) relative Frobenius error <= 1e-12 against the oracle's
computation with the same draws; lower precisions the normwise gate of tests/_helpers.py
and, beside it, an entrywise gate |C - C_oracle|_ij <= t g^L bound_ij with the same t and g
(bound_ij = (|A||B|)_ij on zero-mean inputs; on the badly scaled inputs the recursion mixes
rows and columns of different scales, so the bound sums |A| and |B| over the blocks each entry
is mixed with, tests/_helpers.entrywise_bound).
"""
import numpy as np
import pytest
import torch

from oracle import rbc_oracle as o
from rbc_inputs import gaussian, matrix_pair

from ._helpers import egate, entrywise, formula, gate, gpu_rbc, normwise, oracle_plan, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_07439_gb300 import build as b
    b.build()
    import paper_1905_07439_gb300 as pkg
    return pkg


@pytest.mark.parametrize("decode", [1, 2])
def test_strassen_n128_l2_fp64_seed0(rbc, decode):
    # Randomized Strassen, 2 levels, N = 128, fp64, seed 0, per-node draws, 32 x 32 leaves.
    U, V, W = formula("strassen")
    A, B = gaussian(128, 0), gaussian(128, 1)
    plan = rbc.Plan(U, V, W, levels=2, seed=0)
    C = gpu_rbc(rbc, plan, A, B, torch.float64, rbc.LEAF_F64, decode)
    ref = o.rbc(A, B, oracle_plan(U, V, W, 2, 0))
    assert rel(C, ref) <= 1e-12
    assert rel(C, A @ B) <= 1e-12


CASES_F64 = [
    # formula, L, N (ragged leaf sizes), mode, scope
    ("strassen", 0, 45, o.RAND_FULL, o.DRAW_PER_NODE),
    ("strassen", 1, 74, o.RAND_FULL, o.DRAW_PER_NODE),
    ("strassen", 2, 148, o.RAND_FULL, o.DRAW_PER_LEVEL),
    ("strassen", 3, 88, o.RAND_SIGN, o.DRAW_PER_NODE),
    ("strassen", 4, 16 * 9, o.RAND_PERM, o.DRAW_PER_NODE),
    ("strassen", 5, 32 * 3, o.RAND_FULL, o.DRAW_PER_NODE),      # 2801 draw sets: chunked passes
    ("strassen", 2, 4, o.RAND_FULL, o.DRAW_PER_NODE),          # m = 1
    ("laderman", 1, 3 * 70, o.RAND_FULL, o.DRAW_PER_NODE),
    ("laderman", 2, 9 * 13, o.RAND_FULL, o.DRAW_PER_NODE),
    ("laderman", 3, 27 * 5, o.RAND_NONE, o.DRAW_PER_NODE),
    ("noisy-strassen", 1, 2 * 130, o.RAND_FULL, o.DRAW_PER_NODE),
    ("noisy-strassen", 3, 8 * 17, o.RAND_FULL, o.DRAW_PER_LEVEL),
    ("noisy-laderman", 2, 9 * 11, o.RAND_FULL, o.DRAW_PER_NODE),
    # small leaves (exact-size product kernel unless the decode is fused): L = 0 direct
    # store, odd sizes, the largest small size and the first tiled one
    ("strassen", 0, 20, o.RAND_FULL, o.DRAW_PER_NODE),
    ("laderman", 0, 31, o.RAND_FULL, o.DRAW_PER_NODE),
    ("laderman", 1, 3 * 3, o.RAND_FULL, o.DRAW_PER_NODE),
    ("strassen", 1, 2 * 29, o.RAND_FULL, o.DRAW_PER_NODE),
    ("strassen", 1, 2 * 30, o.RAND_FULL, o.DRAW_PER_LEVEL),
    ("strassen", 1, 2 * 31, o.RAND_FULL, o.DRAW_PER_NODE),
]


@pytest.mark.parametrize("decode", [1, 2])
@pytest.mark.parametrize("name,L,N,mode,scope", CASES_F64)
def test_fp64_leaves_match_oracle(rbc, name, L, N, mode, scope, decode):
    U, V, W = formula(name, seed=1)
    A, B = matrix_pair("normal", N, seed=10 + L)
    seed = 1234 + N
    plan = rbc.Plan(U, V, W, levels=L, seed=seed, rand_mode=mode, draw_scope=scope)
    if decode == 1 and plan.info()["draw_count"] > 1024:
        # the fused decode needs every draw set of the tree in one launch's tables
        with pytest.raises(rbc.RbcError) as e:
            gpu_rbc(rbc, plan, A, B, torch.float64, rbc.LEAF_F64, decode)
        assert e.value.status == 7
        return
    C = gpu_rbc(rbc, plan, A, B, torch.float64, rbc.LEAF_F64, decode)
    ref = o.rbc(A, B, oracle_plan(U, V, W, L, seed, mode, scope))
    assert rel(C, ref) <= 1e-12


CASES_F32 = [
    ("strassen", 1, 2 * 300, "normal"),
    ("strassen", 2, 4 * 300, "normal"),
    ("strassen", 2, 4 * 300, "hard"),
    ("strassen", 3, 8 * 45, "normal"),
    ("laderman", 2, 9 * 100, "normal"),
    ("noisy-strassen", 2, 4 * 260, "normal"),
    ("strassen", 3, 8 * 10, "normal"),     # small leaves
    ("laderman", 1, 3 * 7, "hard"),
    ("strassen", 0, 26, "normal"),
    ("strassen", 1, 2 * 27, "normal"),
    ("noisy-laderman", 2, 9 * 37, "normal"),   # n0 = 3, table-driven encode and sparse decode
    ("noisy-laderman", 1, 3 * 64, "hard"),
]


@pytest.mark.parametrize("decode", [1, 2])
@pytest.mark.parametrize("name,L,N,dist", CASES_F32)
def test_fp32_leaves_match_oracle(rbc, name, L, N, dist, decode):
    U, V, W = formula(name, seed=2)
    A, B = matrix_pair(dist, N, seed=20 + L)
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    plan = rbc.Plan(U, V, W, levels=L, seed=99)
    C = gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_F32, decode)
    ref = o.rbc(A, B, oracle_plan(U, V, W, L, 99))
    n0 = U.shape[0]
    assert normwise(C, ref, A, B) <= gate("f32", n0, L, N)
    assert entrywise(C, ref, A, B, n0, L, mixed=dist == "hard") <= egate("f32", n0, L)


def test_argument_errors(rbc):
    U, V, W = formula("strassen")
    plan = rbc.Plan(U, V, W, levels=2)
    A = torch.zeros((130, 130), dtype=torch.float64, device="cuda")
    with pytest.raises(rbc.RbcError) as e:
        rbc.matmul(plan, A, A, leaf=rbc.LEAF_F64)
    assert e.value.status == 1
    A = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(rbc.RbcError) as e:
        rbc.matmul(plan, A, A, leaf=rbc.LEAF_F64, workspace=ws)
    assert e.value.status == 2
    with pytest.raises(rbc.RbcError) as e:
        rbc.matmul(plan, A, A, leaf=rbc.LEAF_BF16)
    assert e.value.status == 7


def test_norms_match_numpy(rbc):
    rng = np.random.default_rng(0)
    X = rng.standard_normal((333, 517))
    Y = rng.standard_normal((333, 517))
    Xt = torch.tensor(X, device="cuda")
    Yt = torch.tensor(Y, device="cuda", dtype=torch.float32)
    out = rbc.norms(Xt, Yt).cpu().numpy()
    Yf = Y.astype(np.float32).astype(np.float64)
    assert np.isclose(out[0], np.sum((X - Yf) ** 2), rtol=1e-12)
    assert np.isclose(out[1], np.sum(Yf**2), rtol=1e-12)
    out2 = rbc.norms(Xt).cpu().numpy()
    assert np.isclose(out2[0], np.sum(X**2), rtol=1e-12) and out2[1] == 0.0
    # deterministic: repeated calls are bit-identical
    assert np.array_equal(rbc.norms(Xt, Yt).cpu().numpy(), out)


TC_CASES = [
    # formula, L, N: classical ragged, both tile widths (mp % 256 == 0 and != 0), n0 = 3, approximate
    ("strassen", 0, 300),
    ("strassen", 1, 2 * 200),
    ("strassen", 2, 4 * 300),
    ("strassen", 2, 4 * 512),
    ("strassen", 3, 8 * 70),
    ("laderman", 2, 9 * 100),
    ("noisy-strassen", 2, 4 * 260),
    ("noisy-laderman", 2, 9 * 45),   # n0 = 3 outside the built-in formulas: table-driven passes
]


@pytest.mark.parametrize("leaf", ["tf32", "bf16", "f16", "3xbf16", "3xtf32", "bf16x6", "f16x3"])
@pytest.mark.parametrize("decode", [1, 2])
@pytest.mark.parametrize("name,L,N", TC_CASES)
def test_tensor_core_leaves_match_oracle(rbc, name, L, N, decode, leaf):
    U, V, W = formula(name, seed=3)
    A, B = matrix_pair("normal", N, seed=30 + L)
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    plan = rbc.Plan(U, V, W, levels=L, seed=555)
    C = gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_NAMES[leaf], decode)
    ref = o.rbc(A, B, oracle_plan(U, V, W, L, 555))
    err = normwise(C, ref, A, B)
    assert err <= gate(leaf, U.shape[0], L, N), (err, gate(leaf, U.shape[0], L, N))
    ent = entrywise(C, ref, A, B, U.shape[0], L)
    assert ent <= egate(leaf, U.shape[0], L), (ent, egate(leaf, U.shape[0], L))


def test_split_modes_are_fp32_accurate(rbc):
    # The compensated modes must be far more accurate than their single-pass counterparts.
    U, V, W = formula("strassen")
    N, L = 1024, 2
    A, B = matrix_pair("normal", N, seed=5)
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    plan = rbc.Plan(U, V, W, levels=L, seed=1)
    ref = o.rbc(A, B, oracle_plan(U, V, W, L, 1))
    errs = {leaf: rel(gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_NAMES[leaf]), ref)
            for leaf in ("f32", "tf32", "3xtf32", "bf16", "3xbf16")}
    assert errs["3xtf32"] < errs["tf32"] / 50
    assert errs["3xbf16"] < errs["bf16"] / 50
    assert errs["3xtf32"] < 4 * errs["f32"] + 1e-7


BF16X6_CASES = [
    # formula, L, N, distribution: exact and approximate formulas, n0 = 2 and 3, zero-mean and
    # entrywise-positive badly scaled inputs, classical (L = 0)
    ("strassen", 0, 1024, "normal"),
    ("strassen", 2, 4 * 256, "normal"),
    ("strassen", 2, 4 * 256, "hard"),
    ("strassen", 3, 8 * 128, "normal"),
    ("laderman", 2, 9 * 100, "normal"),
    ("laderman", 1, 3 * 300, "hard"),
    ("noisy-strassen", 2, 4 * 260, "normal"),
]


@pytest.mark.parametrize("name,L,N,dist", BF16X6_CASES)
def test_bf16x6_is_as_accurate_as_fp32_leaves(rbc, name, L, N, dist):
    """The six-product bf16 mode stores fp32 leaf operands exactly as three bf16 pieces and
    drops only products below 2^-24 of the leading one, so its distance to the fp64 oracle (same
    draws) is that of fp32 arithmetic: at most twice the fp32 CUDA-core leaves' distance on the
    same inputs, and within the fp32 gate."""
    U, V, W = formula(name, seed=4)
    A, B = matrix_pair(dist, N, seed=40 + L)
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    plan = rbc.Plan(U, V, W, levels=L, seed=808)
    ref = o.rbc(A, B, oracle_plan(U, V, W, L, 808))
    e32 = rel(gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_F32, 2), ref)
    C6 = gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_BF16X6, 2)
    e6 = rel(C6, ref)
    assert e6 <= 2.0 * e32, (e6, e32)
    assert entrywise(C6, ref, A, B, U.shape[0], L, mixed=dist == "hard") <= egate("bf16x6", U.shape[0], L)
    if dist == "normal":
        assert normwise(C6, ref, A, B) <= gate("bf16x6", U.shape[0], L, N)
        # the three-piece split is exact: against the two-piece split it gains by far where the
        # leaf products' rounding dominates (zero-mean inputs; on the scaled positive inputs the
        # fp32 encode of mixed row scales dominates both)
        e3 = rel(gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_3XBF16, 2), ref)
        assert e6 < e3 / 4, (e6, e3)


F16X3_CASES = [
    # formula, L, N, input class: zero-mean, badly scaled rows and columns (1e-3 .. 1e3), and
    # whole matrices far outside the fp16 range (2^-70 / 2^-40, 2^60 / 2^30), ragged leaves,
    # the classical product, both decodes
    ("strassen", 2, 4 * 200, "normal", 2),
    ("strassen", 1, 2 * 300, "hard", 2),
    ("strassen", 2, 4 * 128, "tiny", 1),
    ("strassen", 2, 4 * 128, "huge", 2),
    ("laderman", 2, 9 * 37, "normal", 2),
    ("noisy-strassen", 3, 8 * 50, "hard", 2),
    ("strassen", 0, 300, "huge", 0),
]


@pytest.mark.parametrize("name,L,N,dist,decode", F16X3_CASES)
def test_f16x3_is_as_accurate_as_fp32_leaves(rbc, name, L, N, dist, decode):
    """The f16x3 mode scales each leaf row of S and column of T by a power of two (from the row
    and column maxima of A and B and the formula's growth bound), stores two fp16 pieces (22
    significant bits) and drops only h1*h1' (2^-22 of the leading product): its distance to the
    fp64 oracle (same draws) stays within twice the fp32 CUDA-core leaves' on the same inputs, and
    within the fp32 gates, whatever the inputs' magnitude."""
    U, V, W = formula(name, seed=4)
    base = "normal" if dist in ("tiny", "huge") else dist
    A, B = matrix_pair(base, N, seed=50 + L)
    if dist == "tiny":
        A, B = A * 2.0**-70, B * 2.0**-40
    elif dist == "huge":
        A, B = A * 2.0**60, B * 2.0**30
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    plan = rbc.Plan(U, V, W, levels=L, seed=909)
    ref = o.rbc(A, B, oracle_plan(U, V, W, L, 909))
    e32 = rel(gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_F32, decode), ref)
    C3 = gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_F16X3, decode)
    e3 = rel(C3, ref)
    assert e3 <= 2.0 * e32, (e3, e32)
    n0 = U.shape[0]
    assert entrywise(C3, ref, A, B, n0, L, mixed=dist == "hard") <= egate("f16x3", n0, L)
    if dist != "hard":
        assert normwise(C3, ref, A, B) <= gate("f16x3", n0, L, N)


# Rounding of each leaf mode in the oracle's emulated-precision recursion (Section 2.2 model,
# every operation rounded): fp32 for the fp32-accurate modes, the leaf storage format for the
# others (the GPU accumulates in fp32, so it is never worse than rounding everything).
EMULATED = {"f32": o.round_fp32, "bf16x6": o.round_fp32, "f16x3": o.round_fp32, "3xtf32": o.round_tf32,
            "tf32": o.round_tf32,
            "3xbf16": o.round_bf16, "bf16": o.round_bf16, "f16": o.round_fp16}


@pytest.mark.parametrize("leaf", list(EMULATED))
@pytest.mark.parametrize("name,L,N", [("strassen", 1, 64), ("strassen", 2, 64), ("laderman", 1, 63),
                                      ("noisy-strassen", 2, 48)])
def test_error_within_emulated_precision(rbc, name, L, N, leaf):
    """Cross-check against the floating-point model: the GPU's distance to the fp64 oracle (same
    draws) is at most 4 times the oracle's own emulated-precision recursion's distance plus 1e-7
    (relative Frobenius), at N <= 64."""
    U, V, W = formula(name, seed=6)
    A, B = matrix_pair("normal", N, seed=60 + L)
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    plan = rbc.Plan(U, V, W, levels=L, seed=321)
    p = oracle_plan(U, V, W, L, 321)
    ref = o.rbc(A, B, p)
    emu = rel(o.rbc_emulated(A, B, p, EMULATED[leaf]), ref)
    got = rel(gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_NAMES[leaf]), ref)
    assert got <= 4.0 * emu + 1e-7, (got, emu)


@pytest.mark.parametrize("L,m,scope", [(2, 31, o.DRAW_PER_NODE), (2, 32, o.DRAW_PER_NODE), (2, 33, o.DRAW_PER_LEVEL),
                                       (2, 130, o.DRAW_PER_NODE), (3, 33, o.DRAW_PER_NODE), (3, 36, o.DRAW_PER_LEVEL)])
@pytest.mark.parametrize("leaf", ["f32", "bf16x6", "bf16", "f16x3"])
def test_laderman_two_level_encode(rbc, L, m, scope, leaf):
    """fp32 encodes of Laderman's formula run two levels per pass for leaves of at least 32 (the
    first level in shared memory, 128-position tiles): leaves across that threshold, ragged and
    spanning two tiles, per-node and per-level draws, against the oracle."""
    U, V, W = formula("laderman")
    N = 3**L * m
    A, B = matrix_pair("normal", N, seed=70 + m)
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    plan = rbc.Plan(U, V, W, levels=L, seed=2 * m + L, draw_scope=scope)
    ref = o.rbc(A, B, oracle_plan(U, V, W, L, 2 * m + L, scope=scope))
    C = gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_NAMES[leaf], 2)
    assert normwise(C, ref, A, B) <= gate(leaf, 3, L, N)
    assert entrywise(C, ref, A, B, 3, L) <= egate(leaf, 3, L)


DEEP_N02 = [
    # formula, L, m, draw scope: ragged leaves (element loads of the plain input), aligned ones
    # (vector path), a [1, 4] plan whose second pass chunks its per-node draw sets over launches,
    # dense perturbed coefficients, and the classical rule (R = 8, the largest R of the pass)
    ("strassen", 3, 37, o.DRAW_PER_NODE),
    ("strassen", 4, 21, o.DRAW_PER_NODE),
    ("strassen", 4, 64, o.DRAW_PER_LEVEL),
    ("strassen", 5, 12, o.DRAW_PER_NODE),
    ("noisy-strassen", 3, 40, o.DRAW_PER_NODE),
    ("noisy-strassen", 4, 17, o.DRAW_PER_LEVEL),
    ("classical2", 3, 24, o.DRAW_PER_NODE),
]


@pytest.mark.parametrize("name,L,m,scope", DEEP_N02)
@pytest.mark.parametrize("leaf", ["f32", "bf16x6", "bf16", "tf32", "f16x3"])
def test_n0_2_deep_encode(rbc, name, L, m, scope, leaf):
    """fp32 encodes of n0 = 2 formulas with R <= 8 run three- and four-level passes, the first one
    or two levels split over the CTAs (tf32 leaves keep two-level passes: their last pass
    writes transposed): against the oracle."""
    if name == "classical2":
        from rbc_inputs.formulas import classical_formula
        U, V, W = classical_formula(2)
    else:
        U, V, W = formula(name, seed=4)
    N = 2**L * m
    A, B = matrix_pair("normal", N, seed=90 + m)
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    seed = 3 * m + L
    plan = rbc.Plan(U, V, W, levels=L, seed=seed, draw_scope=scope)
    ref = o.rbc(A, B, oracle_plan(U, V, W, L, seed, scope=scope))
    C = gpu_rbc(rbc, plan, A, B, torch.float32, rbc.LEAF_NAMES[leaf], 2)
    assert normwise(C, ref, A, B) <= gate(leaf, 2, L, N)
    assert entrywise(C, ref, A, B, 2, L) <= egate(leaf, 2, L)


def test_workspace_status_word_clear_after_calls(rbc):
    import ctypes
    U, V, W = formula("strassen")
    plan = rbc.Plan(U, V, W, levels=1, seed=1)
    A = torch.randn((512, 512), device="cuda")
    ws = torch.empty(plan.workspace_size(512, rbc.IO_F32, rbc.LEAF_BF16), dtype=torch.uint8, device="cuda")
    rbc.matmul(plan, A, A, leaf=rbc.LEAF_BF16, workspace=ws)
    st = ctypes.c_int(-1)
    rbc.rbc.check(rbc.lib().rbc_workspace_check(ws.data_ptr(), None, ctypes.byref(st)), "check")
    assert st.value == 0


@pytest.mark.parametrize("leaf,decode", [("bf16", 2), ("3xbf16", 2), ("bf16", 1), ("bf16x6", 2), ("bf16x6", 1),
                                         ("f16x3", 2), ("f16x3", 1)])
def test_expired_wait_reports_timeout_and_the_context_survives(rbc, leaf, decode):
    """Failure detection without a fault.  With the stall test hook the leaf kernel issues no
    operand copies, so its MMA warp's bounded wait (2 s) expires: the kernel records
    RBC_ETIMEOUT in the workspace status word, releases its tensor memory and returns, and
    rbc_workspace_check reports it.  The next call on the same context and workspace is
    correct (the check cleared the word)."""
    import ctypes
    import time
    U, V, W = formula("strassen")
    N = 512
    plan = rbc.Plan(U, V, W, levels=1, seed=11)
    A, B = matrix_pair("normal", N, seed=12)
    A = A.astype(np.float32).astype(np.float64)
    B = B.astype(np.float32).astype(np.float64)
    At = torch.tensor(A, dtype=torch.float32, device="cuda")
    Bt = torch.tensor(B, dtype=torch.float32, device="cuda")
    lf = rbc.LEAF_NAMES[leaf]
    ws = torch.empty(plan.workspace_size(N, rbc.IO_F32, lf, decode), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    st = ctypes.c_int(-1)
    t0 = time.monotonic()
    rbc.matmul(plan, At, Bt, leaf=lf, workspace=ws, decode=decode, stall_leaf_copies=1)
    status = rbc.lib().rbc_workspace_check(ws.data_ptr(), None, ctypes.byref(st))
    waited = time.monotonic() - t0
    assert status == rbc.RBC_ETIMEOUT and st.value == rbc.RBC_ETIMEOUT, (status, st.value)
    assert 1.5 < waited < 60, waited
    C = rbc.matmul(plan, At, Bt, leaf=lf, workspace=ws, decode=decode)
    status = rbc.lib().rbc_workspace_check(ws.data_ptr(), None, ctypes.byref(st))
    assert status == rbc.RBC_OK and st.value == 0
    ref = o.rbc(A, B, oracle_plan(U, V, W, 1, 11))
    assert normwise(C.double().cpu().numpy(), ref, A, B) <= gate(leaf, 2, 1, N)


def test_stall_hook_needs_a_tensor_core_leaf_mode(rbc):
    U, V, W = formula("strassen")
    plan = rbc.Plan(U, V, W, levels=1, seed=11)
    A = torch.zeros((256, 256), device="cuda")
    with pytest.raises(rbc.RbcError) as e:
        rbc.matmul(plan, A, A, leaf=rbc.LEAF_F32, stall_leaf_copies=1)
    assert e.value.status == rbc.RBC_EINVAL
