"""Host-side checks of the C-ABI library (no GPU): every symbol include/rbc.h declares is
exported, plan validation and error codes, and bit-exact agreement of the library's draws
and expanded tables (Prop. 10) with the oracle's independent implementation."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import rbc_oracle as o
from rbc_inputs import laderman, perturbed, strassen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rbc():
    from paper_1905_07439_gb300 import build as b
    b.build()
    import paper_1905_07439_gb300 as pkg
    return pkg


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(rbc_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(rbc):
    L = rbc.lib()
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
    # and the binding knows every one of them
    assert set(declared) <= set(rbc.SIGNATURES), set(declared) - set(rbc.SIGNATURES)
    assert L.rbc_version() >= 100


def test_status_strings(rbc):
    L = rbc.lib()
    for s in range(8):
        assert L.rbc_status_string(s)


def test_plan_validation_errors(rbc):
    U, V, W = strassen()
    with pytest.raises(rbc.RbcError) as e:
        rbc.Plan(U, V, 0.0 * W, levels=1)          # kappa == 1
    assert e.value.status == 6
    with pytest.raises(rbc.RbcError) as e:
        rbc.Plan(U, V, W, levels=9)
    assert e.value.status == 1
    with pytest.raises(rbc.RbcError):
        rbc.Plan(U, V, W, levels=1, rand_mode=7)
    Ub = U.copy()
    Ub[0, 0, 0] = np.nan
    with pytest.raises(rbc.RbcError):
        rbc.Plan(Ub, V, W, levels=1)


@pytest.mark.parametrize("fn,L,mode,scope", [
    (strassen, 2, o.RAND_FULL, o.DRAW_PER_NODE),
    (strassen, 4, o.RAND_FULL, o.DRAW_PER_NODE),
    (laderman, 3, o.RAND_FULL, o.DRAW_PER_NODE),
    (strassen, 3, o.RAND_SIGN, o.DRAW_PER_LEVEL),
    (laderman, 2, o.RAND_PERM, o.DRAW_PER_NODE),
    (strassen, 2, o.RAND_NONE, o.DRAW_PER_NODE),
])
def test_draws_bit_exact_vs_oracle(rbc, fn, L, mode, scope):
    U, V, W = fn()
    seed = 0xDEADBEEF12345
    p = rbc.Plan(U, V, W, levels=L, seed=seed, rand_mode=mode, draw_scope=scope)
    info = p.info()
    op = o.Plan(U, V, W, levels=L, seed=seed, mode=mode, scope=scope)
    n_draws = L if scope == o.DRAW_PER_LEVEL else op.node_count()
    assert info["draw_count"] == n_draws
    assert info["leaf_count"] == op.R ** L
    perms, signs = p.draws()
    for key in range(n_draws):
        d = o.node_draw(seed, key, op.n0, mode)
        assert [tuple(x) for x in perms[key]] == [tuple(x) for x in d.pi], key
        assert [tuple(x) for x in signs[key]] == [tuple(x) for x in d.s], key


@pytest.mark.parametrize("fn", [strassen, laderman])
def test_tables_bit_exact_vs_oracle(rbc, fn):
    U, V, W = perturbed(*fn(), seed=3, std=1e-3)
    p = rbc.Plan(U, V, W, levels=2, seed=77)
    op = o.Plan(U, V, W, levels=2, seed=77)
    info = p.info()
    assert info["kappa"] == op.kappa          # same sequential fp64 loop order
    assert abs(info["tau"] - o.tau(U, V, W)) <= 1e-15 * max(1.0, info["tau"])
    assert abs(info["gamma"] - o.gamma(U, V, W)) <= 1e-14 * info["gamma"]
    assert info["scale"] == op.scale
    for key in range(info["draw_count"]):
        got = p.tables(key)
        want = o.expand_tables(U, V, W, o.node_draw(77, key, op.n0, o.RAND_FULL), op.scale)
        for g, w_ in zip(got, want):
            assert np.array_equal(g, w_), key


def test_workspace_sizes(rbc):
    U, V, W = strassen()
    p = rbc.Plan(U, V, W, levels=2)
    assert p.workspace_size(128, rbc.IO_F64, rbc.LEAF_F64) > 0
    assert p.workspace_size(130, rbc.IO_F64, rbc.LEAF_F64) == 0       # not a multiple of 4
    assert p.workspace_size(128, rbc.IO_F64, rbc.LEAF_BF16) == 0      # fp64 I/O, bf16 leaves
    fused = p.workspace_size(4096, rbc.IO_F32, rbc.LEAF_F32, decode=1)
    staged = p.workspace_size(4096, rbc.IO_F32, rbc.LEAF_F32, decode=2)
    # both levels run in one pass (no intermediate): leaves 49 x 1024^2 per operand; the
    # staged decode adds the 49 leaf products
    assert fused >= 4 * 2 * 49 * 1024**2
    assert staged - fused >= 4 * 49 * 1024**2
    # four levels of Strassen run as one pass (the first two levels split over the CTAs): no
    # intermediate, only the bf16 leaves; beyond them only the 256-byte status word and
    # alignment.  Five levels add a one-level pass before it: one intermediate level (7 blocks
    # of 4096^2 fp32 per operand at N = 8192)
    p4 = rbc.Plan(U, V, W, levels=4)
    ws4 = p4.workspace_size(8192, rbc.IO_F32, rbc.LEAF_BF16, decode=1)
    body = 2 * 2 * 2401 * 512**2
    assert body <= ws4 <= body + 4096
    p5 = rbc.Plan(U, V, W, levels=5, draw_scope=rbc.DRAW_PER_LEVEL)  # fused decode: few draw sets
    ws5 = p5.workspace_size(8192, rbc.IO_F32, rbc.LEAF_BF16, decode=1)
    body5 = 2 * 4 * 7 * 4096**2 + 2 * 2 * 16807 * 256**2
    assert body5 <= ws5 <= body5 + 4096
    # split leaves store two bf16 panels per operand, bf16x6 three: the leaf operand bytes
    # grow by one and two panels; f16x3 stores two fp16 panels and six scale vectors of mp = 512
    # entries (row and column maxima, scales and their inverses)
    panel = 2 * 2 * 2401 * 512**2
    ws4_3x = p4.workspace_size(8192, rbc.IO_F32, rbc.LEAF_3XBF16, decode=1)
    ws4_6x = p4.workspace_size(8192, rbc.IO_F32, rbc.LEAF_BF16X6, decode=1)
    ws4_h3 = p4.workspace_size(8192, rbc.IO_F32, rbc.LEAF_F16X3, decode=1)
    assert ws4_3x - ws4 == panel and ws4_6x - ws4 == 2 * panel
    assert ws4_h3 - ws4 == panel + 6 * 512 * 4
    assert p4.workspace_size(8192, rbc.IO_F64, rbc.LEAF_F16X3) == 0   # fp32 I/O only


def test_laderman_encode_passes_cover_two_levels(rbc):
    """fp32 encodes of Laderman's formula run two levels per pass once leaves reach 32 (the first
    level in shared memory): at L = 3 only the depth-1 intermediate (23 blocks of 2187 rows in the
    padded layout: 9 column segments of 243 padded to 244) is stored per operand; below m = 32
    every level is a pass."""
    U, V, W = laderman()
    p3 = rbc.Plan(U, V, W, levels=3)
    ws = p3.workspace_size(6561, rbc.IO_F32, rbc.LEAF_BF16, decode=1)
    leaves = 2 * 2 * 12167 * 256**2
    body = 2 * 4 * 23 * 2187 * (9 * 244) + leaves
    assert body <= ws <= body + 4096
    small = rbc.Plan(U, V, W, levels=2)   # m = 27: one-level passes, depth-1 intermediate
    ws2 = small.workspace_size(9 * 27, rbc.IO_F32, rbc.LEAF_BF16, decode=1)
    assert ws2 >= 2 * 4 * 23 * 81 * 84


def test_empty_and_ragged_sizes_are_refused(rbc):
    """N must be a positive multiple of n0^L (the recursion splits N into n0^L equal blocks);
    an empty product and a ragged N are refused with RBC_EINVAL before any device memory is
    touched, and need no workspace."""
    U, V, W = strassen()
    p = rbc.Plan(U, V, W, levels=2)
    for n in (0, -4, 6):
        assert p.workspace_size(n, rbc.IO_F32, rbc.LEAF_BF16) == 0
    L = rbc.lib()
    fake = C.c_void_p(1 << 20)   # never dereferenced: the size check comes first
    for n in (0, -4, 6):
        st = L.rbc_matmul(p.handle, fake, fake, fake, n, max(n, 1), max(n, 1), max(n, 1),
                          rbc.IO_F32, rbc.LEAF_BF16, None, 0, None)
        assert st == 1, (n, st)


def test_builtin_formulas_are_recognised(rbc):
    """The library recognises exactly the Strassen and Laderman tensors (Section 1) and runs
    their one-level passes with compiled-in sparsity; any other formula is generic."""
    from rbc_inputs import formula_by_name, laderman, perturbed, strassen
    assert rbc.Plan(*strassen(), levels=1).info()["builtin_formula"] == 1
    assert rbc.Plan(*laderman(), levels=1).info()["builtin_formula"] == 2
    assert rbc.Plan(*formula_by_name("noisy-strassen"), levels=1).info()["builtin_formula"] == 0
    assert rbc.Plan(*perturbed(*laderman(), seed=3), levels=1).info()["builtin_formula"] == 0
    U, V, W = strassen()
    W = W.copy()
    W[0, 0, 0] = 2.0  # one coefficient changed: generic
    assert rbc.Plan(U, V, W, levels=1).info()["builtin_formula"] == 0


def _fake_group(rbc, specs, leaf):
    """A group over fake device pointers: creation computes layouts and the tile-width
    eligibility on the host and touches no memory."""
    from paper_1905_07439_gb300.rbc import rbc_group_item
    plans = [rbc.Plan(*fn(), levels=L, seed=1) for fn, L, _ in specs]
    items = (rbc_group_item * len(specs))()
    for i, (p, (_, _, N)) in enumerate(zip(plans, specs)):
        fake = C.c_void_p(1 << 30)
        items[i] = rbc_group_item(p.handle, fake, fake, fake, N, N, N, N)
    h = C.c_void_p()
    assert rbc.lib().rbc_group_create(items, len(specs), leaf, C.byref(h)) == 0
    return h, plans


def test_group_configuration_validation(rbc):
    """rbc_group_configure admits bn 128 always and bn 256 only when every padded leaf size is
    a multiple of 256; group orders 0, 1, 2, 4, 8, 16; two CTAs per SM only for plain leaf
    modes with bn 128.  Checked on the host (no launch)."""
    from paper_1905_07439_gb300.rbc import rbc_group_tuning
    L = rbc.lib()
    aligned = [(strassen, 1, 512), (strassen, 2, 1024), (laderman, 1, 768)]   # m = 256 each
    ragged = [(strassen, 1, 512), (strassen, 1, 2 * 320)]                       # m = 320 pads to 384
    cases = [
        (aligned, rbc.LEAF_BF16, [(128, 0, 1), (128, 8, 2), (256, 16, 1), (128, 2, 2)],
         [(64, 0, 1), (128, 3, 1), (128, 0, 3), (256, 0, 2)]),
        (aligned, rbc.LEAF_3XBF16, [(128, 1, 1), (256, 4, 1)], [(128, 0, 2), (256, 8, 2)]),
        (ragged, rbc.LEAF_TF32, [(128, 8, 1), (128, 0, 2)], [(256, 0, 1), (256, 8, 2)]),
        # three panels per operand: only 128-wide tiles fit two stages
        (aligned, rbc.LEAF_BF16X6, [(128, 0, 1), (128, 8, 1)], [(256, 0, 1), (128, 0, 2)]),
        # main and cross-term accumulator buffers fill TMEM at 128-wide tiles
        (aligned, rbc.LEAF_F16X3, [(128, 0, 1), (128, 4, 1)], [(256, 0, 1), (128, 0, 2)]),
    ]
    for specs, leaf, good, bad in cases:
        h, plans = _fake_group(rbc, specs, leaf)
        try:
            for bn, grp, ctas in good:
                t = rbc_group_tuning(bn=bn, group=grp, candidates=0, best_ms=0.0, ctas_per_sm=ctas)
                assert L.rbc_group_configure(h, C.byref(t)) == 0, (leaf, bn, grp, ctas)
            for bn, grp, ctas in bad:
                t = rbc_group_tuning(bn=bn, group=grp, candidates=0, best_ms=0.0, ctas_per_sm=ctas)
                assert L.rbc_group_configure(h, C.byref(t)) == 1, (leaf, bn, grp, ctas)
            assert L.rbc_group_configure(h, None) == 1
        finally:
            L.rbc_group_destroy(h)


def test_stall_hook_is_refused_for_simt_leaves(rbc):
    """The stall test hook applies to the tensor-core leaf kernel only; with a CUDA-core leaf
    mode rbc_matmul_ex refuses it before any device work."""
    from paper_1905_07439_gb300.rbc import rbc_matmul_opts
    p = rbc.Plan(*strassen(), levels=1, seed=1)
    fake = C.c_void_p(1 << 20)
    for leaf in (rbc.LEAF_F32, rbc.LEAF_F64):
        io = rbc.IO_F64 if leaf == rbc.LEAF_F64 else rbc.IO_F32
        o = rbc_matmul_opts(2, 1)
        st = rbc.lib().rbc_matmul_ex(p.handle, fake, fake, fake, 256, 256, 256, 256, io, leaf,
                                     fake, 1 << 30, None, C.byref(o))
        assert st == 1, (leaf, st)
