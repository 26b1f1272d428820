"""The allocation-free entry point rbc_matmul_static.

Some callers cannot obtain device memory at the moment they multiply: a framework that has
already reserved the whole device heap for its own allocator, programs allowed to allocate
only at start-up, code paths that have no way to recover from a failed allocation.  For
them the library offers rbc_matmul_static, which takes its scratch from a fixed array in
the library's device image.  These tests call it through the C ABI and check that it
returns the same product as rbc_matmul with a caller-provided workspace, on two calls in a
row with the same plan (the array keeps the previous call's contents), that a warmed-up call
changes the device's free memory by nothing, that an expired bounded wait is reported
through rbc_static_scratch_check, and that it refuses products whose scratch would not fit,
with a clear error.
"""
import ctypes

import numpy as np
import pytest
import torch

from ._helpers import formula, gate, normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_07439_gb300 import build as b
    b.build()
    import paper_1905_07439_gb300 as pkg
    return pkg


def _static_call(rbc, plan, A, B, C, leaf):
    N = A.shape[0]
    io = rbc.IO_F32 if A.dtype == torch.float32 else rbc.IO_F64
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return rbc.lib().rbc_matmul_static(plan.handle, A.data_ptr(), B.data_ptr(), C.data_ptr(), N,
                                       A.stride(0), B.stride(0), C.stride(0), io, leaf, stream)


def test_static_scratch_matches_workspace_entry_point(rbc):
    cases = [("strassen", 2, 4 * 192, "bf16", torch.float32),
             ("laderman", 1, 3 * 120, "3xbf16", torch.float32),
             ("strassen", 1, 2 * 300, "f16x3", torch.float32),   # leaf scales in the array too
             ("noisy-strassen", 2, 4 * 40, "f64", torch.float64)]
    g = torch.Generator(device="cuda")
    for i, (name, L, N, leaf_name, dt) in enumerate(cases):
        U, V, W = formula(name, seed=4)
        plan = rbc.Plan(U, V, W, levels=L, seed=100 + i)
        leaf = rbc.LEAF_NAMES[leaf_name]
        assert 0 < plan.workspace_size(N, rbc.IO_F32 if dt == torch.float32 else rbc.IO_F64, leaf) \
            <= rbc.lib().rbc_static_scratch_bytes()
        g.manual_seed(7 + i)
        A = torch.randn((N, N), generator=g, device="cuda", dtype=dt)
        B = torch.randn((N, N), generator=g, device="cuda", dtype=dt)
        C_static = torch.full((N, N), float("nan"), device="cuda", dtype=dt)
        rbc.rbc.check(_static_call(rbc, plan, A, B, C_static, leaf), "rbc_matmul_static")
        C_ref = rbc.matmul(plan, A, B, leaf=leaf)
        torch.cuda.synchronize()
        Cs, Cr = C_static.double().cpu().numpy(), C_ref.double().cpu().numpy()
        An, Bn = A.double().cpu().numpy(), B.double().cpu().numpy()
        assert np.isfinite(Cs).all()
        tol = 1e-12 if leaf_name == "f64" else gate(leaf_name, U.shape[0], L, N)
        assert normwise(Cs, Cr, An, Bn) <= tol


def test_static_scratch_allocates_nothing_and_keeps_no_stale_state(rbc):
    """A warmed-up static call leaves the device's free memory unchanged (it allocates nothing),
    and a second call with the same plan on new inputs gives that call's product: nothing the
    first call left in the shared array leaks into it."""
    U, V, W = formula("strassen")
    plan = rbc.Plan(U, V, W, levels=2, seed=17)
    N, leaf = 4 * 160, rbc.LEAF_BF16X6
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    A1, B1, A2, B2 = (torch.randn((N, N), generator=g, device="cuda") for _ in range(4))
    C1 = torch.full((N, N), float("nan"), device="cuda")
    C2 = torch.full((N, N), float("nan"), device="cuda")
    rbc.rbc.check(_static_call(rbc, plan, A1, B1, C1, leaf), "rbc_matmul_static")  # warm-up: modules loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rbc.rbc.check(_static_call(rbc, plan, A1, B1, C1, leaf), "rbc_matmul_static")
    rbc.rbc.check(_static_call(rbc, plan, A2, B2, C2, leaf), "rbc_matmul_static")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    st = ctypes.c_int(-1)
    assert rbc.lib().rbc_static_scratch_check(None, ctypes.byref(st)) == rbc.RBC_OK and st.value == 0
    for A, B, Cs in ((A1, B1, C1), (A2, B2, C2)):
        Cr = rbc.matmul(plan, A, B, leaf=leaf)
        torch.cuda.synchronize()
        An, Bn = A.double().cpu().numpy(), B.double().cpu().numpy()
        assert normwise(Cs.double().cpu().numpy(), Cr.double().cpu().numpy(), An, Bn) <= gate("bf16x6", 2, 2, N)


def test_static_scratch_status_word_reports_an_expired_wait(rbc):
    """The bounded waits of the tensor-core leaf kernel record RBC_ETIMEOUT in the status word at
    the start of the static array; rbc_static_scratch_check reports it and clears it.  The wait
    is made to expire without a fault by the stall test hook of rbc_matmul_ex (the array's
    address, from rbc_static_scratch_ptr, as its workspace): the kernel then issues no operand
    copies and its MMA warp gives up after 2 s."""
    U, V, W = formula("strassen")
    plan = rbc.Plan(U, V, W, levels=1, seed=23)
    N, leaf = 512, rbc.LEAF_BF16
    A = torch.randn((N, N), device="cuda")
    B = torch.randn((N, N), device="cuda")
    C = torch.empty((N, N), device="cuda")
    L = rbc.lib()
    ptr = L.rbc_static_scratch_ptr()
    assert ptr and ptr % 256 == 0
    o = rbc.rbc.rbc_matmul_opts(2, 1)   # staged decode, stall the leaf kernel's copies
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rbc.rbc.check(L.rbc_matmul_ex(plan.handle, A.data_ptr(), B.data_ptr(), C.data_ptr(), N, N, N, N, rbc.IO_F32,
                                  leaf, ptr, L.rbc_static_scratch_bytes(), stream, ctypes.byref(o)), "rbc_matmul_ex")
    st = ctypes.c_int(-1)
    assert L.rbc_static_scratch_check(None, ctypes.byref(st)) == rbc.RBC_ETIMEOUT
    assert st.value == rbc.RBC_ETIMEOUT
    assert L.rbc_static_scratch_check(None, ctypes.byref(st)) == rbc.RBC_OK and st.value == 0  # cleared
    # the context and the array stay usable
    Cs = torch.full((N, N), float("nan"), device="cuda")
    rbc.rbc.check(_static_call(rbc, plan, A, B, Cs, leaf), "rbc_matmul_static")
    Cr = rbc.matmul(plan, A, B, leaf=leaf)
    torch.cuda.synchronize()
    An, Bn = A.double().cpu().numpy(), B.double().cpu().numpy()
    assert normwise(Cs.double().cpu().numpy(), Cr.double().cpu().numpy(), An, Bn) <= gate("bf16", 2, 1, N)


def test_static_scratch_rejects_oversized_products(rbc):
    U, V, W = formula("strassen")
    plan = rbc.Plan(U, V, W, levels=2, seed=1)
    N = 4096
    assert plan.workspace_size(N, rbc.IO_F32, rbc.LEAF_BF16) > rbc.lib().rbc_static_scratch_bytes()
    A = torch.zeros((N, N), device="cuda")
    C = torch.zeros((N, N), device="cuda")
    st = _static_call(rbc, plan, A, A, C, rbc.LEAF_BF16)
    assert st == 2  # RBC_ENOMEM
    assert b"64 MiB" in rbc.lib().rbc_last_error()
