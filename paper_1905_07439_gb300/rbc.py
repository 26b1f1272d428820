"""ctypes binding of librbc (include/rbc.h): the same entry points, argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts Python/torch
arguments to pointers and sizes and turns non-zero statuses into exceptions.  There is no
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

# enums (include/rbc.h)
RBC_OK, RBC_EINVAL, RBC_ENOMEM, RBC_ECUDA, RBC_ETIMEOUT, RBC_EBUSY, RBC_EKAPPA, RBC_EUNSUPPORTED = range(8)
IO_F64, IO_F32 = 0, 1
LEAF_F64, LEAF_F32, LEAF_TF32, LEAF_BF16, LEAF_F16, LEAF_3XBF16, LEAF_3XTF32, LEAF_BF16X6, LEAF_F16X3 = range(9)
RAND_FULL, RAND_SIGN, RAND_PERM, RAND_NONE = range(4)
DRAW_PER_NODE, DRAW_PER_LEVEL = 0, 1
ERR_EACH, ERR_AVERAGE = 0, 1
LEAF_NAMES = {"f64": LEAF_F64, "f32": LEAF_F32, "tf32": LEAF_TF32, "bf16": LEAF_BF16,
              "f16": LEAF_F16, "3xbf16": LEAF_3XBF16, "3xtf32": LEAF_3XTF32, "bf16x6": LEAF_BF16X6,
              "f16x3": LEAF_F16X3}


class rbc_plan_desc(C.Structure):
    _fields_ = [("U", C.POINTER(C.c_double)), ("V", C.POINTER(C.c_double)), ("W", C.POINTER(C.c_double)),
                ("R", C.c_int), ("n0", C.c_int), ("levels", C.c_int), ("seed", C.c_uint64),
                ("rand_mode", C.c_int), ("draw_scope", C.c_int), ("rescale_kappa", C.c_int)]


class rbc_plan_info(C.Structure):
    _fields_ = [("R", C.c_int), ("n0", C.c_int), ("levels", C.c_int), ("rand_mode", C.c_int),
                ("draw_scope", C.c_int), ("draw_count", C.c_int64), ("leaf_count", C.c_int64),
                ("kappa", C.c_double), ("tau", C.c_double), ("gamma", C.c_double),
                ("scale", C.c_double), ("seed", C.c_uint64), ("builtin_formula", C.c_int)]


class rbc_group_item(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("A", C.c_void_p), ("B", C.c_void_p), ("C", C.c_void_p),
                ("N", C.c_int64), ("lda", C.c_int64), ("ldb", C.c_int64), ("ldc", C.c_int64)]


class rbc_group_tuning(C.Structure):
    _fields_ = [("bn", C.c_int), ("group", C.c_int), ("candidates", C.c_int), ("best_ms", C.c_float),
                ("ctas_per_sm", C.c_int)]


RBC_GROUP_GRAPH = 1


class rbc_request(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("A", C.c_void_p), ("B", C.c_void_p), ("C", C.c_void_p),
                ("N", C.c_int64), ("lda", C.c_int64), ("ldb", C.c_int64), ("ldc", C.c_int64),
                ("io_dtype", C.c_int), ("leaf_dtype", C.c_int)]


class rbc_queue_info(C.Structure):
    _fields_ = [("pending", C.c_int64), ("running", C.c_int64), ("admitted", C.c_uint64),
                ("completed", C.c_uint64), ("workspace_used", C.c_size_t), ("workspace_peak", C.c_size_t),
                ("workspace_cap", C.c_size_t), ("peak_running", C.c_int)]


class rbc_matmul_opts(C.Structure):
    _fields_ = [("decode", C.c_int), ("stall_leaf_copies", C.c_int), ("reserved", C.c_int * 6),
                ("events", C.c_void_p * 4),
                ("launches", C.c_int64)]


# name -> (restype, argtypes): every function include/rbc.h declares
_P = C.c_void_p
SIGNATURES = {
    "rbc_plan_create": (C.c_int, [C.POINTER(C.c_double)] * 3 + [C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(_P)]),
    "rbc_plan_create_ex": (C.c_int, [C.POINTER(rbc_plan_desc), C.POINTER(_P)]),
    "rbc_plan_destroy": (None, [_P]),
    "rbc_plan_query": (C.c_int, [_P, C.POINTER(rbc_plan_info)]),
    "rbc_plan_draws": (C.c_int, [_P, C.c_int64, C.c_int64, C.POINTER(C.c_int8), C.POINTER(C.c_int8)]),
    "rbc_plan_tables": (C.c_int, [_P, C.c_int64] + [C.POINTER(C.c_double)] * 3),
    "rbc_workspace_size": (C.c_size_t, [_P, C.c_int64, C.c_int, C.c_int]),
    "rbc_workspace_size_ex": (C.c_size_t, [_P, C.c_int64, C.c_int, C.c_int, C.POINTER(rbc_matmul_opts)]),
    "rbc_matmul": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int,
                             _P, C.c_size_t, _P]),
    "rbc_matmul_ex": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int,
                                _P, C.c_size_t, _P, C.POINTER(rbc_matmul_opts)]),
    "rbc_workspace_check": (C.c_int, [_P, _P, C.POINTER(C.c_int)]),
    "rbc_group_create": (C.c_int, [C.POINTER(rbc_group_item), C.c_int, C.c_int, C.POINTER(_P)]),
    "rbc_group_workspace_size": (C.c_size_t, [_P]),
    "rbc_group_run": (C.c_int, [_P, _P, C.c_size_t, _P, C.c_int]),
    "rbc_group_tune": (C.c_int, [_P, _P, C.c_size_t, _P, C.POINTER(rbc_group_tuning)]),
    "rbc_group_configure": (C.c_int, [_P, C.POINTER(rbc_group_tuning)]),
    "rbc_group_destroy": (None, [_P]),
    "rbc_queue_create": (C.c_int, [C.c_int, C.c_size_t, C.c_int, C.POINTER(_P)]),
    "rbc_batch_submit": (C.c_int, [_P, C.POINTER(rbc_request), C.c_int, C.POINTER(C.c_uint64)]),
    "rbc_batch_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_int)]),
    "rbc_queue_stats": (C.c_int, [_P, C.POINTER(rbc_queue_info)]),
    "rbc_queue_destroy": (None, [_P]),
    "rbc_matmul_static": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int,
                                    C.c_int, _P]),
    "rbc_static_scratch_bytes": (C.c_size_t, []),
    "rbc_static_scratch_check": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "rbc_static_scratch_ptr": (C.c_void_p, []),
    "rbc_norms": (C.c_int, [_P, _P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int, _P, _P,
                            C.c_size_t, _P]),
    "rbc_norms_work_size": (C.c_size_t, []),
    "rbc_realizations_workspace_size": (C.c_size_t, [_P, C.c_int64, C.c_int, C.c_int, C.c_int64]),
    "rbc_matmul_realizations": (C.c_int, [_P, C.POINTER(C.c_uint64), C.c_int64, _P, _P, _P, C.c_int64, C.c_int64,
                                          C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int, _P, C.c_size_t, _P]),
    "rbc_realization_errors": (C.c_int, [_P, C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_int64, _P, C.c_int64,
                                         C.c_int, _P, _P, C.c_size_t, _P]),
    "rbc_realization_errors_work_size": (C.c_size_t, [C.c_int64, C.c_int64]),
    "rbc_status_string": (C.c_char_p, [C.c_int]),
    "rbc_last_error": (C.c_char_p, []),
    "rbc_version": (C.c_int, []),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded librbc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_1905_07439_gb300.build.build()")
        L = C.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class RbcError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.rbc_last_error().decode()
        super().__init__(f"{where}: {L.rbc_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def check(status: int, where: str):
    if status != RBC_OK:
        raise RbcError(status, where)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Plan:
    """Owner of an rbc_plan_t (rbc_plan_create_ex)."""

    def __init__(self, U, V, W, levels: int, seed: int = 0, rand_mode: int = RAND_FULL,
                 draw_scope: int = DRAW_PER_NODE, rescale_kappa: int = -1):
        L = lib()
        self._keep = [np.ascontiguousarray(np.asarray(t, dtype=np.float64)) for t in (U, V, W)]
        U_, V_, W_ = self._keep
        n0, n0b, R = U_.shape
        if n0 != n0b or V_.shape != U_.shape or W_.shape != U_.shape:
            raise ValueError("U, V, W must all have shape (n0, n0, R)")
        d = rbc_plan_desc(_dptr(U_), _dptr(V_), _dptr(W_), R, n0, levels, seed & (2**64 - 1),
                          rand_mode, draw_scope, rescale_kappa)
        h = _P()
        check(L.rbc_plan_create_ex(C.byref(d), C.byref(h)), "rbc_plan_create_ex")
        self.handle = h
        self.n0, self.R, self.levels = n0, R, levels

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib().rbc_plan_destroy(h)
            self.handle = None

    def info(self) -> dict:
        i = rbc_plan_info()
        check(lib().rbc_plan_query(self.handle, C.byref(i)), "rbc_plan_query")
        return {f: getattr(i, f) for f, _ in rbc_plan_info._fields_}

    def draws(self, first: int = 0, count: int | None = None):
        info = self.info()
        count = info["draw_count"] - first if count is None else count
        perms = np.zeros((count, 3, self.n0), dtype=np.int8)
        signs = np.zeros((count, 3, self.n0), dtype=np.int8)
        check(lib().rbc_plan_draws(self.handle, first, count,
                                   perms.ctypes.data_as(C.POINTER(C.c_int8)),
                                   signs.ctypes.data_as(C.POINTER(C.c_int8))), "rbc_plan_draws")
        return perms, signs

    def tables(self, key: int):
        out = [np.zeros((self.n0, self.n0, self.R)) for _ in range(3)]
        check(lib().rbc_plan_tables(self.handle, key, *[_dptr(t) for t in out]), "rbc_plan_tables")
        return tuple(out)

    def workspace_size(self, N: int, io: int, leaf: int, decode: int = 0) -> int:
        o = rbc_matmul_opts(decode)
        return int(lib().rbc_workspace_size_ex(self.handle, N, io, leaf, C.byref(o)))


def _io_of(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return IO_F64
    if t.dtype == torch.float32:
        return IO_F32
    raise TypeError("A, B, C must be float32 or float64 CUDA tensors")


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def matmul(plan: Plan, A, B, C_out=None, leaf: int = LEAF_F32, workspace=None, stream=None,
           decode: int = 0, events=None, stall_leaf_copies: int = 0):
    """C = F^(L)(A, B) through rbc_matmul_ex on torch CUDA tensors (row-major, unit column stride)."""
    import torch
    N = A.shape[0]
    if A.shape != (N, N) or B.shape != (N, N):
        raise ValueError("square N x N inputs required")
    if A.stride(1) != 1 or B.stride(1) != 1:
        raise ValueError("A and B need unit column stride")
    io = _io_of(A)
    if _io_of(B) != io:
        raise TypeError("A and B must have the same dtype")
    if C_out is None:
        C_out = torch.empty((N, N), dtype=A.dtype, device=A.device)
    need = plan.workspace_size(N, io, leaf, decode)
    if need == 0 and N > 0:
        # let the library report why (invalid combination)
        pass
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=A.device)
    o = rbc_matmul_opts(decode, stall_leaf_copies)
    if events is not None:
        for i, ev in enumerate(events):
            o.events[i] = ev.cuda_event if ev is not None else None
    check(lib().rbc_matmul_ex(plan.handle, A.data_ptr(), B.data_ptr(), C_out.data_ptr(), N,
                              A.stride(0), B.stride(0), C_out.stride(0), io, leaf,
                              workspace.data_ptr(), workspace.numel(), _stream_ptr(stream), C.byref(o)),
          "rbc_matmul_ex")
    return C_out


def norms(X, Y=None, stream=None, work=None, out=None):
    """(sum (X-Y)^2, sum Y^2) in fp64 via rbc_norms (device reduction); returns a 2-element
    float64 CUDA tensor."""
    import torch
    rows, cols = X.shape
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=X.device)
    if work is None:
        work = torch.empty(int(lib().rbc_norms_work_size()), dtype=torch.uint8, device=X.device)
    yt = _io_of(Y) if Y is not None else 0
    check(lib().rbc_norms(X.data_ptr(), Y.data_ptr() if Y is not None else None, rows, cols,
                          X.stride(0), Y.stride(0) if Y is not None else 0, _io_of(X), yt,
                          out.data_ptr(), work.data_ptr(), work.numel(), _stream_ptr(stream)),
          "rbc_norms")
    return out


def realizations(plan: Plan, seeds, A, B, C_out=None, leaf: int = LEAF_F32, workspace=None, stream=None,
                 batch=None):
    """Independent realizations of `plan`'s product, realization k drawn from seeds[k]
    (rbc_matmul_realizations); returns (or fills) a K x N x N tensor.  `batch` bounds how
    many realizations share the workspace at once (default: all)."""
    import torch
    sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64).reshape(-1))
    K, N = sd.size, A.shape[0]
    if A.shape != (N, N) or B.shape != (N, N) or A.stride(1) != 1 or B.stride(1) != 1:
        raise ValueError("square N x N inputs with unit column stride required")
    io = _io_of(A)
    if _io_of(B) != io:
        raise TypeError("A and B must have the same dtype")
    if C_out is None:
        C_out = torch.empty((K, N, N), dtype=A.dtype, device=A.device)
    if C_out.shape != (K, N, N) or C_out.stride(2) != 1:
        raise ValueError("C_out must be K x N x N with unit column stride")
    if workspace is None:
        b = K if batch is None else max(1, min(K, batch))
        need = int(lib().rbc_realizations_workspace_size(plan.handle, N, io, leaf, b))
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=A.device)
    check(lib().rbc_matmul_realizations(plan.handle, sd.ctypes.data_as(C.POINTER(C.c_uint64)), K, A.data_ptr(),
                                        B.data_ptr(), C_out.data_ptr(), N, A.stride(0), B.stride(0),
                                        C_out.stride(1), C_out.stride(0), io, leaf, workspace.data_ptr(),
                                        workspace.numel(), _stream_ptr(stream)),
          "rbc_matmul_realizations")
    return C_out


def realization_errors(Cs, Ref, mode: int = ERR_EACH, stream=None, work=None, out=None):
    """Relative Frobenius errors of the K x N x N realizations Cs against the fp64 reference
    Ref (rbc_realization_errors): per realization (ERR_EACH) or of the running average
    (ERR_AVERAGE).  Returns a K-element float64 CUDA tensor."""
    import torch
    K, N, _ = Cs.shape
    if Ref.dtype != torch.float64 or Ref.shape != (N, N) or Ref.stride(1) != 1 or Cs.stride(2) != 1:
        raise ValueError("Ref must be an N x N float64 tensor; Cs and Ref need unit column stride")
    if out is None:
        out = torch.empty(K, dtype=torch.float64, device=Cs.device)
    if work is None:
        work = torch.empty(int(lib().rbc_realization_errors_work_size(K, N)), dtype=torch.uint8, device=Cs.device)
    check(lib().rbc_realization_errors(Cs.data_ptr(), _io_of(Cs), K, N, Cs.stride(1), Cs.stride(0), Ref.data_ptr(),
                                       Ref.stride(0), mode, out.data_ptr(), work.data_ptr(), work.numel(),
                                       _stream_ptr(stream)), "rbc_realization_errors")
    return out


class Group:
    """Owner of an rbc_group_t: a batch of products whose leaf products share one launch."""

    def __init__(self, plans, As, Bs, Cs, leaf: int):
        self.items = (rbc_group_item * len(plans))()
        for i, (p, A, B, Cm) in enumerate(zip(plans, As, Bs, Cs)):
            N = A.shape[0]
            self.items[i] = rbc_group_item(p.handle.value, A.data_ptr(), B.data_ptr(), Cm.data_ptr(), N,
                                           A.stride(0), B.stride(0), Cm.stride(0))
        self._keep = (list(plans), list(As), list(Bs), list(Cs))
        h = _P()
        check(lib().rbc_group_create(self.items, len(plans), leaf, C.byref(h)), "rbc_group_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib().rbc_group_destroy(h)
            self.handle = None

    def workspace_size(self) -> int:
        return int(lib().rbc_group_workspace_size(self.handle))

    def run(self, workspace, stream=None, graph: bool = False):
        import torch
        if graph and stream is None:
            # graphs are captured on a created stream: run on a side stream ordered after and
            # before the caller's current stream
            cur = torch.cuda.current_stream()
            if getattr(self, "_side", None) is None:
                self._side = torch.cuda.Stream()
            self._side.wait_stream(cur)
            self.run(workspace, stream=self._side, graph=True)
            cur.wait_stream(self._side)
            return
        check(lib().rbc_group_run(self.handle, workspace.data_ptr(), workspace.numel(), _stream_ptr(stream),
                                  RBC_GROUP_GRAPH if graph else 0), "rbc_group_run")

    def tune(self, workspace, stream=None) -> dict:
        t = rbc_group_tuning()
        check(lib().rbc_group_tune(self.handle, workspace.data_ptr(), workspace.numel(), _stream_ptr(stream),
                                   C.byref(t)), "rbc_group_tune")
        return {"bn": t.bn, "group": t.group, "candidates": t.candidates, "best_ms": t.best_ms,
                "ctas_per_sm": t.ctas_per_sm}

    def configure(self, bn: int = 128, group: int = 0, ctas_per_sm: int = 1) -> None:
        """Apply a tile configuration (rbc_group_configure)."""
        t = rbc_group_tuning(bn=bn, group=group, candidates=0, best_ms=0.0, ctas_per_sm=ctas_per_sm)
        check(lib().rbc_group_configure(self.handle, C.byref(t)), "rbc_group_configure")


class Queue:
    """Owner of an rbc_queue_t (continuous-admission serving queue)."""

    def __init__(self, device: int = 0, workspace_cap: int = 1 << 30, streams: int = 16):
        h = _P()
        check(lib().rbc_queue_create(device, workspace_cap, streams, C.byref(h)), "rbc_queue_create")
        self.handle = h
        self._live = {}   # ticket -> tensors kept alive until collected

    def close(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib().rbc_queue_destroy(h)
            self.handle = None
            self._live.clear()

    __del__ = close

    def submit(self, plan: "Plan", A, B, C_out, leaf: int) -> int:
        io = _io_of(A)
        r = rbc_request(plan.handle.value, A.data_ptr(), B.data_ptr(), C_out.data_ptr(), A.shape[0],
                        A.stride(0), B.stride(0), C_out.stride(0), io, leaf)
        t = C.c_uint64()
        check(lib().rbc_batch_submit(self.handle, C.byref(r), 1, C.byref(t)), "rbc_batch_submit")
        self._live[t.value] = (plan, A, B, C_out)
        return t.value

    def poll(self, ticket: int) -> bool:
        """True once the request has finished (raises RbcError if it failed)."""
        d = C.c_int()
        st = lib().rbc_batch_poll(self.handle, ticket, C.byref(d))
        if d.value:
            self._live.pop(ticket, None)
        check(st, "rbc_batch_poll")
        return bool(d.value)

    def stats(self) -> dict:
        i = rbc_queue_info()
        check(lib().rbc_queue_stats(self.handle, C.byref(i)), "rbc_queue_stats")
        return {f: getattr(i, f) for f, _ in rbc_queue_info._fields_}
