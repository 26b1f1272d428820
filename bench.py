"""Benchmark of the randomized bilinear computation on GB300.

Workload (one "step"): the at-scale fp32 sweep of exact and approximate formulas --
randomized Strassen N = 8192 with L = 1..4, randomized Laderman N = 6561 with L = 1..3,
and a perturbed Strassen (Section 3.1 recipe, std 1e-3) N = 4096 with L = 1..3 -- ten
rbc_matmul calls on fp32 I/O with A, B i.i.d. N(0,1) (seeded), per-node draws.

Metric: effective TFLOP/s = sum of 2 N^3 over the step / step time (device time, CUDA
events, inputs resident in HBM).  Every operand is larger than L2 or is followed by
workspace writes larger than L2 before its next use.  `e2e` times the same calls with the
host-to-device copies of A, B and the device-to-host copy of C inside the timed region.

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the
same workload.  Multi-GPU: the path does not shard (no collectives): N replicas.

Other workloads (--workload): precision (Strassen N = 16384, every leaf mode), batch (512
uneven instances in one grouped launch), serve (10,000 Poisson requests through the queue),
experiments (the Section 3 error experiments), peaks (cuBLAS GEMM throughput per dtype, as
context for the derived roofline peaks).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "effective TFLOP/s (2n³/t) + rel. Frobenius error vs FP64 oracle; served p50/p99"
WORKLOAD = "rbc-fp32-sweep: strassen n=8192 L=1..4, laderman n=6561 L=1..3, noisy-strassen(std 1e-3) n=4096 L=1..3"
CASES = [("strassen", 8192, L) for L in (1, 2, 3, 4)] + \
        [("laderman", 6561, L) for L in (1, 2, 3)] + \
        [("noisy-strassen", 4096, L) for L in (1, 2, 3)]
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x fp32 lanes x 2 flop x max clock
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense tensor rates (PFLOP/s): tf32 / bf16
NOMINAL_HBM_GBS = 8000.0     # nominal HBM3e bandwidth, beside the measured copy figure


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--leaf", default=None,
                    help="leaf mode; default for the sweep f16x3: fp32 I/O with three-product scaled fp16 "
                         "tensor-core leaves, as accurate as fp32 arithmetic (bf16x6 the six-product bf16 "
                         "alternative; 3xbf16, bf16, ... are the precision sweep); "
                         "default for the batch workload bf16")
    ap.add_argument("--cases", default="all", help="'all' or comma list of indices into the sweep")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--decode", type=int, default=0, help="0 auto, 1 fused, 2 staged")
    ap.add_argument("--no-errors", action="store_true", help="skip the error pass after the timing")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "batch", "serve", "experiments", "precision", "peaks"],
                    help="sweep: the at-scale fp32 sweep (default); batch: 512 uneven instances in one "
                         "grouped leaf launch replayed from a CUDA graph")
    ap.add_argument("--instances", type=int, default=512)
    ap.add_argument("--precision-n", type=int, default=16384, help="matrix size of the precision workload")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the bounded serving sub-run of the default sweep (0: skip)")
    ap.add_argument("--rate", type=float, default=2000.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--cap-gb", type=float, default=120.0, help="workspace admission cap of the queue")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Several GPUs run independent replicas of the workload (the path does not shard): one process
# per GPU, a barrier around the timed region, and the slowest rank's time for the whole job.
def init_dist(world, device):
    """Process group of the replicas: NCCL between GPUs, gloo on the host."""
    if world <= 1:
        return
    import torch.distributed as dist
    if not dist.is_initialized():
        if device.type == "cuda":
            dist.init_process_group("nccl", device_id=device)
        else:
            dist.init_process_group("gloo")


def max_over_ranks(x, world, device):
    """The largest x over the replicas (every rank gets it)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units every replica processed together, per second of the slowest replica."""
    return world * units_per_rank / seconds_max


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the step's ten leaf launches,
# summed over one ncu capture of the full sweep, keyed by (leaf mode, library version): a
# capture describes the kernel it measured only, so another library version reports null.
LEAF_TRAFFIC_STEP = {("bf16x6", 200): 46_604_675_328, ("f16x3", 201): 34_500_083_968}
# Stored panels per leaf operand and tensor-core products per leaf product of each leaf mode.
LEAF_PANELS = {"f32": 1, "tf32": 1, "bf16": 1, "f16": 1, "3xbf16": 2, "3xtf32": 2, "bf16x6": 3, "f16x3": 2}
LEAF_PRODUCTS = {"f32": 1, "tf32": 1, "bf16": 1, "f16": 1, "3xbf16": 3, "3xtf32": 3, "bf16x6": 6, "f16x3": 3}
LEAF_BYTES = {"f32": 4, "tf32": 4, "3xtf32": 4, "bf16": 2, "f16": 2, "3xbf16": 2, "bf16x6": 2, "f16x3": 2}


def case_flops(n, L, R, n0):
    m = n // n0**L
    return 2.0 * n**3, 2.0 * R**L * m**3


def run_ours(args):
    import numpy as np
    import torch

    import paper_1905_07439_gb300 as rbc
    from rbc_inputs import formula_by_name

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_dist(world, dev)
    leaf = rbc.LEAF_NAMES[args.leaf]
    sel = list(range(len(CASES))) if args.cases == "all" else [int(x) for x in args.cases.split(",")]
    cases = [CASES[i] for i in sel]

    # Inputs: per distinct N one seeded N(0,1) pair, resident on the device, plus pinned host copies.
    gen = torch.Generator(device="cpu")
    inputs = {}
    for _, n, _ in cases:
        if n in inputs:
            continue
        gen.manual_seed(1000 + n)
        A = torch.randn((n, n), generator=gen, dtype=torch.float32)
        B = torch.randn((n, n), generator=gen, dtype=torch.float32)
        inputs[n] = {"hA": A.pin_memory(), "hB": B.pin_memory(), "A": A.to(dev), "B": B.to(dev),
                     "C": torch.empty((n, n), dtype=torch.float32, device=dev),
                     "hC": torch.empty((n, n), dtype=torch.float32).pin_memory()}
    plans = []
    for name, n, L in cases:
        U, V, W = formula_by_name(name, seed=7)
        plans.append(rbc.Plan(U, V, W, levels=L, seed=2024 + L))
    ws_bytes = max(p.workspace_size(n, rbc.IO_F32, leaf, args.decode) for p, (_, n, _) in zip(plans, cases))
    if ws_bytes == 0:
        raise RuntimeError("invalid leaf mode for this workload")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def new_events():
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for e in evs:
            e.record(stream)   # materialize the CUDA event before handing it to the library
        return evs

    def step(events=None, counts=None):
        for i, (plan, (name, n, L)) in enumerate(zip(plans, cases)):
            x = inputs[n]
            o = rbc.rbc.rbc_matmul_opts(args.decode)
            if events is not None:
                for j, e in enumerate(events[i]):
                    o.events[j] = e.cuda_event
            import ctypes as C
            rbc.rbc.check(rbc.lib().rbc_matmul_ex(
                plan.handle, x["A"].data_ptr(), x["B"].data_ptr(), x["C"].data_ptr(), n, n, n, n,
                rbc.IO_F32, leaf, ws.data_ptr(), ws.numel(), C.c_void_p(stream.cuda_stream), C.byref(o)),
                "rbc_matmul_ex")
            if counts is not None:
                counts.append(o.launches)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    barrier()
    ev_sets = [[new_events() for _ in cases] for _ in range(args.steps)]
    counts = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        t0.record(stream)
        for s in range(args.steps):
            step(ev_sets[s], counts)
        t1.record(stream)
        barrier()
    ms_total = max_over_ranks(t0.elapsed_time(t1), world, dev)
    ms_step = ms_total / args.steps
    eff_flops = sum(case_flops(n, L, formula_by_name(nm, 7)[0].shape[2], formula_by_name(nm, 7)[0].shape[0])[0]
                    for nm, n, L in cases)
    value = whole_job_rate(eff_flops, world, ms_step * 1e-3) / 1e12

    # Leaf-product kernel (with fused decode): the dominant kernel.
    leaf_ms, leaf_flops, enc_ms, enc_bytes = 0.0, 0.0, 0.0, 0.0
    per_case, case_model = [], []
    leaf_bytes = 0.0
    es_leaf = LEAF_BYTES[args.leaf]
    split = LEAF_PRODUCTS[args.leaf]   # MMA passes per leaf product
    panels = LEAF_PANELS[args.leaf]    # stored operand panels
    reads_ab = 2 if args.leaf == "f16x3" else 1  # reads of A and B in the encode phase
    for i, (nm, n, L) in enumerate(cases):
        U = formula_by_name(nm, 7)[0]
        R, n0 = U.shape[2], U.shape[0]
        m = n // n0**L
        g = statistics.mean(ev_sets[s][i][1].elapsed_time(ev_sets[s][i][2]) for s in range(args.steps))
        e = statistics.mean(ev_sets[s][i][0].elapsed_time(ev_sets[s][i][1]) for s in range(args.steps))
        tot = statistics.mean(ev_sets[s][i][0].elapsed_time(ev_sets[s][i][3]) for s in range(args.steps))
        dec = statistics.mean(ev_sets[s][i][2].elapsed_time(ev_sets[s][i][3]) for s in range(args.steps))
        lf = split * 2.0 * R**L * m**3
        leaf_ms += g
        leaf_flops += lf
        # algorithmic leaf bytes: read both operands (all panels), write the fp32 products
        leaf_bytes += (2 * es_leaf * panels + 4) * R**L * m * m
        # algorithmic encode bytes: read A, B (twice for f16x3: the row / column maxima that set
        # the leaf scales, then the encode), write the leaf operands once
        eb = reads_ab * 2 * 4 * n * n + 2 * es_leaf * panels * R**L * m * m
        enc_ms += e
        enc_bytes += eb
        per_case.append({"formula": nm, "n": n, "L": L, "ms": round(tot, 3),
                         "eff_tflops": round(2.0 * n**3 / tot / 1e9, 2),
                         "leaf_ms": round(g, 3), "leaf_tflops": round(lf / g / 1e9, 2),
                         "encode_ms": round(e, 3), "encode_gbs": round(eb / e / 1e6, 1),
                         "decode_ms": round(dec, 3)})
        case_model.append((lf, eb + es_leaf * panels * 2 * R**L * m * m + 4 * n * n + 4 * 2 * R**L * m * m, tot))
    pk, pk_kind = peaks()
    if args.leaf in ("f32",):
        bound, peak, unit = "alu", FP32_PEAK_TFLOPS, "TFLOP/s"
        peak_note = "fp32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (derived)"
    else:
        # the leaf launches last about a millisecond each (their event times are summed), so the
        # burst figure is the ceiling; the sustained one is reported beside it
        ratio = TF32_PER_BF16 if args.leaf in ("tf32", "3xtf32") else 1.0
        bound, unit = "tensor", "TFLOP/s"
        peak = pk["bf16_tflops"] * ratio
        peak_note = (f"{pk_kind} bf16 burst x {ratio:.4f} (nominal {args.leaf}/bf16 ratio); achieved counts "
                     f"{split} tensor-core products per leaf product")
    achieved = leaf_flops / (leaf_ms * 1e-3) / 1e12
    roof = {"kernel": "tc_gemm_kernel / simt_gemm_kernel: the leaf products of all cases of the step "
                      "(achieved = their algorithmic flops / their summed event time)",
            "bound": bound, "achieved": round(achieved, 2),
            "peak": round(peak, 1), "unit": unit, "frac": round(achieved / peak, 4),
            "frac_of_sustained": (round(achieved / (pk["bf16_tflops_sustained"] * ratio), 4)
                                  if bound == "tensor" else None),
            "traffic": None,
            "algorithmic_bytes": round(leaf_bytes),
            "peak_source": peak_note,
            "encode": {"achieved_gbs": round(enc_bytes / (enc_ms * 1e-3) / 1e9, 1),
                       "peak_gbs": pk["hbm_gbs"], "frac": round(enc_bytes / (enc_ms * 1e-3) / 1e9 / pk["hbm_gbs"], 4),
                       "frac_of_nominal_8000": round(enc_bytes / (enc_ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
                       "bytes": round(enc_bytes),
                       "note": (f"algorithmic bytes: {reads_ab} read(s) of A and B, one write of the leaf "
                                "operands" + (" (f16x3: the row and column maxima read A and B first)"
                                              if reads_ab == 2 else ""))}}
    key = (args.leaf, int(rbc.lib().rbc_version()))
    if key in LEAF_TRAFFIC_STEP and len(cases) == len(CASES) and args.decode == 0:
        roof["traffic"] = LEAF_TRAFFIC_STEP[key]
        roof["traffic_note"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum over the step's 10 leaf "
                                f"launches (one capture of library version {key[1]}); compare algorithmic_bytes")
    # Whole-call model: leaf flops at the peak beside the algorithmic bytes (read A, B; write and
    # read the leaf operands; write and read M; write C) at the measured HBM bandwidth.
    t_sum = sum(f / (peak * 1e12) + b / (pk["hbm_gbs"] * 1e9) for f, b, _ in case_model) * 1e3
    t_max = sum(max(f / (peak * 1e12), b / (pk["hbm_gbs"] * 1e9)) for f, b, _ in case_model) * 1e3
    roof["whole_call"] = {"ms_measured": round(sum(t for _, _, t in case_model), 3),
                          "ms_model_sum": round(t_sum, 3), "ms_model_max": round(t_max, 3),
                          "frac_of_sum_model": round(t_sum / sum(t for _, _, t in case_model), 4),
                          "note": "model_sum = leaf flops / peak + algorithmic bytes / HBM per case; "
                                  "model_max takes the larger of the two per case"}
    launches_per_step = sum(counts) // max(1, args.steps)

    # End to end through the public API.  Every step copies its three input pairs (one per
    # size) from pinned host memory, runs the ten calls and copies their ten results back.
    # Copies run on their own streams: an input pair is copied once, when its first product
    # needs it, into one of two buffer sets alternating between steps; results go through two
    # alternating device buffers; so copies overlap computation.  The products run grouped by
    # size, smallest first, so that each group's input copy hides behind the previous group's
    # products; the cheapest product of the smallest size runs last, so that the result copy
    # after the last call is short.
    e2e = None
    if not args.no_e2e:
        h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        sizes = sorted({c[1] for c in cases})
        small = [i for i in range(len(cases)) if cases[i][1] == sizes[0]]
        last = min(small, key=lambda i: cases[i][2])
        order = [i for i in small if i != last] + \
                [i for n in sizes[1:] for i in range(len(cases)) if cases[i][1] == n] + [last]
        dins = [{n: {"A": inputs[n]["A"], "B": inputs[n]["B"]} for n in inputs},
                {n: {k: torch.empty_like(inputs[n]["A"]) for k in ("A", "B")} for n in inputs}]
        douts = [{n: inputs[n]["C"] for n in inputs}, {n: torch.empty_like(inputs[n]["C"]) for n in inputs}]
        hout = [{n: inputs[n]["hC"] for n in inputs},
                {n: torch.empty_like(inputs[n]["hC"]).pin_memory() for n in inputs}]
        last_read = {}  # (buffer set, n) -> event after the last product that read it
        e2e_count = [0]

        def e2e_step():
            sset = e2e_count[0] % 2
            e2e_count[0] += 1
            start = torch.cuda.Event()
            start.record(stream)
            h2d.wait_event(start)
            d2h.wait_event(start)
            copied, ev_c, ev_d = {}, {}, {}
            for j, i in enumerate(order):
                plan, (nm, n, L) = plans[i], cases[i]
                x, d = inputs[n], dins[sset][n]
                if n not in copied:
                    if (sset, n) in last_read:
                        h2d.wait_event(last_read[(sset, n)])  # the step before last is done with it
                    with torch.cuda.stream(h2d):
                        d["A"].copy_(x["hA"], non_blocking=True)
                        d["B"].copy_(x["hB"], non_blocking=True)
                    copied[n] = torch.cuda.Event()
                    copied[n].record(h2d)
                stream.wait_event(copied[n])
                k = j % 2
                if j >= 2:
                    stream.wait_event(ev_d[j - 2])  # that product's result has left this C
                Cd = douts[k][n]
                rbc.matmul(plan, d["A"], d["B"], Cd, leaf=leaf, workspace=ws, decode=args.decode, stream=stream)
                ev_c[j] = torch.cuda.Event()
                ev_c[j].record(stream)
                last_read[(sset, n)] = ev_c[j]
                d2h.wait_event(ev_c[j])
                with torch.cuda.stream(d2h):
                    hout[k][n].copy_(Cd, non_blocking=True)
                ev_d[j] = torch.cuda.Event()
                ev_d[j].record(d2h)
            stream.wait_event(ev_d[len(order) - 1])  # the step ends with its last result on the host
        for _ in range(2):  # warm-up: both buffer sets once (first touch of their memory)
            e2e_step()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        a0.record(stream)
        for k in range(args.steps):
            e2e_step()
            marks[k].record(stream)
        a1.record(stream)
        barrier()
        e_ms = a0.elapsed_time(a1) / args.steps
        step_ms = [round((a0 if k == 0 else marks[k - 1]).elapsed_time(marks[k]), 3) for k in range(args.steps)]
        med = statistics.median(step_ms)
        e2e = {"value": round(world * eff_flops / (e_ms * 1e-3) / 1e12, 3), "unit": "TFLOP/s",
               "ms_per_step": round(e_ms, 3), "step_ms": step_ms,
               "median_step_value": round(world * eff_flops / (med * 1e-3) / 1e12, 3),
               "h2d_bytes_per_step": sum(2 * 4 * n * n for n in sorted({c[1] for c in cases})),
               "d2h_bytes_per_step": sum(4 * n * n for _, n, _ in cases)}

    # Error against our own fp64 classical product (L = 0, fp64 SIMT GEMM), per distinct input.
    errors = []
    if not args.no_errors:
        truths = {}
        one = rbc.Plan(*formula_by_name("strassen"), levels=0)
        for _, n, _ in cases:
            if n in truths:
                continue
            A64 = inputs[n]["A"].double()
            B64 = inputs[n]["B"].double()
            truths[n] = rbc.matmul(one, A64, B64, leaf=rbc.LEAF_F64)
            del A64, B64
        for plan, (nm, n, L) in zip(plans, cases):
            x = inputs[n]
            rbc.matmul(plan, x["A"], x["B"], x["C"], leaf=leaf, workspace=ws, decode=args.decode)
            nr = rbc.norms(x["C"], truths[n]).cpu().numpy()
            errors.append({"formula": nm, "n": n, "L": L, "rel_fro_vs_fp64_ab": float(np.sqrt(nr[0] / nr[1]))})
        torch.cuda.synchronize(dev)
        del truths
        # the hard case: Uniform[0,1] with rows of A and columns of B scaled by 10^U(-3,3)
        from rbc_inputs.matrices import matrix_pair
        hard = {}
        for plan, (nm, n, L) in zip(plans, cases):
            if n not in hard:
                hard.clear()
                torch.cuda.empty_cache()
                Ah, Bh = matrix_pair("hard", n, 500 + n)
                hA = torch.tensor(Ah, dtype=torch.float32, device=dev)
                hB = torch.tensor(Bh, dtype=torch.float32, device=dev)
                hard[n] = (hA, hB, rbc.matmul(one, hA.double(), hB.double(), leaf=rbc.LEAF_F64))
                del Ah, Bh
            hA, hB, ht = hard[n]
            x = inputs[n]
            rbc.matmul(plan, hA, hB, x["C"], leaf=leaf, workspace=ws, decode=args.decode)
            nr = rbc.norms(x["C"], ht).cpu().numpy()
            for e in errors:
                if (e["formula"], e["n"], e["L"]) == (nm, n, L):
                    e["rel_fro_vs_fp64_ab_hard"] = float(np.sqrt(nr[0] / nr[1]))
        hard.clear()
        torch.cuda.synchronize(dev)

    # Our own classical product (L = 0, same leaf mode) on the same inputs, for comparison.
    classical = {}
    if not args.no_errors:
        one = rbc.Plan(*formula_by_name("strassen"), levels=0)
        for _, n, _ in cases:
            if str(n) in classical:
                continue
            x = inputs[n]
            wsz = one.workspace_size(n, rbc.IO_F32, leaf)
            wsc = torch.empty(wsz, dtype=torch.uint8, device=dev)
            for _ in range(2):
                rbc.matmul(one, x["A"], x["B"], x["C"], leaf=leaf, workspace=wsc)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                rbc.matmul(one, x["A"], x["B"], x["C"], leaf=leaf, workspace=wsc)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / 3
            classical[str(n)] = {"ms": round(ms, 3), "eff_tflops": round(2.0 * n**3 / ms / 1e9, 1)}
            del wsc

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(budget_s=15.0, gpu_check=(plans, cases, inputs, ws, leaf))

    # The served form of the metric (p50/p99 latency beside requests/s): a bounded sub-run of
    # the serving workload, after the timed sweep, with the sweep's buffers released.
    served = None
    if args.serve_requests > 0:
        del ws
        inputs.clear()
        torch.cuda.empty_cache()
        specs = serve_specs(args.serve_requests, args.rate)
        served = serve_measure(specs, args.cap_gb, dev, local, baseline_sample=100)
        served["config"] = serve_config(len(specs), args.rate, args.cap_gb)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.leaf == "f32" else f"f32 io, {args.leaf} leaves",
        "data": "synthetic (seeded N(0,1); perturbed Strassen per Section 3.1)",
        "config": {"workload": WORKLOAD, "io": "f32", "leaf": args.leaf, "draws": "per-node",
                   "cases": len(cases), "parallelism": f"replicas x{world}",
                   "l2": "inputs and per-case workspaces larger than L2 (129 MB)"},
        "roofline": roof, "clocks": clk.summary(), "gpu_launches": launches_per_step * args.steps,
        "gpu_launches_per_step": launches_per_step,
        "e2e": e2e, "cpu_baseline": cpu, "classical_same_leaf": classical, "cases": per_case,
        "errors": errors, "served": served,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _oracle_cases(budget_s):
    """Cases for the bounded CPU sample: cheapest first, until the budget is spent."""
    order = [i for i, c in sorted(enumerate(CASES), key=lambda ic: ic[1][1] ** 3 * 0.9 ** ic[1][2])]
    return order


def cpu_baseline(budget_s=15.0, gpu_check=None):
    """The FP64 oracle on the host cores, bounded sample of the workload (cheapest cases
    first until about `budget_s` seconds of CPU work)."""
    import numpy as np

    from oracle import rbc_oracle as o
    from rbc_inputs import formula_by_name

    done, flops, secs, errs = [], 0.0, 0.0, []
    rng_cache = {}
    for i in _oracle_cases(budget_s):
        nm, n, L = CASES[i]
        if secs > budget_s:
            break
        if gpu_check is not None and n not in gpu_check[2]:
            continue
        if n not in rng_cache:
            if gpu_check is not None:
                x = gpu_check[2][n]
                rng_cache[n] = (x["hA"].numpy().astype(np.float64), x["hB"].numpy().astype(np.float64))
            else:
                g = np.random.Generator(np.random.PCG64(1000 + n))
                rng_cache[n] = (g.standard_normal((n, n)).astype(np.float32).astype(np.float64),
                                g.standard_normal((n, n)).astype(np.float32).astype(np.float64))
        A, B = rng_cache[n]
        U, V, W = formula_by_name(nm, seed=7)
        t = time.perf_counter()
        C = o.rbc(A, B, o.Plan(U, V, W, levels=L, seed=2024 + L))
        dt = time.perf_counter() - t
        secs += dt
        flops += 2.0 * n**3
        done.append(f"{nm} n={n} L={L}")
        if gpu_check is not None:
            plans, cases, inputs, ws, leaf = gpu_check
            import torch

            import paper_1905_07439_gb300 as rbc
            j = cases.index((nm, n, L)) if (nm, n, L) in cases else None
            if j is not None:
                x = inputs[n]
                rbc.matmul(plans[j], x["A"], x["B"], x["C"], leaf=leaf, workspace=ws)
                Cg = x["C"].double().cpu().numpy()
                errs.append({"case": f"{nm} n={n} L={L}",
                             "rel_fro_vs_oracle": float(np.linalg.norm(Cg - C) / np.linalg.norm(C)),
                             "normwise_vs_oracle": float(np.linalg.norm(Cg - C) / (np.linalg.norm(A) * np.linalg.norm(B)))})
        del C
    return {"value": round(flops / secs / 1e12, 5), "unit": "TFLOP/s", "cores": os.cpu_count(),
            "kind": "oracle", "sample": "; ".join(done) + f" ({secs:.1f} s, numpy fp64)",
            "parity": errs}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    per = []
    for _ in range(args.warmup):
        cpu_baseline(budget_s=0.0)  # untimed: the same product as a timed step
    t0 = time.perf_counter()
    res = None
    for _ in range(args.steps):
        res = cpu_baseline(budget_s=0.0)  # one product per step: the sweep's cheapest case
        per.append(res["value"])
    dt = time.perf_counter() - t0
    value = statistics.mean(per)
    line = {"metric": METRIC, "value": round(value, 5), "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded N(0,1))", "impl": "reference",
            "config": {"workload": WORKLOAD, "io": "f64 oracle"},
            "cpu_baseline": {"value": round(value, 5), "unit": "TFLOP/s", "cores": res["cores"],
                             "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": round(value, 5), "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def batch_specs(count: int, seed: int = 4):
    """Uneven instances: n log-uniform in [256, 4096] rounded up to a multiple of n0^L * 64,
    formula Strassen / Laderman with equal odds, L uniform in {1, 2}, per-instance seed."""
    import math

    import numpy as np
    g = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(count):
        name = "strassen" if g.random() < 0.5 else "laderman"
        L = int(g.integers(1, 3))
        q = (2 if name == "strassen" else 3) ** L * 64
        n = math.exp(g.uniform(math.log(256), math.log(4096)))
        n = int(math.ceil(n / q) * q)
        specs.append((name, L, n, 7000 + i))
    return specs


def run_batch(args):
    import torch

    import paper_1905_07439_gb300 as rbc
    from rbc_inputs import formula_by_name

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_dist(world, dev)
    leaf_name = args.leaf or "bf16"  # the batched workload runs bf16 leaves
    leaf = rbc.LEAF_NAMES[leaf_name]
    specs = batch_specs(args.instances)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    plans, As, Bs, Cs = [], [], [], []
    for name, L, n, seed in specs:
        plans.append(rbc.Plan(*formula_by_name(name), levels=L, seed=seed))
        As.append(torch.randn((n, n), generator=gen, device=dev))
        Bs.append(torch.randn((n, n), generator=gen, device=dev))
        Cs.append(torch.empty((n, n), device=dev))
    eff_flops = sum(2.0 * n**3 for _, _, n, _ in specs)
    grp = rbc.Group(plans, As, Bs, Cs, leaf)
    ws = torch.empty(grp.workspace_size(), dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream(dev)
    tuning = grp.tune(ws, stream=side)
    for _ in range(max(1, args.warmup)):
        grp.run(ws, stream=side, graph=True)
    torch.cuda.synchronize(dev)
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(side)
        for _ in range(args.steps):
            grp.run(ws, stream=side, graph=True)
        e1.record(side)
        torch.cuda.synchronize(dev)
        barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev) / args.steps
    # one product at a time through rbc_matmul (same leaf mode, staged decode) for comparison
    wmax = max(p.workspace_size(n, rbc.IO_F32, leaf) for p, (_, _, n, _) in zip(plans, specs))
    ws1 = torch.empty(wmax, dtype=torch.uint8, device=dev)
    for p, A, B, Cm in zip(plans, As, Bs, Cs):
        rbc.matmul(p, A, B, Cm, leaf=leaf, workspace=ws1)
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for p, A, B, Cm in zip(plans, As, Bs, Cs):
        rbc.matmul(p, A, B, Cm, leaf=leaf, workspace=ws1)
    s1.record()
    torch.cuda.synchronize(dev)
    ms_seq = s0.elapsed_time(s1)
    # The grouped leaf launch: algorithmic flops 2 R^L m^3 and bytes R^L m^2 (2 bf16 operands
    # read + the fp32 product written) per instance; the model takes, per instance, the larger
    # of its padded MMA work at the bf16 peak and its padded operand/product bytes at the HBM
    # bandwidth (tiles are 128 x 128 or 128 x 256, so m pads to a multiple of 128).
    pk, pk_kind = peaks()
    leaf_flops = leaf_bytes = model_s = 0.0
    es = 4 if leaf_name in ("tf32", "f32") else 2
    for name, L, n, _ in specs:
        U = formula_by_name(name)[0]
        m = n // U.shape[0] ** L
        mp = (m + 127) // 128 * 128
        leaves = U.shape[2] ** L
        leaf_flops += 2.0 * leaves * m**3
        leaf_bytes += leaves * m * m * (2.0 * es + 4.0)
        model_s += max(2.0 * leaves * mp**3 / (pk["bf16_tflops_sustained"] * 1e12),
                       leaves * mp * mp * (2.0 * es + 4.0) / (pk["hbm_gbs"] * 1e9))
    leaf_s = tuning["best_ms"] * 1e-3
    leaf_tf = leaf_flops / leaf_s / 1e12
    leaf_gbs = leaf_bytes / leaf_s / 1e9
    line = {
        "metric": METRIC, "value": round(whole_job_rate(eff_flops, world, ms * 1e-3) / 1e12, 3), "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"f32 io, {leaf_name} leaves",
        "data": "synthetic (seeded N(0,1))",
        "config": {"workload": f"rbc-batch: {len(specs)} uneven instances, n log-uniform [256,4096] rounded to "
                               "n0^L*64, strassen/laderman 50/50, L in {1,2}, per-instance seed; one grouped "
                               "leaf launch, CUDA graph replay, autotuned tiles",
                   "instances": len(specs), "parallelism": f"replicas x{world}"},
        "roofline": {"kernel": "tc_gemm_kernel (grouped, all instances' leaves in one launch)", "bound": "hbm",
                     "achieved": round(leaf_gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": round(leaf_gbs / pk["hbm_gbs"], 4), "traffic": None,
                     "peak_source": f"{pk_kind} HBM copy",
                     "algorithmic_bytes": round(leaf_bytes), "leaf_ms": round(leaf_s * 1e3, 3),
                     "tensor": {"achieved_tflops": round(leaf_tf, 2), "peak": pk["bf16_tflops_sustained"],
                                "frac": round(leaf_tf / pk["bf16_tflops_sustained"], 4)},
                     "model": {"ms_model": round(model_s * 1e3, 3), "frac_of_model": round(model_s / leaf_s, 4),
                               "note": "per instance max(padded MMA flops / bf16 peak, padded operand + "
                                       "product bytes / HBM)"}},
        "tuning": tuning, "one_at_a_time_ms": round(ms_seq, 3),
        "speedup_vs_one_at_a_time": round(ms_seq / ms, 3), "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


PRECISION_LEAVES = ["tf32", "bf16", "f16", "3xbf16", "3xtf32", "bf16x6", "f16x3", "f32"]


def run_precision(args):
    """Precision sweep: randomized Strassen N = 16384, L = 1..3, every leaf mode with fp32
    encode/decode, plus the fp64 leaf mode (fp64 I/O), on N(0,1) and row/column-scaled inputs.
    Each result's error is measured against the fp64 standard product (on the GPU) and, on
    sampled entries, against the oracle's RBC with the same draws."""
    import numpy as np
    import torch

    import paper_1905_07439_gb300 as rbc
    from oracle import rbc_oracle as o
    from rbc_inputs import formula_by_name
    from rbc_inputs.matrices import matrix_pair

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, levels = args.precision_n, (1, 2, 3)
    U, V, W = formula_by_name("strassen")
    plans = {L: rbc.Plan(U, V, W, levels=L, seed=2024 + L) for L in levels}
    one = rbc.Plan(U, V, W, levels=0)
    rng = np.random.default_rng(77)
    rows, cols = rng.integers(0, N, 48), rng.integers(0, N, 48)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    results, tot_flops, tot_ms = [], 0.0, 0.0
    with ClockSampler(local) as clk:
        for dist in ("normal", "hard"):
            An, Bn = matrix_pair(dist, N, 31)
            An = An.astype(np.float32).astype(np.float64)
            Bn = Bn.astype(np.float32).astype(np.float64)
            A64 = torch.tensor(An, device=dev)
            B64 = torch.tensor(Bn, device=dev)
            A, B = A64.float(), B64.float()
            truth = rbc.matmul(one, A64, B64, leaf=rbc.LEAF_F64)
            orc = {L: o.rbc_entries(An, Bn, o.Plan(U, V, W, levels=L, seed=2024 + L), rows, cols) for L in levels}
            ri, ci = torch.as_tensor(rows, device=dev), torch.as_tensor(cols, device=dev)
            truth_s = truth[ri, ci].cpu().numpy()
            C = torch.empty((N, N), dtype=torch.float32, device=dev)
            for leaf_name in PRECISION_LEAVES + ["f64"]:
                for L in levels:
                    leaf = rbc.LEAF_NAMES[leaf_name]
                    f64 = leaf_name == "f64"
                    X, Y = (A64, B64) if f64 else (A, B)
                    Cx = torch.empty((N, N), dtype=torch.float64, device=dev) if f64 else C
                    io = rbc.IO_F64 if f64 else rbc.IO_F32
                    ws = torch.empty(plans[L].workspace_size(N, io, leaf), dtype=torch.uint8, device=dev)
                    run = lambda: rbc.matmul(plans[L], X, Y, Cx, leaf=leaf, workspace=ws)
                    reps = 1 if f64 else (2 if leaf_name == "f32" else 3)
                    if dist == "normal":
                        ms = timed(run, reps)
                    else:
                        run()
                        ms = None
                    nr = rbc.norms(Cx, truth).cpu().numpy()
                    cs = Cx[ri, ci].double().cpu().numpy()
                    row = {"dist": dist, "leaf": leaf_name, "L": L,
                           "rel_fro_vs_fp64_ab": float(np.sqrt(nr[0] / nr[1])),
                           "sampled_rel_vs_oracle_rbc": float(np.linalg.norm(cs - orc[L]) / np.linalg.norm(orc[L])),
                           "sampled_rel_oracle_vs_ab": float(np.linalg.norm(orc[L] - truth_s) / np.linalg.norm(truth_s))}
                    if ms is not None:
                        row["ms"] = round(ms, 3)
                        row["eff_tflops"] = round(2.0 * N**3 / ms / 1e9, 1)
                        if not f64:
                            tot_flops += 2.0 * N**3
                            tot_ms += ms
                    results.append(row)
                    del ws
            del A64, B64, A, B, truth, C
            torch.cuda.empty_cache()
    line = {
        "metric": METRIC, "value": round(world * tot_flops / (tot_ms * 1e-3) / 1e12, 3), "unit": "TFLOP/s",
        "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": round(tot_ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 io; " + ", ".join(PRECISION_LEAVES) + " leaves; f64",
        "data": "synthetic (seeded N(0,1); Uniform[0,1] with rows of A / columns of B scaled by 10^U(-3,3))",
        "config": {"workload": f"rbc-precision: strassen n={N} L=1..3, leaf modes " + "/".join(PRECISION_LEAVES)
                               + " (fp32 encode/decode) and fp64 leaves (fp64 I/O); value = sum 2n^3 / summed time "
                               "over the fp32-I/O products on N(0,1)", "parallelism": f"replicas x{world}"},
        "results": results, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))


# Section 3's two experiment shapes: (figure, formula, io, N, Q, realizations, inputs)
EXP_CONFIGS = [("fig2", "noisy-strassen", "f64", 80, 3, 10_000, "normal"),
               ("fig5", "strassen", "f32", 320, 5, 100, "adv3")]


def _exp_setup(dev):
    import numpy as np

    import paper_1905_07439_gb300 as rbc
    from paper_1905_07439_gb300 import experiments as ex
    from rbc_inputs import formula_by_name
    from rbc_inputs.matrices import matrix_pair

    import torch
    out = []
    for fig, fname, io, N, Q, K, dist in EXP_CONFIGS:
        U, V, W = formula_by_name(fname, seed=0)
        A, B = matrix_pair(dist, N, 1000)
        run = ex.Runner(U, V, W, A, B, io, device=str(dev))
        plan = run.plan(Q, rbc.RAND_FULL, rbc.DRAW_PER_LEVEL)
        seeds = np.arange(K, dtype=np.uint64) + (Q << 24)
        one = int(rbc.lib().rbc_realizations_workspace_size(plan.handle, N, run.io, run.leaf, 1))
        batch = max(1, min(K, (8 << 30) // one))
        ws = torch.empty(int(rbc.lib().rbc_realizations_workspace_size(plan.handle, N, run.io, run.leaf, batch)),
                         dtype=torch.uint8, device=dev)
        Cs = torch.empty((K, N, N), dtype=run.dtype, device=dev)
        err = torch.empty(K, dtype=torch.float64, device=dev)
        work = torch.empty(int(rbc.lib().rbc_realization_errors_work_size(K, N)), dtype=torch.uint8, device=dev)
        mode = rbc.ERR_AVERAGE if fig == "fig2" else rbc.ERR_EACH
        out.append(dict(fig=fig, fname=fname, io=io, N=N, Q=Q, K=K, dist=dist, run=run, plan=plan, seeds=seeds,
                        ws=ws, Cs=Cs, err=err, work=work, mode=mode, A=A, B=B, batch=batch))
    return out


def _exp_step(cfgs, stream, host=None):
    """One step: every configuration's realizations and their error reduction.  With `host`,
    A and B are copied from pinned host memory first and the errors back after."""
    import paper_1905_07439_gb300 as rbc
    for i, c in enumerate(cfgs):
        r = c["run"]
        if host is not None:
            r.A.copy_(host[i]["A"], non_blocking=True)
            r.B.copy_(host[i]["B"], non_blocking=True)
        rbc.realizations(c["plan"], c["seeds"], r.A, r.B, c["Cs"], leaf=r.leaf, workspace=c["ws"], stream=stream)
        rbc.realization_errors(c["Cs"], r.ref, c["mode"], stream=stream, work=c["work"], out=c["err"])
        if host is not None:
            host[i]["err"].copy_(c["err"], non_blocking=True)


def exp_cpu_baseline(cfg, budget_s=12.0):
    """The oracle on the host cores: realizations of the Figure 2 shape (perturbed Strassen,
    N = 80, Q = 3, fp64) and their error, until about `budget_s` seconds."""
    import numpy as np

    from oracle import rbc_oracle as o
    from rbc_inputs import formula_by_name
    U, V, W = formula_by_name(cfg["fname"], seed=0)
    A, B = cfg["A"], cfg["B"]
    AB = A @ B
    t0 = time.perf_counter()
    n, acc, errs = 0, np.zeros_like(AB), []
    while time.perf_counter() - t0 < budget_s:
        C = o.rbc(A, B, o.Plan(U, V, W, levels=cfg["Q"], seed=int(cfg["seeds"][n]), mode=o.RAND_FULL,
                              scope=o.DRAW_PER_LEVEL))
        acc += C
        n += 1
        errs.append(float(np.linalg.norm(acc / n - AB) / np.linalg.norm(AB)))
    dt = time.perf_counter() - t0
    return {"value": round(n / dt, 3), "unit": "realizations/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} realizations of {cfg['fname']} N={cfg['N']} Q={cfg['Q']} fp64 per-level draws "
                      f"with their error of average ({dt:.1f} s, numpy fp64)",
            "errors": errs}


def run_experiments(args):
    """Section 3 experiment shapes: realizations per second (all realizations of both
    configurations, with their error reductions, per step)."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfgs = _exp_setup(dev)
    stream = torch.cuda.Stream(dev)
    for _ in range(max(3, args.warmup)):
        _exp_step(cfgs, stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            _exp_step(cfgs, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    per_step = sum(c["K"] for c in cfgs)
    # per configuration, one step each
    parts = []
    for c in cfgs:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _exp_step([c], stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        e = c["err"].cpu().numpy()
        parts.append({"figure": c["fig"], "formula": c["fname"], "io": c["io"], "N": c["N"], "Q": c["Q"],
                      "realizations": c["K"], "inputs": c["dist"], "batch": c["batch"],
                      "ms": round(a.elapsed_time(b), 3),
                      "realizations_per_s": round(c["K"] / (a.elapsed_time(b) * 1e-3), 1),
                      "error": ({"first": float(e[0]), "last": float(e[-1])} if c["mode"] == 1 else
                                {"median": float(np.median(e)), "min": float(e.min()), "max": float(e.max())})})
    # end to end: inputs from pinned host memory, errors back to the host, every step
    host = [{"A": c["run"].A.cpu().pin_memory(), "B": c["run"].B.cpu().pin_memory(),
             "err": torch.empty(c["K"], dtype=torch.float64).pin_memory()} for c in cfgs]
    _exp_step(cfgs, stream, host)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _exp_step(cfgs, stream, host)
    stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = sum(h["A"].numel() * h["A"].element_size() * 2 for h in host)
    d2h = sum(h["err"].numel() * 8 for h in host)
    line = {
        "metric": "Section 3 realizations/s (realizations + error reductions)", "value":
            round(world * per_step / (ms * 1e-3), 1), "unit": "realizations/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (fig2 shape), f32 (fig5 shape)",
        "data": "synthetic (seeded N(0,1); type-3 adversarial)",
        "config": {"workload": "rbc-experiments: 10^4 realizations of perturbed Strassen N=80 Q=3 fp64 with the "
                               "error of their running average + 100 realizations of Strassen N=320 Q=5 fp32 "
                               "on adversarial type-3 inputs with per-realization errors; per-level draws",
                   "parallelism": f"replicas x{world}", "l2": "outputs of each step (0.6 GB) exceed L2"},
        "parts": parts,
        "e2e": {"value": round(world * per_step / e2e_s, 1), "unit": "realizations/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = exp_cpu_baseline(cfgs[0])
        ce = line["cpu_baseline"].pop("errors")
        g = cfgs[0]["err"].cpu().numpy()[: len(ce)]
        line["cpu_baseline"]["parity_error_of_average_max_rel_diff"] = float(np.max(np.abs(g - ce) / np.abs(ce)))
    if rank == 0:
        print(json.dumps(line))


SERVE_LEAF = {"fp32": "f16x3", "bf16-leaf": "bf16", "3xbf16-leaf": "3xbf16"}


def serve_specs(count: int, rate: float, seed: int = 5):
    """Requests: exponential inter-arrival gaps (rate per second), n log-uniform in
    [128, 8192], formula uniform over {strassen, laderman, noisy-strassen}, L uniform in
    {1, 2, 3} but at most max(1, floor(log_n0(n / 64))) so that small n stay small, n rounded
    up to a multiple of n0^L * 64, dtype uniform over {fp32, bf16-leaf, 3xbf16-leaf}."""
    import math

    import numpy as np
    g = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += g.exponential(1.0 / rate)
        name = ["strassen", "laderman", "noisy-strassen"][int(g.integers(0, 3))]
        n0 = 3 if name == "laderman" else 2
        n = math.exp(g.uniform(math.log(128), math.log(8192)))
        L = int(g.integers(1, 4))
        L = max(1, min(L, int(math.floor(math.log(max(n, 64) / 64.0) / math.log(n0) + 1e-9))))
        q = n0**L * 64
        n = int(math.ceil(n / q) * q)
        dt = ["fp32", "bf16-leaf", "3xbf16-leaf"][int(g.integers(0, 3))]
        out.append({"t": t, "formula": name, "n": n, "L": L, "dtype": dt, "seed": 50000 + i})
    return out


def serve_measure(specs, cap_gb, dev, local, baseline_sample=300):
    """Serve `specs` through the queue: a closed-loop warm-up, the paced run (Poisson arrival
    times) for latency, a closed-loop run (every request available at once) for capacity, and
    one-at-a-time runs on a sample of the requests (fp32 CUDA-core leaves; the served leaf
    modes).  Returns a dict of the measured figures."""
    import time as _t

    import numpy as np
    import torch

    import paper_1905_07439_gb300 as rbc
    from rbc_inputs import formula_by_name

    nmax = max(r["n"] for r in specs)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(17)
    A = torch.randn((nmax, nmax), generator=gen, device=dev)   # request i uses the leading n x n block
    B = torch.randn((nmax, nmax), generator=gen, device=dev)
    forms = {nm: formula_by_name(nm, seed=7) for nm in ("strassen", "laderman", "noisy-strassen")}
    plans = [rbc.Plan(*forms[r["formula"]], levels=r["L"], seed=r["seed"]) for r in specs]
    slots = [torch.empty((nmax, nmax), device=dev) for _ in range(40)]
    free = list(range(len(slots)))

    def run_queue(paced: bool):
        q = rbc.Queue(device=local, workspace_cap=int(cap_gb * (1 << 30)), streams=16)
        live = {}  # ticket -> (index, slot)
        done_t = [0.0] * len(specs)
        t0 = _t.perf_counter()
        i = 0

        def collect():
            for t in list(live):
                if q.poll(t):
                    idx, sl = live.pop(t)
                    done_t[idx] = _t.perf_counter() - t0
                    free.append(sl)

        while i < len(specs) or live:
            now = _t.perf_counter() - t0
            while i < len(specs) and (not paced or specs[i]["t"] <= now) and free:
                r = specs[i]
                sl = free.pop()
                n = r["n"]
                Cv = slots[sl][:n, :n]
                tk = q.submit(plans[i], A[:n, :n], B[:n, :n], Cv, rbc.LEAF_NAMES[SERVE_LEAF[r["dtype"]]])
                live[tk] = (i, sl)
                i += 1
            collect()
        stats = q.stats()
        q.close()
        return done_t, stats

    run_queue(False)                       # warm-up (kernels loaded, pools touched)
    done_t, stats = run_queue(True)        # Poisson arrivals
    arrive = np.array([r["t"] for r in specs])
    lat = (np.array(done_t) - arrive) * 1e3
    span = max(done_t) - arrive[0]
    closed_t, _ = run_queue(False)         # all requests available at once: capacity
    cap_rps = len(specs) / max(closed_t)
    # one at a time, fp32 leaves on the CUDA cores, on a sample of the requests
    sample = list(range(0, len(specs), max(1, len(specs) // baseline_sample)))
    ws = torch.empty(max(plans[i].workspace_size(specs[i]["n"], rbc.IO_F32, rbc.LEAF_F32) for i in sample),
                     dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    t1 = _t.perf_counter()
    for i in sample:
        n = specs[i]["n"]
        rbc.matmul(plans[i], A[:n, :n], B[:n, :n], slots[0][:n, :n], leaf=rbc.LEAF_F32, workspace=ws)
        torch.cuda.synchronize(dev)
    base_rps = len(sample) / (_t.perf_counter() - t1)
    # one at a time with the served leaf modes (isolates the effect of the queue)
    t1 = _t.perf_counter()
    for i in sample:
        n = specs[i]["n"]
        lf = rbc.LEAF_NAMES[SERVE_LEAF[specs[i]["dtype"]]]
        wsz = plans[i].workspace_size(n, rbc.IO_F32, lf)
        if wsz > ws.numel():
            ws = torch.empty(wsz, dtype=torch.uint8, device=dev)
        rbc.matmul(plans[i], A[:n, :n], B[:n, :n], slots[0][:n, :n], leaf=lf, workspace=ws)
        torch.cuda.synchronize(dev)
    same_rps = len(sample) / (_t.perf_counter() - t1)
    del ws, slots, A, B
    torch.cuda.empty_cache()
    eff = sum(2.0 * r["n"] ** 3 for r in specs)
    return {
        "requests": len(specs),
        "requests_per_s": round(len(specs) / span, 2), "span_ms": round(span * 1e3, 1),
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3),
                       "max": round(float(lat.max()), 3)},
        "effective_tflops": round(eff / span / 1e12, 2),
        "capacity_requests_per_s": round(cap_rps, 1),
        "one_at_a_time_fp32_requests_per_s": round(base_rps, 1),
        "one_at_a_time_same_leaves_requests_per_s": round(same_rps, 1),
        "capacity_vs_one_at_a_time_fp32": round(cap_rps / base_rps, 2),
        "capacity_vs_one_at_a_time_same_leaves": round(cap_rps / same_rps, 2),
        "queue": {k: stats[k] for k in ("admitted", "completed", "workspace_peak", "peak_running")},
    }


def serve_config(n_requests, rate, cap_gb):
    return (f"rbc-serve: {n_requests} requests, Poisson {rate:g}/s, n log-uniform [128,8192], "
            "strassen/laderman/noisy-strassen, L in {1,2,3} (clamped for small n), dtype in {fp32, bf16-leaf, "
            f"3xbf16-leaf}} (fp32 served by f16x3 leaves), workspace admission cap {cap_gb:g} GB, 16 streams")


def run_serve(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = serve_specs(args.requests, args.rate)
    with ClockSampler(local) as clk:
        m = serve_measure(specs, args.cap_gb, dev, local)
    line = {
        "metric": METRIC, "value": m["requests_per_s"], "unit": "requests/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": m["span_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 io; leaves per request (fp32 -> f16x3, bf16, 3xbf16)",
        "data": "synthetic (seeded N(0,1); Poisson arrivals)",
        "config": {"workload": serve_config(len(specs), args.rate, args.cap_gb), "parallelism": "replicas x1"},
        "clocks": clk.summary(),
    }
    line.update({k: v for k, v in m.items() if k not in ("requests_per_s", "span_ms")})
    if rank == 0:
        print(json.dumps(line))


def run_peaks(args):
    """cuBLAS GEMM throughput per dtype on this GPU (torch.matmul of n x n operands, n^3
    multiply-adds): a measured context for the leaf modes whose roofline peaks are derived
    (fp32 FMA from unit counts and clock, tf32 and f16 from the measured bf16 peak and the
    nominal rate ratios).  Each dtype: a burst of about 0.3 s, then a loop of about 3 s
    (sustained).  One JSON line; not a step of the method."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    res = {}
    cases = [("f32", torch.float32, False, 8192), ("tf32", torch.float32, True, 8192),
             ("f16", torch.float16, False, 8192), ("bf16", torch.bfloat16, False, 8192),
             ("f64", torch.float64, False, 4096)]
    prev = torch.backends.cuda.matmul.allow_tf32
    with ClockSampler(0) as clk:
        for name, dtype, tf32, n in cases:
            torch.backends.cuda.matmul.allow_tf32 = tf32
            g = torch.Generator(device=dev)
            g.manual_seed(n)
            a = torch.randn((n, n), generator=g, device=dev, dtype=torch.float32).to(dtype)
            b = torch.randn((n, n), generator=g, device=dev, dtype=torch.float32).to(dtype)
            c = torch.empty((n, n), device=dev, dtype=dtype)
            for _ in range(3):
                torch.matmul(a, b, out=c)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize(dev)
            one = max(e0.elapsed_time(e1), 1e-3)
            out = {}
            for label, secs in (("burst", 0.3), ("sustained", 3.0)):
                reps = max(3, int(secs * 1e3 / one))
                e0.record()
                for _ in range(reps):
                    torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize(dev)
                out[label] = round(2.0 * n**3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12, 1)
            out["n"] = n
            res[name] = out
            del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = prev
    print(json.dumps({"metric": "cuBLAS GEMM TFLOP/s per dtype (torch.matmul)", "unit": "TFLOP/s", "n_gpus": 1,
                      "peaks": res, "derived_fp32_fma_tflops": round(FP32_PEAK_TFLOPS, 1),
                      "nominal_tf32_per_bf16": round(TF32_PER_BF16, 4), "clocks": clk.summary()}))


def main():
    args = parse()
    if args.workload == "peaks":
        run_peaks(args)
        return
    if args.workload == "serve" and args.impl != "reference":
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "experiments":
        run_experiments(args)
    elif args.workload == "precision":
        run_precision(args)
    else:
        args.leaf = args.leaf or "f16x3"
        run_ours(args)


if __name__ == "__main__":
    main()
