#!/usr/bin/env python
"""Benchmark: batched NTT polynomial products over Z/pZ on GB300.

Workload (one step): 256 independent products mod p = 3*2^30+1 of two
length-2^15 operands with residues uniform in [0, p) (seeded), through
size-2^16 transforms: two forward transforms, pointwise product, inverse
transform (Section 5.2 of van der Hoeven-Lecerf-Quintin).  The fused
schedule is the measured value; the one-launch-per-radix-2-stage schedule
("plain") is measured beside it on the same inputs.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
(schoolbook, OpenMP over coefficients) on a bounded sample of the same
workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched NTT polymul products/s and GB/s (% of HBM peak), batched vs plain"
UNIT = "products/s"
WORKLOAD = {"workload": "256 products mod 3*2^30+1, operands 2^15 uint32, size-2^16 NTTs",
            "p": 3221225473, "batch": 256, "na": 1 << 15, "nb": 1 << 15, "log2n": 16,
            "word": "u32"}
SM_COUNT = 152
INT_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
L2_BYTES = 129 * 1024 * 1024

# 32-bit-instruction counts of the word policy's arithmetic (Mont32, any odd
# p < 2^32): modular add, subtract, fixed-multiplicand product, general
# (Montgomery) product.
OPS32 = {"add": 3, "sub": 3, "mulw": 6, "mulg": 7}


# 32-bit-instruction counts of the 64-bit word policy's forms (Shoup64L,
# p < 2^62, lazy residues in [0, 2p)), from their decomposition into 32-bit
# instructions: a 64-bit add or subtract is 2 (low word with carry, high
# word); the sign test of a 64-bit difference 1 (its high word); a 64-bit
# select 2; the low 64 bits of a 64 x 64 product 3 (one wide multiply and
# two multiply-adds into the high word); the high 64 bits 6 (the high word
# of the low partial product, three wide multiply-adds with 64-bit addends,
# one 64-bit add).
#   add      red2(x + y): add 2, then t = s - 2p 2, sign of t 1, select 2: 7
#   sub      red2(x + 2p - y) (one three-input add per word): 7
#   sub_lazy x + 2p - y, feeding a twiddle product: 2
#   mulw     Function 8: high product 6, two low products 6, subtract 2: 14
#   mulg     Montgomery: 128-bit product 8, q = lo p' 3, high product 6,
#            subtract 2, sign 1, corrected select 4: 24
#   canon    [0, 2p) -> [0, p): subtract 2, sign 1, select 2: 5
OPS64 = {"add": 7, "sub": 7, "sub_lazy": 2, "mulw": 14, "mulg": 24, "canon": 5}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--plain-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", default=None, choices=["fused"],
                    help="run only the fused timed steps (for profiler captures)")
    ap.add_argument("--workload", default="polymul",
                    choices=["polymul", "serve", "modmul", "suite", "fp64", "tft", "single_product",
                             "transform_2e24_u64", "products_2e12_u64", "products_2e16_u64", "uneven_10000",
                             "serving"],
                    help="polymul: the batched product (headline); serve: the Poisson "
                         "stream of integer products through the serving loop; modmul: "
                         "throughput of each reduction; suite: the other workloads and the "
                         "matrix products, one context line each; fp64: transforms over "
                         "doubles (Function 16) against the integer ones at Table 12's sizes; "
                         "tft: 2^16-point products by output length class (truncated "
                         "transforms against the full length); single_product, "
                         "transform_2e24_u64, products_2e12_u64, products_2e16_u64, uneven_10000, "
                         "serving: one of "
                         "the workloads the default line carries, alone (profiler captures)")
    ap.add_argument("--requests", type=int, default=48, help="serve: requests per stream")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shape (profiler captures)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other workloads (single product, 64-bit transform and products, "
                         "uneven batch, serving) that the default N=1 line carries")
    return ap.parse_args()


# ---------------------------------------------------------------- algorithmic counts

def dif_counts(L: int):
    """(nontrivial, trivial) radix-2 butterflies of a length-L transform."""
    k = L.bit_length() - 1
    total = (L // 2) * k
    trivial = L - 1
    return total - trivial, trivial


def fused_kernel_ops(log2n: int, na: int, nb: int, batch: int, tile_max_log: int):
    """Algorithmic 32-bit integer operations per launch of each fused kernel."""
    o = OPS32
    N = 1 << log2n
    nc = na + nb - 1

    def transform_ops(L):
        nt, tr = dif_counts(L)
        return nt * (o["add"] + o["sub"] + o["mulw"]) + tr * (o["add"] + o["sub"])

    if log2n <= tile_max_log:
        per = 3 * transform_ops(N) + N * o["mulg"] + nc * o["mulw"]
        return {"k_tile_polymul": per * batch}
    k2 = log2n // 2
    k1 = log2n - k2
    n1, n2 = 1 << k1, 1 << k2
    step2 = (N - n1 - n2 + 1) * o["mulw"]
    col_fwd = 2 * (n1 * transform_ops(n2) + step2)
    row = 3 * n2 * transform_ops(n1) + N * o["mulg"]
    col_inv = step2 + n1 * transform_ops(n2) + nc * o["mulw"]
    ops = {"k_col_fwd": col_fwd * batch, "k_row_polymul": row * batch, "k_col_inv": col_inv * batch}
    # the direct 2^16-point kernels do the same work in the same three launches
    ops.update({name + "_d": v for name, v in ops.items()})
    ops["k_col_fwd_tma"] = ops["k_col_fwd"]            # the same pass with its input tile by TMA
    return ops


def transform_ops64(L: int) -> int:
    """64-bit-word transform of length L on the radix-2 network: every
    butterfly has a sum; differences that feed a twiddle product are lazy."""
    o = OPS64
    nt, tr = dif_counts(L)
    return nt * (o["add"] + o["sub_lazy"] + o["mulw"]) + tr * (o["add"] + o["sub"])


def ntt64_ops(L: int, batch: int = 1) -> int:
    """One forward (or inverse, its scaling folded into a twiddle table)
    transform per vector, canonical output words."""
    return batch * (transform_ops64(L) + L * OPS64["canon"])


def polymul64_ops(log2n: int, na: int, nb: int, batch: int) -> int:
    """Products with 64-bit words: three transforms, n pointwise products,
    the final scaling and canonical store of every output word."""
    o = OPS64
    n, nc = 1 << log2n, na + nb - 1
    return batch * (3 * transform_ops64(n) + n * o["mulg"] + nc * (o["mulw"] + o["canon"]))


def alg_bytes(na, nb, batch, wb):
    return batch * (na + nb + (na + nb - 1)) * wb


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, flags in rows:
            for nm, fl in zip(names, flags[1:]):
                if fl.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------- distributed

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_value(products_per_rank: int, world: int, max_seconds: float) -> float:
    """Weak scaling: every rank runs the full workload; whole-job rate is the
    units all ranks processed over the slowest rank's time."""
    return products_per_rank * world / max_seconds


# ---------------------------------------------------------------- inputs

def make_inputs():
    from paper_1407_3383_gb300 import workloads as W
    p, a, b = W.config1()
    return p, a, b


KERNEL_SOURCES = ["engine.cuh", "modarith.cuh", "tft.cuh", "direct.cuh", "subvec.cuh", "ntt_kernels.cuh",
                  "ntt_u32.cu", "ntt_u64.cu"]


def source_hash() -> str:
    """Hash of the sources that define the transform/product kernels, with
    line comments removed (a comment edit does not change a kernel)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1407_3383_gb300", "csrc")
    for name in KERNEL_SOURCES:
        h.update(name.encode())
        text = open(os.path.join(csrc, name), encoding="utf-8").read()
        code = "\n".join(re.sub(r"//.*$", "", line).rstrip() for line in text.splitlines())
        h.update(code.encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        data = json.load(open(path))
    except Exception:
        return None
    ent = data.get(kernel)
    if not ent or ent.get("source_hash") != source_hash():
        return None
    return ent.get("bytes_per_launch")


# ---------------------------------------------------------------- CPU oracle timing

def time_oracle(p, a, b, target_s: float = 12.0):
    """The oracle's schoolbook product on a bounded sample of the workload's
    products, on this host's cores.  Returns (products/s, cores, sample text)."""
    import numpy as np
    import oracle as O
    cores = O.num_threads()
    # calibrate on one product, then size the sample to about target_s
    t0 = time.perf_counter()
    O.polymul_batch(p, a[:1].astype(np.uint64), b[:1].astype(np.uint64))
    one = time.perf_counter() - t0
    count = int(max(1, min(a.shape[0], target_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    prods = O.polymul_batch(p, a[:count].astype(np.uint64), b[:count].astype(np.uint64))
    dt = time.perf_counter() - t0
    sample = (f"{count} of the {a.shape[0]} products (schoolbook, all {a.shape[1] + b.shape[1] - 1} "
              f"coefficients each), {dt:.1f} s wall on {cores} threads")
    return count / dt, cores, sample, prods


def time_cpu_ntt(p, a, b, target_s: float = 3.0):
    """The textbook radix-2 transform product (oracle/cpu_ntt.c, the
    O(n log n) CPU reference) on a bounded sample of the workload's products,
    on this host's cores.  Returns (products/s, cores, sample text, products)."""
    import numpy as np
    import oracle as O
    cores = O.num_threads()
    k = min(a.shape[0], cores)
    t0 = time.perf_counter()
    O.ntt_polymul_batch(p, a[:k].astype(np.uint64), b[:k].astype(np.uint64))
    one_round = time.perf_counter() - t0
    count = int(max(k, min(a.shape[0], k * target_s / max(one_round, 1e-6))))
    t0 = time.perf_counter()
    prods = O.ntt_polymul_batch(p, a[:count].astype(np.uint64), b[:count].astype(np.uint64))
    dt = time.perf_counter() - t0
    sample = (f"{count} of the {a.shape[0]} products (textbook radix-2 transforms of "
              f"{1 << (a.shape[1] + b.shape[1] - 2).bit_length()} points, u128 remainders), "
              f"{dt:.2f} s wall on {cores} threads")
    return count / dt, cores, sample, prods


def run_reference(args, world, rank, target_s: float = 120.0):
    """The oracle (schoolbook) as the reference arm, on this host's cores.
    Each step is a bounded sample of the workload sized so that warm-up and
    timed steps together take about target_s: whole products (up to 4) when
    the per-step budget allows, otherwise the first m coefficients of one
    product, which the schoolbook gets exactly from the length-m prefixes of
    its operands with m^2 multiply-adds.  The rate counts product-equivalents:
    multiply-adds done / (na * nb) per second, the schoolbook's cost being
    exactly its number of multiply-adds."""
    if rank != 0:
        return
    p, a, b = make_inputs()
    import numpy as np
    import oracle as O
    cores = O.num_threads()
    batch, na = a.shape
    nb = b.shape[1]
    full = na * nb
    # calibrate the oracle's multiply-add rate on one 4096-word prefix product
    c0 = min(4096, na, nb)
    t0 = time.perf_counter()
    O.polymul_batch(p, a[:1, :c0].astype(np.uint64), b[:1, :c0].astype(np.uint64))
    rate = c0 * c0 / max(time.perf_counter() - t0, 1e-6)
    budget = target_s / max(1, args.steps + max(0, args.warmup))
    if rate * budget >= full:
        per_step = int(min(4, rate * budget // full))
        m = None
        sample = f"{per_step} of {batch} whole products per step"
    else:
        per_step = 1
        m = int(min(na, nb, max(256, (rate * budget) ** 0.5)))
        sample = (f"the first {m} coefficients of one product per step (its operands' length-{m} prefixes, "
                  f"{m * m} of the {full} multiply-adds)")

    def step(s):
        i0 = (s * per_step) % batch
        if m is None:
            aa = a[i0:i0 + per_step].astype(np.uint64)
            bb = b[i0:i0 + per_step].astype(np.uint64)
            O.polymul_batch(p, aa, bb)
            return per_step * full
        O.polymul_batch(p, a[i0:i0 + 1, :m].astype(np.uint64), b[i0:i0 + 1, :m].astype(np.uint64))
        return m * m

    for s in range(max(0, args.warmup)):
        step(s)
    times, work = [], 0
    for s in range(args.steps):
        t0 = time.perf_counter()
        work += step(s)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = work / full / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(WORKLOAD, timed_sample=sample),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample}, schoolbook, {args.steps} steps; rate in whole-product "
                                   f"equivalents (multiply-adds / {full})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- native timing

def timed_steps(step, flush, steps, stream):
    """Per-step device time with CUDA events on the launching stream; the L2
    flush between steps is outside the events."""
    import torch
    evs = []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def profile_window(G, step, flush, steps):
    """Run `steps` steps with launch profiling on; returns per-kernel lists of ms."""
    import ctypes
    import torch
    lib = G.lib()
    lib.ntt_profile_begin.restype = ctypes.c_int
    lib.ntt_profile_end.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int)]
    per = {}
    launches = 0
    for _ in range(steps):
        flush()
        torch.cuda.synchronize()
        lib.ntt_profile_begin()
        step()
        cap = 256
        ms = (ctypes.c_float * cap)()
        names = (ctypes.c_char_p * cap)()
        cnt = ctypes.c_int()
        rc = lib.ntt_profile_end(cap, ms, names, ctypes.byref(cnt))
        assert rc == 0
        launches += cnt.value
        for i in range(min(cnt.value, cap)):
            per.setdefault(names[i].decode(), []).append(ms[i])
    return per, launches / max(1, steps)


def measured_hbm_gbs() -> float:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)).get("hbm_gbs", 6800.0)
    return 6800.0


def measure_probes(G, stream) -> dict:
    """Integer operations/s of each probe kind (G op/s)."""
    out = {}
    for kind, name in [(G.NTT_PROBE_IMAD, "imad"), (G.NTT_PROBE_ALU, "iadd_lop"),
                       (G.NTT_PROBE_MIXED, "mixed"), (G.NTT_PROBE_WIDE, "imad_wide")]:
        try:
            out[name + "_gops"] = round(G.ntt_int_probe(kind, SM_COUNT * 8, 256, 4096, stream) / 1e9, 1)
        except Exception:
            pass
    return out


def alu_roofline(ops: float, seconds: float, peak_gops: float) -> dict:
    ach = ops / seconds / 1e9
    return {"bound": "alu", "achieved": ach, "peak": peak_gops, "unit": "Gop/s", "frac": ach / peak_gops,
            "alg_gop": ops / 1e9}


def hbm_roofline(nbytes: float, seconds: float, hbm: float) -> dict:
    ach = nbytes / seconds / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "alg_bytes": nbytes}


def run_workloads(G, dev, stream, flush, peak_gops: float, hbm: float, only=None) -> dict:
    """The workloads other than the headline, each with its own config and
    rooflines: one 4096-point product (latency), one 2^24-point transform and
    1024 products of 2^12 words mod a 62-bit prime, the 10,000-product uneven
    batch against one library call per product, and a closed-loop serving
    run (`only` selects one of them by name).  Device time with CUDA events
    on the launching stream, L2 flushed before each timed repetition; every
    result is checked (against the oracle, a round trip, or another
    schedule)."""
    import statistics as _st
    import torch

    def med(step, reps, warm=3):
        for _ in range(warm):
            step()
        torch.cuda.synchronize()
        return _st.median(timed_steps(step, flush, reps, stream))

    parts = {
        "single_product": lambda: wl_single_product(G, dev, stream, med, flush, peak_gops),
        "transform_2e24_u64": lambda: wl_transform_2e24(G, dev, stream, med, peak_gops, hbm),
        "products_2e12_u64": lambda: wl_products_2e12(G, dev, stream, med, peak_gops, hbm),
        "products_2e16_u64": lambda: wl_products_2e16(G, dev, stream, med, peak_gops, hbm),
        "uneven_10000": lambda: uneven_batch(G, dev, stream, flush, med),
        "serving": lambda: serve_closed_loop(G, requests=48),
    }
    res = {}
    for name, fn in parts.items():
        if only and name != only:
            continue
        t0 = time.perf_counter()
        res[name] = fn()
        res[name]["wall_s"] = time.perf_counter() - t0
    return res


def wl_single_product(G, dev, stream, med, flush, peak_gops: float) -> dict:
    """One product of two length-2048 operands mod 998244353 (4096 points):
    latency per call with L2 flushed (CUDA events around the call, so the
    host's launch path is inside), the kernel's own device time (events the
    library records around it), and the graph-replayed rate."""
    import numpy as np
    import torch
    import oracle as O
    from paper_1407_3383_gb300 import workloads as W
    p, a, b = W.config0()
    with G.Plan(p, 12) as plan:
        da = torch.from_numpy(a.astype(np.uint32)).to(dev)
        db = torch.from_numpy(b.astype(np.uint32)).to(dev)
        dc = torch.empty(4095, dtype=torch.uint32, device=dev)
        ms = med(lambda: G.polymul_mod_p(plan, da, 2048, db, 2048, dc, stream=stream), 50)
        ok = bool((dc.cpu().numpy().astype(np.uint64) == O.polymul(p, a, b)).all())
        side = torch.cuda.Stream(device=dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            G.polymul_mod_p(plan, da, 2048, db, 2048, dc, stream=side)
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=side):
                for _ in range(100):
                    G.polymul_mod_p(plan, da, 2048, db, 2048, dc, stream=side)
        gms = med(lambda: graph.replay(), 10)
        per, _ = profile_window(G, lambda: G.polymul_mod_p(plan, da, 2048, db, 2048, dc, stream=stream), flush, 20)
        kern = {k: 1e3 * statistics.median(v) for k, v in per.items()}
        ops = fused_kernel_ops(12, 2048, 2048, 1, plan.info.tile_max_log)["k_tile_polymul"]
        return {
            "config": {"workload": "1 product 2048 x 2048 mod 998244353 (119*2^23+1), 4096-point NTTs, u32",
                       "l2": "flushed before each call"},
            "metric": "latency per product", "value": 1e3 * ms, "unit": "us", "higher_is_better": False,
            "graph_replayed_products_per_s": 100 / (gms * 1e-3), "kernel_us": kern,
            "roofline": dict(alu_roofline(ops, ms * 1e-3, peak_gops), bound="latency",
                             note="one 8-CTA thread-block cluster (8 of 152 SMs)"),
            "matches_oracle": ok}


def wl_transform_2e24(G, dev, stream, med, peak_gops: float, hbm: float) -> dict:
    """One 2^24-point transform mod P1, forward then inverse."""
    import torch
    from paper_1407_3383_gb300 import workloads as W
    p, x = W.config2_transform()
    with G.Plan(p, 24) as plan:
        dx = torch.from_numpy(x).to(dev)
        fms = med(lambda: G.ntt_forward(plan, dx, 1, stream=stream), 10)
        ims = med(lambda: G.ntt_inverse(plan, dx, 1, stream=stream), 10)
        ok = bool((dx.cpu().numpy() == x).all())          # equal numbers of forwards and inverses
        n = 1 << 24
        ops = 2 * ntt64_ops(n)
        nbytes = 2 * 2 * n * 8                              # each transform reads and writes n words once
        sec = (fms + ims) * 1e-3
        return {
            "config": {"workload": "one 2^24-point transform mod P1 = 2097222*2^40+1 (62-bit), forward then "
                                   "inverse, u64", "l2": "flushed before each transform"},
            "metric": "forward + inverse time", "value": fms + ims, "unit": "ms", "higher_is_better": False,
            "forward_ms": fms, "inverse_ms": ims,
            "roofline": alu_roofline(ops, sec, peak_gops), "hbm": hbm_roofline(nbytes, sec, hbm),
            "round_trip_exact": ok}


def wl_products_2e12(G, dev, stream, med, peak_gops: float, hbm: float) -> dict:
    """1024 products of length 2^12 mod P1 (2^13 points, u64)."""
    import torch
    import oracle as O
    from paper_1407_3383_gb300 import workloads as W
    p, a, b = W.config2_products()
    with G.Plan(p, 13) as plan:
        da = torch.from_numpy(a.reshape(-1)).to(dev)
        db = torch.from_numpy(b.reshape(-1)).to(dev)
        dc = torch.empty(1024 * 8191, dtype=torch.uint64, device=dev)
        ms = med(lambda: G.polymul_mod_p_batch(plan, da, 4096, db, 4096, 1024, dc, stream=stream), 20)
        sel = [0, 511, 1023]
        want = O.polymul_batch(p, a[sel], b[sel])
        ok = bool((dc.view(1024, 8191).cpu().numpy()[sel] == want).all())
        ops = polymul64_ops(13, 4096, 4096, 1024)
        nbytes = 1024 * (2 * 4096 + 8191) * 8
        return {
            "config": {"workload": "1024 products 2^12 x 2^12 mod P1 (62-bit), 2^13-point NTTs, u64",
                       "l2": "flushed before each call"},
            "metric": "products/s", "value": 1024 / (ms * 1e-3), "unit": "products/s", "higher_is_better": True,
            "ms": ms, "roofline": alu_roofline(ops, ms * 1e-3, peak_gops),
            "hbm": hbm_roofline(nbytes, ms * 1e-3, hbm),
            "oracle_checked_products": len(sel), "matches_oracle": ok}


def wl_products_2e16(G, dev, stream, med, peak_gops: float, hbm: float) -> dict:
    """256 products of length 2^15 mod P1 (2^16 points, u64): the direct
    256 x 256 kernels with 64-bit words, the stage that dominates the uneven
    batch (its 2^16-point products and the rows of its longer ones)."""
    import numpy as np
    import torch
    import oracle as O
    from paper_1407_3383_gb300 import workloads as W
    p, batch, n = W.P1, 256, 1 << 15
    g = W.SplitMix64(W.SEED_BASE + 21)
    a = g.uniform_mod(p, batch * n).reshape(batch, n)
    b = g.uniform_mod(p, batch * n).reshape(batch, n)
    with G.Plan(p, 16) as plan:
        da = torch.from_numpy(a.reshape(-1)).to(dev)
        db = torch.from_numpy(b.reshape(-1)).to(dev)
        dc = torch.empty(batch * (2 * n - 1), dtype=torch.uint64, device=dev)
        ws = G.alloc_workspace(plan, batch)
        ms = med(lambda: G.polymul_mod_p_batch(plan, da, n, db, n, batch, dc, G.NTT_SCHED_FUSED, ws,
                                               stream=stream), 20)
        sel = [0, batch - 1]
        want = O.polymul_batch(p, a[sel], b[sel])
        ok = bool((dc.view(batch, 2 * n - 1).cpu().numpy()[sel] == want).all())
        ops = polymul64_ops(16, n, n, batch)
        nbytes = batch * (4 * n - 1) * 8
        return {
            "config": {"workload": "256 products 2^15 x 2^15 mod P1 (62-bit), 2^16-point NTTs, u64",
                       "l2": "flushed before each call"},
            "metric": "products/s", "value": batch / (ms * 1e-3), "unit": "products/s", "higher_is_better": True,
            "ms": ms, "roofline": alu_roofline(ops, ms * 1e-3, peak_gops),
            "hbm": hbm_roofline(nbytes, ms * 1e-3, hbm),
            "oracle_checked_products": len(sel), "matches_oracle": ok}


def uneven_batch(G, dev, stream, flush, med) -> dict:
    """The 10,000-product uneven batch (lengths log-uniform in [2^6, 2^18],
    modulus uniform over P1..P3) in its three run modes, and the same
    products as one polymul_mod_p call per product (its own plan per modulus
    and power-of-two size, issued back to back from the host)."""
    import ctypes
    import numpy as np
    import torch
    from paper_1407_3383_gb300 import workloads as W
    lengths, pidx = W.config3_shapes()
    _, al, bl = W.config3_operands(lengths, pidx)
    primes = [W.P1, W.P2, W.P3]
    count = len(al)
    with G.BatchPlan(primes, [v.size for v in al], [v.size for v in bl], pidx) as bp:
        a = torch.from_numpy(np.concatenate(al)).to(dev)
        b = torch.from_numpy(np.concatenate(bl)).to(dev)
        del al, bl
        c = torch.empty(bp.c_words, dtype=torch.uint64, device=dev)
        ws = torch.empty(bp.workspace_size(), dtype=torch.uint8, device=dev)
        modes = {}
        for mode, nm in [(G.NTT_BATCH_DIRECT, "direct"), (G.NTT_BATCH_STREAMS, "streams"),
                         (G.NTT_BATCH_GRAPH, "graph")]:
            modes[nm + "_ms"] = med(lambda: bp.run(a, b, c, ws, mode, stream=stream), 5, warm=2)
        # device time by kernel in one direct-mode run (launch profiling)
        per, _ = profile_window(G, lambda: bp.run(a, b, c, ws, G.NTT_BATCH_DIRECT, stream=stream), flush, 1)
        by_kernel = {k: round(sum(v), 4) for k, v in sorted(per.items(), key=lambda kv: -sum(kv[1]))}
        # one call per product
        L = np.asarray(lengths, dtype=np.int64)
        logn = np.array([max(1, int(2 * v - 2).bit_length()) for v in L])   # ceil(log2(2 L - 1))
        plans = {}
        for pi, k in set(zip(pidx.tolist(), logn.tolist())):
            plans[(pi, k)] = G.Plan(primes[pi], k)
        ws1 = max(G.polymul_workspace_size(pl, 1) for pl in plans.values())
        wsp = torch.empty(max(ws1, 256), dtype=torch.uint8, device=dev)
        c2 = torch.empty_like(c)
        offa = np.concatenate([[0], np.cumsum(L)[:-1]]) * 8
        offc = np.concatenate([[0], np.cumsum(2 * L - 1)[:-1]]) * 8
        lib = G.lib()
        fn = lib.polymul_mod_p
        st = stream.cuda_stream
        calls = [(plans[(int(pidx[t]), int(logn[t]))].handle, a.data_ptr() + int(offa[t]), int(L[t]),
                  b.data_ptr() + int(offa[t]), int(L[t]), c2.data_ptr() + int(offc[t])) for t in range(count)]
        wp, wb_ = wsp.data_ptr(), wsp.numel()

        def per_product():
            for h, pa, la, pb, lb, pc in calls:
                rc = fn(h, pa, la, pb, lb, pc, wp, wb_, st)
                if rc:
                    raise G.NttError(rc, "polymul_mod_p")

        loop_ms = med(per_product, 3, warm=1)
        same = bool(torch.equal(c.view(torch.int64), c2.view(torch.int64)))
        for pl in plans.values():
            pl.close()
        del a, b, c, c2, ws, wsp
    best = min(modes.values())
    return {"config": {"workload": "10,000 products, lengths log-uniform in [2^6, 2^18] (both operands), "
                                   "modulus uniform over three 62-bit primes k*2^40+1, u64",
                       "l2": "flushed before each run"},
            "metric": "products/s", "value": count / (modes["graph_ms"] * 1e-3), "unit": "products/s",
            "higher_is_better": True, **modes,
            "per_product_calls_ms": loop_ms,
            "per_product_note": "one polymul_mod_p call per product, back to back on one stream from a "
                                "Python loop over prebuilt ctypes arguments (power-of-two sizes, no TFT)",
            "batched_over_per_product": loop_ms / modes["graph_ms"],
            "best_mode_products_per_s": count / (best * 1e-3),
            "direct_mode_kernel_ms": by_kernel,
            "per_product_equals_batched": same}


def serve_closed_loop(G, requests: int = 48) -> dict:
    """A closed-loop run of the serving loop: `requests` integer products
    (operand bits log-uniform in [2^14, 2^28]) submitted at once after a
    warm-up pass; products/s and p50/p99 latency."""
    import numpy as np
    import torch
    from paper_1407_3383_gb300 import workloads as W
    _, limbs = W.config4_requests(requests, rate=1.0)
    g = W.SplitMix64(W.SEED_BASE + 4 + (1 << 32))
    reqs = []
    for n in limbs:
        n = int(n)
        reqs.append((torch.from_numpy(g.limbs(n)).pin_memory(), torch.from_numpy(g.limbs(n)).pin_memory(),
                     torch.empty(2 * n, dtype=torch.uint32).pin_memory()))
    srv = G.Server(max_limbs=int(limbs.max()), mem_bytes=8 << 30, slots=4)

    def burst():
        start = time.perf_counter()
        ids = [srv.submit(G.NTT_REQ_INTMUL, a, b, c) for a, b, c in reqs]
        lat = []
        for rid in ids:
            lat.append(srv.wait(rid, 600000))
            srv.release(rid)
        return np.array(lat), time.perf_counter() - start

    burst()
    lat, span = burst()
    # one request checked against Python integers (the product of the limbs)
    k = int(np.argmin(limbs))
    a, b, c = reqs[k]
    to_int = lambda v: int.from_bytes(v.numpy().astype("<u4").tobytes(), "little")
    ok = to_int(c) == to_int(a) * to_int(b)
    stats = srv.stats()
    srv.close()
    return {"config": {"workload": f"closed loop of {requests} integer products, operand bits log-uniform in "
                                   "[2^14, 2^28], three 62-bit primes, minimal-d chunks (80-91 bits), CRT + carry",
                       "slots": 4, "arena_gib": 8, "mean_bits": float(limbs.mean() * 32)},
            "metric": "integer products/s", "value": requests / span, "unit": "products/s",
            "higher_is_better": True, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "peak_inflight": stats["peak_inflight"],
            "checked_smallest_request": ok}


def run_one_workload(args, world, rank, local):
    """One of the default line's other workloads, alone, as a JSON line."""
    import torch
    import paper_1407_3383_gb300 as G
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    probe = measure_probes(G, stream)
    peak = probe.get("mixed_gops") or SM_COUNT * INT_LANES_PER_SM * SM_MAX_MHZ * 1e-3
    res = run_workloads(G, dev, stream, lambda: flush_buf.fill_(1), peak, measured_hbm_gbs(), only=args.workload)
    if rank == 0:
        print(json.dumps(dict(res[args.workload], name=args.workload, n_gpus=world, int_probe=probe)), flush=True)


def run_native(args, world, rank, local):
    import numpy as np
    import torch
    import paper_1407_3383_gb300 as G

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    p, a, b = make_inputs()
    batch, na = a.shape
    nb = b.shape[1]
    nc = na + nb - 1
    log2n = WORKLOAD["log2n"]
    plan = G.Plan(p, log2n, G.NTT_FLAG_PLAIN)
    wb = plan.word_bytes
    da = torch.from_numpy(a.reshape(-1)).to(dev)
    db = torch.from_numpy(b.reshape(-1)).to(dev)
    dc = torch.empty(batch * nc, dtype=torch.uint32, device=dev)
    ws_f = G.alloc_workspace(plan, batch, G.NTT_SCHED_FUSED)
    ws_p = G.alloc_workspace(plan, batch, G.NTT_SCHED_PLAIN)
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    # the project's autotuner picks the launch shape for this (word size, n)
    # before anything is timed
    tuned_ms = None if args.no_autotune else G.ntt_autotune(plan, batch, stream=stream)
    shape = dict(zip(["log2_products_per_block", "log2_columns_per_block", "log2_rows_per_block"],
                     G.ntt_tune_get(plan.word_bytes, log2n)))
    direct = log2n >= 16 and shape["log2_columns_per_block"] == 0
    shape["kernels"] = ("direct 256 x 256" + (", operand tiles by TMA" if shape["log2_products_per_block"] & 1
                                              else "") if direct else "generic")
    if direct:
        del shape["log2_products_per_block"], shape["log2_columns_per_block"], shape["log2_rows_per_block"]

    def flush():
        flush_buf.fill_(1)

    def step_fused():
        G.polymul_mod_p_batch(plan, da, na, db, nb, batch, dc, G.NTT_SCHED_FUSED, ws_f,
                              stream=stream)

    def step_plain():
        G.polymul_mod_p_batch(plan, da, na, db, nb, batch, dc, G.NTT_SCHED_PLAIN, ws_p,
                              stream=stream)

    for _ in range(max(3, args.warmup)):
        step_fused()
        if args.only is None:
            step_plain()
    torch.cuda.synchronize()

    if args.only == "fused":
        ms = timed_steps(step_fused, flush, args.steps, stream)
        if rank == 0:
            print(json.dumps({"only": "fused", "ms_per_step": sum(ms) / len(ms),
                              "value": batch / (sum(ms) / len(ms) / 1e3), "unit": UNIT}))
        plan.close()
        return

    # ---- fused: the reported value
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ms = timed_steps(step_fused, flush, args.steps, stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_s = reduce_max(sum(ms) / 1e3, world)
    value = whole_job_value(batch, world, total_s / args.steps)
    ms_per_step = 1e3 * total_s / args.steps

    # ---- per-kernel device time (launch profiling, same steps)
    per_kernel, launches_per_step = profile_window(G, step_fused, flush, max(5, args.steps // 4))
    kops = fused_kernel_ops(log2n, na, nb, batch, plan.info.tile_max_log)
    shares = {k: sum(v) for k, v in per_kernel.items()}
    dom = max(shares, key=shares.get)
    dom_ms = statistics.mean(per_kernel[dom])
    dom_ops = kops.get(dom, 0)

    # ---- plain schedule, same inputs
    psteps = args.plain_steps or max(3, args.steps // 4)
    pms = timed_steps(step_plain, flush, psteps, stream)
    plain_s = reduce_max(sum(pms) / 1e3, world)
    plain_value = whole_job_value(batch, world, plain_s / psteps)

    # ---- end to end: pinned host buffers, copies inside the timed region.
    # polymul_mod_p_batch_host uploads, multiplies and downloads chunk by
    # chunk on overlapping streams; the chunk size is picked from a short
    # sweep (3 calls each) before the timed calls.
    ha = torch.from_numpy(a.reshape(-1)).pin_memory()
    hb = torch.from_numpy(b.reshape(-1)).pin_memory()
    hc = torch.empty(batch * nc, dtype=torch.uint32).pin_memory()
    e2e_steps = max(3, args.steps // 4)
    chunks = sorted({c for c in (16, 32, 48, 64, 80, 128, batch) if c <= batch})
    stage = torch.empty(max(G.polymul_host_stage_size(plan, na, nb, c) for c in chunks),
                        dtype=torch.uint8, device=dev)

    def e2e_seconds(chunk, reps):
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(reps):
            G.polymul_mod_p_batch_host(plan, ha, na, hb, nb, batch, hc, chunk, stage, stream=stream)
        torch.cuda.synchronize()
        return reduce_max(time.perf_counter() - t0, world) / reps

    sweep = {}
    for c in chunks:
        e2e_seconds(c, 1)
        sweep[c] = e2e_seconds(c, 3)
    e2e_chunk = min(sweep, key=sweep.get)
    e2e_value = whole_job_value(batch, world, e2e_seconds(e2e_chunk, e2e_steps))
    e2e_ok = bool((hc.numpy() == dc.cpu().numpy()).all())

    # ---- fused and plain give the same words (dc holds the plain result)
    plain_out = dc.clone()
    step_fused()
    torch.cuda.synchronize()
    fused_equals_plain = bool(torch.equal(dc.view(torch.int32), plain_out.view(torch.int32)))
    del plain_out

    # ---- integer-issue probes: the roof of the integer-bound kernels
    probe = measure_probes(G, stream)
    peak_gops = probe.get("mixed_gops") or SM_COUNT * INT_LANES_PER_SM * SM_MAX_MHZ * 1e-3
    peak_basis = ("measured: ntt_int_probe mixed kind (independent 32-bit multiply-add and add/xor chains "
                  "1:1, 152 x 8 blocks of 256 threads), this run" if probe.get("mixed_gops") else
                  "152 SMs x 128 int32 lanes x 2070 MHz (unit counts and max clock; the probe failed)")
    achieved_gops = dom_ops / (dom_ms * 1e-3) / 1e9

    bytes_step = alg_bytes(na, nb, batch, wb)
    hbm = measured_hbm_gbs()
    gbps = bytes_step / (ms_per_step * 1e-3) / 1e9

    # ---- the other workloads (N = 1 line only)
    workloads = None
    if world == 1 and not args.no_workloads:
        workloads = run_workloads(G, dev, stream, flush, peak_gops, hbm)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import numpy as np
        cv, cores, sample, prods = time_oracle(p, a, b)
        got = dc.view(batch, nc)[:prods.shape[0]].cpu().numpy().astype(np.uint64)
        cpu = {"value": cv, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "parity_checked_products": int(prods.shape[0]),
               "parity_ok": bool((got == prods).all())}
        nv, ncores, nsample, nprods = time_cpu_ntt(p, a, b)
        ngot = dc.view(batch, nc)[:nprods.shape[0]].cpu().numpy().astype(np.uint64)
        cpu["ntt_reference"] = {"value": nv, "unit": UNIT, "cores": ncores,
                                "kind": "textbook radix-2 transform product (O(n log n) CPU reference)",
                                "sample": nsample, "equals_device_result": bool((ngot == nprods).all()),
                                "gpu_over_cpu_ntt": value / nv}

    if rank != 0:
        plan.close()
        return
    traffic = ncu_traffic(dom)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(WORKLOAD, l2="flushed between timed steps (256 MiB write)",
                       schedule="fused", parallelism=f"replicas x{world}", launch_shape=shape,
                       autotune_best_ms=tuned_ms),
        "gbps_algorithmic": gbps,
        "hbm_frac_of_measured": gbps / hbm,
        "plain": {"value": plain_value, "ms_per_step": 1e3 * plain_s / psteps,
                  "fused_over_plain": value / plain_value},
        "roofline": {"bound": "alu", "achieved": achieved_gops, "peak": peak_gops,
                     "unit": "Gop/s", "frac": achieved_gops / peak_gops, "traffic": traffic,
                     "kernel": dom, "kernel_ms": dom_ms, "peak_basis": peak_basis,
                     "unit_count_peak_gops": SM_COUNT * INT_LANES_PER_SM * SM_MAX_MHZ * 1e-3,
                     "int_probe": probe},
        "fused_equals_plain": fused_equals_plain,
        "kernels": {k: {"ms_mean": statistics.mean(v), "share": shares[k] / sum(shares.values()),
                        "alg_gop_per_launch": kops.get(k, 0) / 1e9} for k, v in per_kernel.items()},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": (na + nb) * batch * wb,
                "d2h_bytes_per_step": nc * batch * wb,
                "call": "polymul_mod_p_batch_host (pinned host buffers, chunked upload/product/download overlap)",
                "chunk": e2e_chunk, "chunk_sweep_ms": {str(k): round(v * 1e3, 4) for k, v in sweep.items()},
                "matches_device_result": e2e_ok},
        "clocks": clk,
        "cpu_baseline": cpu,
        "workloads": workloads,
    }
    print(json.dumps(line), flush=True)
    plan.close()


# ---------------------------------------------------------------- serving workload

def run_serve(args, world, rank, local):
    """Poisson stream of integer products (operand sizes log-uniform in
    [2^14, 2^28] bits) through the serving loop: a closed-loop run gives the
    saturating rate; open-loop runs at 0.5/0.8/1.0/1.2 of it give p50/p99
    latency beside the achieved rate."""
    import numpy as np
    import torch
    import paper_1407_3383_gb300 as G
    from paper_1407_3383_gb300 import workloads as W

    torch.cuda.set_device(local)
    _, limbs = W.config4_requests(args.requests, rate=1.0)
    g = W.SplitMix64(W.SEED_BASE + 4 + (1 << 32))
    reqs = []
    for n in limbs:
        n = int(n)
        a = torch.from_numpy(g.limbs(n)).pin_memory()
        b = torch.from_numpy(g.limbs(n)).pin_memory()
        c = torch.empty(2 * n, dtype=torch.uint32).pin_memory()
        reqs.append((a, b, c))
    max_limbs = int(limbs.max())
    t0 = time.perf_counter()
    srv = G.Server(max_limbs=max_limbs, mem_bytes=24 << 30, slots=4)
    setup_s = time.perf_counter() - t0

    def stream(arrivals):
        ids, lat = [], []
        start = time.perf_counter()
        for (a, b, c), t_arr in zip(reqs, arrivals):
            now = time.perf_counter() - start
            if t_arr > now:
                time.sleep(t_arr - now)
            ids.append(srv.submit(G.NTT_REQ_INTMUL, a, b, c))
        for rid in ids:
            lat.append(srv.wait(rid, 600000))
            srv.release(rid)
        span = time.perf_counter() - start
        return np.array(lat), span

    stream(np.zeros(len(reqs)))                           # warm-up: every size class launched once
    lat, span = stream(np.zeros(len(reqs)))                # closed loop: all at once
    sat = len(reqs) / span
    runs = [{"load": "closed", "products_per_s": sat, "p50_ms": float(np.percentile(lat, 50)),
             "p99_ms": float(np.percentile(lat, 99))}]
    for f in [0.5, 0.8, 1.0, 1.2]:
        arr, _ = W.config4_requests(len(reqs), rate=f * sat)
        lat, span = stream(arr)
        runs.append({"load": f, "offered_per_s": f * sat, "products_per_s": len(reqs) / span,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))})
    stats = srv.stats()
    srv.close()
    bits = limbs * 32
    if rank == 0:
        print(json.dumps({
            "metric": "serving: integer products/s and p50/p99 latency (3-prime NTT + CRT + carry)",
            "value": sat, "unit": "products/s", "n_gpus": world, "higher_is_better": True,
            "data": "synthetic", "dtype": "u64",
            "config": {"workload": f"Poisson stream of {len(reqs)} integer products, operand bits "
                                   "log-uniform in [2^14, 2^28], 3 primes k*2^40+1, minimal-d chunks (80-91 bits)",
                       "mean_bits": float(bits.mean()), "max_bits": int(bits.max()),
                       "slots": 4, "arena_gib": 24},
            "runs": runs, "peak_inflight": stats["peak_inflight"], "server_setup_s": setup_s,
        }), flush=True)


def run_modmul(args, world, rank, local):
    """Throughput of each modular-product variant (Functions 6, 8, 13, 16 and
    the kernels' Remark 8 form) on register-resident operands: the
    floating-point-quotient ablation against the integer reductions."""
    import paper_1407_3383_gb300 as G
    from paper_1407_3383_gb300 import workloads as W
    import torch
    torch.cuda.set_device(local)
    names = {G.NTT_MM_BARRETT: "barrett_f6", G.NTT_MM_SHOUP: "shoup_f8",
             G.NTT_MM_MONTGOMERY: "montgomery_f13", G.NTT_MM_FMA: "fp64_fma_f16",
             G.NTT_MM_MONT_FIXED: "montgomery_fixed_remark8"}
    cases = [(W.P_TABLE11, 4, "469762049 (29-bit, u32)"), (W.P_B, 4, "3*2^30+1 (32-bit, u32)"),
             (W.P_TABLE12, 8, "1108307720798209 (50-bit, u64)"), (W.P1, 8, "P1 (62-bit, u64)")]
    res = {}
    for p, wb, label in cases:
        row = {}
        for kind, nm in names.items():
            try:
                row[nm] = G.ntt_modmul_rate(p, kind, wb, 2048) / 1e9
            except G.NttError:
                row[nm] = None
        res[label] = row
    if rank == 0:
        print(json.dumps({"metric": "modular products per second by reduction (G/s), register-resident",
                          "unit": "Gmulmod/s", "results": res, "n_gpus": world}), flush=True)


def run_suite(args, world, rank, local):
    """Context lines for the workloads other than the headline: one 4096-point
    product (latency, and graph-replayed rate), 1024 products of 2^12 words
    and one 2^24-point transform mod P1, the 10,000-product uneven batch, the
    polynomial matrix product at Table 15's largest shape and the integer
    matrix product at Table 17's.  Device time with CUDA events on the
    launching stream, L2 flushed before every timed repetition."""
    import numpy as np
    import torch
    import paper_1407_3383_gb300 as G
    from paper_1407_3383_gb300 import workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    def flush():
        flush_buf.fill_(1)

    def med(step, reps, warm=3):
        for _ in range(warm):
            step()
        torch.cuda.synchronize()
        return statistics.median(timed_steps(step, flush, reps, stream))

    def emit(name, **kw):
        if rank == 0:
            print(json.dumps(dict(workload=name, n_gpus=world, context=True, **kw)), flush=True)

    # one product of two length-2048 operands mod 998244353 (4096 points)
    p, a, b = W.config0()
    with G.Plan(p, 12) as plan:
        da = torch.from_numpy(a.astype(np.uint32)).to(dev)
        db = torch.from_numpy(b.astype(np.uint32)).to(dev)
        dc = torch.empty(4095, dtype=torch.uint32, device=dev)
        ms = med(lambda: G.polymul_mod_p(plan, da, 2048, db, 2048, dc, stream=stream), 50)
        side = torch.cuda.Stream(device=dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            G.polymul_mod_p(plan, da, 2048, db, 2048, dc, stream=side)
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=side):
                for _ in range(100):
                    G.polymul_mod_p(plan, da, 2048, db, 2048, dc, stream=side)
        gms = med(lambda: graph.replay(), 10)
        emit("1 product 2048 x 2048 mod 998244353 (4096 points, u32)",
             us_per_product=1e3 * ms, graph_replayed_products_per_s=100 / (gms * 1e-3))

    # 1024 products of length 2^12 mod P1 (2^13 points, u64)
    p, a, b = W.config2_products()
    with G.Plan(p, 13) as plan:
        da = torch.from_numpy(a.reshape(-1)).to(dev)
        db = torch.from_numpy(b.reshape(-1)).to(dev)
        dc = torch.empty(1024 * 8191, dtype=torch.uint64, device=dev)
        ms = med(lambda: G.polymul_mod_p_batch(plan, da, 4096, db, 4096, 1024, dc, stream=stream), 20)
        emit("1024 products 2^12 x 2^12 mod P1 (2^13 points, u64)", ms=ms,
             products_per_s=1024 / (ms * 1e-3), gbps_algorithmic=1024 * (2 * 4096 + 8191) * 8 / (ms * 1e-3) / 1e9)

    # one 2^24-point transform mod P1, forward then inverse
    p, x = W.config2_transform()
    with G.Plan(p, 24) as plan:
        dx = torch.from_numpy(x).to(dev)
        fms = med(lambda: G.ntt_forward(plan, dx, 1, stream=stream), 10)
        ims = med(lambda: G.ntt_inverse(plan, dx, 1, stream=stream), 10)
        emit("one 2^24-point transform mod P1 (u64)", forward_ms=fms, inverse_ms=ims,
             gbps_algorithmic_one_sweep_each=2 * 2 * (1 << 24) * 8 / ((fms + ims) * 1e-3) / 1e9)

    # 10,000 uneven products, lengths log-uniform in [2^6, 2^18], primes P1..P3
    lengths, pidx = W.config3_shapes()
    _, al, bl = W.config3_operands(lengths, pidx)
    with G.BatchPlan([W.P1, W.P2, W.P3], [v.size for v in al], [v.size for v in bl], pidx) as bp:
        a = torch.from_numpy(np.concatenate(al)).to(dev)
        b = torch.from_numpy(np.concatenate(bl)).to(dev)
        c = torch.empty(bp.c_words, dtype=torch.uint64, device=dev)
        ws = torch.empty(bp.workspace_size(), dtype=torch.uint8, device=dev)
        modes = {}
        for mode, nm in [(G.NTT_BATCH_DIRECT, "direct"), (G.NTT_BATCH_STREAMS, "streams"),
                         (G.NTT_BATCH_GRAPH, "graph")]:
            modes[nm + "_ms"] = med(lambda: bp.run(a, b, c, ws, mode, stream=stream), 5, warm=2)
        del a, b, c, ws
        emit("10,000 uneven products mod P1..P3 (u64)", **modes,
             products_per_s=10000 / (min(modes.values()) * 1e-3))

    # polynomial matrix product, n = 32, degree < 2^15 mod 469762049 (Table 15's largest)
    p, n, d = W.P_TABLE11, 32, 1 << 15
    g = W.SplitMix64(W.SEED_BASE + 15)
    with G.Plan(p, 16) as plan:
        A = torch.from_numpy(g.uniform_mod(p, n * n * d).astype(np.uint32)).to(dev)
        B = torch.from_numpy(g.uniform_mod(p, n * n * d).astype(np.uint32)).to(dev)
        C = torch.empty(n * n * (2 * d - 1), dtype=torch.uint32, device=dev)
        ws = torch.empty(G.polymat_workspace_size(plan, n), dtype=torch.uint8, device=dev)
        step = lambda: G.polymat_mul(plan, A, B, n, d, C, ws, stream=stream)
        ms = med(step, 10)
        per, _ = profile_window(G, step, flush, 3)
        freq_ms = statistics.mean(per.get("k_polymat_freq", [ms]))
        macs = n ** 3 * (1 << 16) / (freq_ms * 1e-3)
        imad_peak = SM_COUNT * 64 * 2.07e9              # one 32-bit multiply-add pipe: 64 lanes per SM
        emit("polynomial matrix product 32 x 32, degree < 2^15, mod 469762049 (u32)", ms=ms,
             kernels_ms={k: statistics.mean(v) for k, v in per.items()},
             freq_mulmod_per_s=macs,
             freq_roofline={"bound": "alu (wide multiply-add pipe)", "achieved": macs, "peak": imad_peak,
                            "frac": macs / imad_peak, "unit": "multiply-adds/s",
                            "peak_basis": "152 SMs x 64 lanes x 2070 MHz; one wide multiply-add per term"})
        del A, B, C, ws

    # one integer product of two equal operands (three 62-bit primes, minimal-d
    # chunks, Garner CRT, carry) at 2^20 .. 2^26 bits
    g = W.SplitMix64(W.SEED_BASE + 16)
    rows = []
    with G.IntmulPlan(1 << 21) as plan:
        for bits in (20, 22, 24, 26):
            nl = (1 << bits) // 32
            A = torch.from_numpy(g.limbs(nl)).to(dev)
            B = torch.from_numpy(g.limbs(nl)).to(dev)
            C = torch.empty(2 * nl, dtype=torch.uint32, device=dev)
            ws = torch.empty(G.intmul_workspace_size(plan, nl, nl), dtype=torch.uint8, device=dev)
            ms = med(lambda: G.intmul_crt(plan, A, nl, B, nl, C, ws, stream=stream), 10)
            rows.append({"bits": 1 << bits, "ms": round(ms, 4)})
            del A, B, C, ws
    emit("one integer product of two equal operands (three 62-bit primes)", rows=rows)

    # integer matrix product, n = 32, entries of 2^15 limbs (Table 17's shape)
    n, na = 32, 1 << 15
    g = W.SplitMix64(W.SEED_BASE + 17)
    with G.IntmulPlan(1 << 16) as plan:
        A = torch.from_numpy(g.limbs(n * n * na)).to(dev)
        B = torch.from_numpy(g.limbs(n * n * na)).to(dev)
        C = torch.empty(n * n * (2 * na + 1), dtype=torch.uint32, device=dev)
        ws = torch.empty(G.intmat_workspace_size(plan, n, na, na), dtype=torch.uint8, device=dev)
        step = lambda: G.intmat_mul(plan, A, na, B, na, n, C, ws, stream=stream)
        ms = med(step, 5)
        per, _ = profile_window(G, step, flush, 2)
        emit("integer matrix product 32 x 32, entries of 2^15 limbs (2^20 bits)", ms=ms,
             kernels_ms={k: statistics.mean(v) for k, v in per.items()})


def run_fp64(args, world, rank, local):
    """Table 12's sizes (n = 2^8 .. 2^20, p = 1108307720798209): batched
    forward transforms over doubles with Function 16 (NTT_FLAG_FP64) against
    the integer Shoup transforms of the same prime, 2^24 words per launch,
    device time per transform (CUDA events, L2 flushed before each)."""
    import numpy as np
    import torch
    import paper_1407_3383_gb300 as G
    from paper_1407_3383_gb300 import workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    p = W.P_TABLE12
    total = 1 << 24
    x = W.SplitMix64(W.SEED_BASE + 12).uniform_mod(p, total)
    rows = []
    for log2n in range(8, 21):
        batch = total >> log2n
        res = {"log2n": log2n, "batch": batch}
        for flag, name, dt in [(G.NTT_FLAG_FP64, "fp64_fma_us", np.float64), (0, "int_shoup_us", np.uint64)]:
            with G.Plan(p, log2n, flag) as plan:
                d = torch.from_numpy(x.astype(dt)).to(dev)
                step = lambda: G.ntt_forward(plan, d, batch, stream=stream)
                for _ in range(3):
                    step()
                torch.cuda.synchronize()
                ms = statistics.median(timed_steps(step, lambda: flush_buf.fill_(1), 10, stream))
                res[name] = 1e3 * ms / batch
        res["int_over_fp64_speed"] = res["fp64_fma_us"] / res["int_shoup_us"]
        rows.append(res)
    if rank == 0:
        print(json.dumps({"metric": "forward transform time per transform (us), Table 12 sizes",
                          "p": p, "words_per_launch": total, "n_gpus": world, "rows": rows}), flush=True)


def run_tft(args, world, rank, local):
    """256 products mod 3*2^30+1 with n = 2^16 whose outputs need B of the 16
    row blocks (na = nb = 2048 B): the truncated transforms (TFT, Section
    5.1) against the full-length step that zero padding to n would cost."""
    import numpy as np
    import torch
    import paper_1407_3383_gb300 as G
    from paper_1407_3383_gb300 import workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    batch = 256
    g = W.SplitMix64(W.SEED_BASE + 51)
    for p, dt in [(W.P_B, np.uint32), (W.P1, np.uint64)]:
        rows = []
        with G.Plan(p, 16) as plan:
            ws = G.alloc_workspace(plan, batch)
            for beta in [16, 14, 13, 12, 11, 10, 8, 6, 4, 2, 1]:
                na = nb = 2048 * beta
                a = torch.from_numpy(g.uniform_mod(p, batch * na).astype(dt)).to(dev)
                b = torch.from_numpy(g.uniform_mod(p, batch * nb).astype(dt)).to(dev)
                c = torch.empty(batch * (na + nb - 1), dtype=a.dtype, device=dev)
                step = lambda: G.polymul_mod_p_batch(plan, a, na, b, nb, batch, c, G.NTT_SCHED_FUSED, ws,
                                                     stream=stream)
                for _ in range(3):
                    step()
                torch.cuda.synchronize()
                ms = statistics.median(timed_steps(step, lambda: flush_buf.fill_(1), 20, stream))
                rows.append({"blocks": beta, "na": na, "nb": nb, "ms": ms,
                             "products_per_s": batch / (ms * 1e-3)})
                del a, b, c
        full = rows[0]["ms"]
        for r in rows:
            r["time_vs_padded"] = r["ms"] / full
        if rank == 0:
            print(json.dumps({"metric": "2^16-point products by output length (truncated transforms)",
                              "p": p, "batch": batch, "n_gpus": world, "rows": rows}), flush=True)
    # one-block sizes and the two-pass sizes below 2^16: 2^23 output words
    # per call; the output needs kb of the 16 blocks of n/16 positions, and
    # kb = 16 is what padding to n costs at every kb
    for p, dt in [(W.P_B, np.uint32), (W.P1, np.uint64)]:
        for log2n in range(8, 16):
            n = 1 << log2n
            batch = max(16, (1 << 23) >> log2n)
            rows = []
            with G.Plan(p, log2n) as plan:
                ws = G.alloc_workspace(plan, batch)
                for kb in [16, 14, 12, 10, 9]:
                    L = kb * n // 16
                    na = (L + 1) // 2
                    nb = L + 1 - na
                    a = torch.from_numpy(g.uniform_mod(p, batch * na).astype(dt)).to(dev)
                    b = torch.from_numpy(g.uniform_mod(p, batch * nb).astype(dt)).to(dev)
                    c = torch.empty(batch * L, dtype=a.dtype, device=dev)
                    step = lambda: G.polymul_mod_p_batch(plan, a, na, b, nb, batch, c, G.NTT_SCHED_FUSED,
                                                         ws, stream=stream)
                    for _ in range(3):
                        step()
                    torch.cuda.synchronize()
                    ms = statistics.median(timed_steps(step, lambda: flush_buf.fill_(1), 20, stream))
                    rows.append({"blocks": kb, "na": na, "nb": nb, "ms": round(ms, 5)})
                    del a, b, c
            for r in rows:
                r["time_vs_padded"] = round(r["ms"] / rows[0]["ms"], 3)
            if rank == 0:
                print(json.dumps({"metric": "products by output length (truncated transforms)", "p": p,
                                  "log2n": log2n, "batch": batch, "rows": rows}), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.workload == "modmul" and args.impl == "native":
        run_modmul(args, world, rank, local)
    elif args.workload == "serve" and args.impl == "native":
        run_serve(args, world, rank, local)
    elif args.workload == "suite" and args.impl == "native":
        run_suite(args, world, rank, local)
    elif args.workload == "fp64" and args.impl == "native":
        run_fp64(args, world, rank, local)
    elif args.workload == "tft" and args.impl == "native":
        run_tft(args, world, rank, local)
    elif args.workload in ("single_product", "transform_2e24_u64", "products_2e12_u64", "products_2e16_u64",
                           "uneven_10000", "serving") and args.impl == "native":
        run_one_workload(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_native(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
