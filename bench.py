#!/usr/bin/env python
"""Benchmark of C = A B over GF(2) on GB300: square n = 32768, Bernoulli(1/2) bits.

One step is one whole product through the library: Strassen-Winograd
additions (Algorithm 4) at every level, the base case on all leaves, and the
recombination.  The packed Method-of-the-Four-Russians base case and the
tensor-core base case are timed side by side on the same resident inputs;
the faster one is the headline.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank multiplies its own pair of matrices (the
problems are independent, no data-path collective); the value is the bit
operations of all ranks over the slowest rank's time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "effective GF(2) bit-ops/s (2mnk/t) at n=32768, bit-exact"

# DRAM traffic of the dominant kernel from an ncu capture of it (see
# profiles/m4rm_kernel_n16384_depth2.md): bytes read + written per byte of leaf
# operands (A, B, C slabs), valid while the code of the kernel sources (comments
# and blank lines removed) hashes to "sha".
NCU_TRAFFIC = {
    "m4rm": {"sha": "1e46ef05f46c7c8d", "sources": ["paper_0811_1714_gb300/csrc/m4rm.cu",
                                                  "paper_0811_1714_gb300/csrc/m4rm_dev.cuh"],
             "bytes_per_operand_byte": 0.8845},
    # profiles/tc_mma_kernel_fp4_n8192_depth1.md: 128.5 MB per launch against 117.4 MB of
    # expanded leaf operands + 14.7 MB of packed leaf products
    "tc_fp4": {"sha": "b9164bcf051a8560", "sources": ["paper_0811_1714_gb300/csrc/tc_mma.cu",
                                                    "paper_0811_1714_gb300/csrc/tcgen05.cuh"],
               "bytes_per_operand_byte": 0.973},
    # profiles/tc_mma_kernel_fp8_n8192_depth1.md: 249.1 MB against 234.9 + 14.7 MB
    "tc_fp8": {"sha": "b9164bcf051a8560", "sources": ["paper_0811_1714_gb300/csrc/tc_mma.cu",
                                                    "paper_0811_1714_gb300/csrc/tcgen05.cuh"],
               "bytes_per_operand_byte": 0.998},
}


def code_sha(paths):
    """sha256 prefix of the sources' code: // and /* */ comments, trailing
    blanks and empty lines removed, so that editing a comment keeps a capture
    valid and any change to the code does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in paths:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


# int8 warp-level tensor rate (mma.sync m16n8k32 .s8, dense) measured on a GB300
# with register-resident operands: the peak for the int8 base case.
S8_MMA_SYNC_TOPS = 157.9
# binary warp-level tensor rate (mma.sync m16n8k256 .b1 .and.popc: AND + popcount
# per bit pair), measured the same way: the peak for the binary base case.
B1_MMA_SYNC_TOPS = 154.2
# shared-memory read bandwidth of all 152 SMs measured on a GB300 at 2070 MHz by a
# probe with the M4RM lookup pattern (each quarter-warp reads one 128-byte row as
# 8 x 16 bytes, four independent rows in flight per thread, one 256-thread CTA per
# SM): 126.1 B/clk/SM, 98.5 % of the nominal 128 B/clk (152 x 128 B x 2070 MHz =
# 40.3 TB/s).  The peak for the packed M4RM base cases (profiles/peaks.md).
SMEM_LOOKUP_GBS = 39690.0
# dense throughput of one tcgen05.mma.cta_group::1 stream per SM (M = 128, N = 256,
# both operands in shared memory, 4 instructions per 128-byte K block) measured on a
# GB300 at 2070 MHz: kind::f8f6f4 (E4M3) and kind::mxf4 (E2M1, scale factors in
# tensor memory).  Context for the tensor-core rooflines (profiles/peaks.md).
MMA_ONLY_TFLOPS = {"tc_fp8": 4855.9, "tc_fp4": 9710.9}


def smem_peak(peaks):
    """(peak GB/s, note) of shared-memory reads: the measured lookup-pattern
    rate, scaled when the clock differs from the 2070 MHz it was taken at."""
    mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = SMEM_LOOKUP_GBS * mhz / 2070.0
    return peak, ("measured shared-memory read rate with the lookup pattern, %.1f TB/s "
                  "(nominal 152 SMs x 128 B/clk x %.0f MHz = %.1f TB/s)" %
                  (peak / 1000.0, mhz, 152 * 128 * mhz / 1e6))


def operand_bytes(fam, leaves, M, L, N):
    """Bytes of the leaf operands a base-case launch reads and writes once:
    packed A, B and C for M4RM; the expanded A and B^T rows (FP8 bytes or
    FP4 nibbles, K rounded up to a 128-byte row) and packed C for the
    tcgen05 forms."""
    if fam in ("tc_fp8", "tc_fp4"):
        epr, eb = (128, 1.0) if fam == "tc_fp8" else (256, 0.5)
        kp = -(-L // epr) * epr
        return leaves * ((M + N) * kp * eb + M * N / 8.0)
    return leaves * (M * L + L * N + M * N) / 8.0


def ncu_traffic(fam, leaves, M, L, N):
    """Per-launch DRAM bytes scaled from the capture, or None if the kernel changed."""
    ent = NCU_TRAFFIC.get(fam)
    if not ent:
        return None
    try:
        if code_sha(ent["sources"]) != ent["sha"]:
            return None
    except OSError:
        return None
    return ent["bytes_per_operand_byte"] * operand_bytes(fam, leaves, M, L, N)
UNIT = "bit-ops/s"
DEFAULT_PATHS = "m4rm,tc_fp8,tc_fp4,tc_s8,tc_b1"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--p", type=float, default=0.5, help="density of one bits (square workload)")
    ap.add_argument("--paths", default=DEFAULT_PATHS, help="base cases to time")
    ap.add_argument("--depth", type=int, default=-1)
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--t", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (config 1, 2, 3 at n=65536, 4, 5) after the headline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of one CPU-oracle sample")
    ap.add_argument("--workload", choices=["square", "batched", "chain", "sweep", "sharded", "peaks"],
                    default="square",
                    help="square: the n x n product (default); batched: 4096 products, "
                         "dimensions log-uniform in [64, 2048], one persistent launch; "
                         "sweep: packed M4RM over Strassen depth x k at n = 8192, 16384, "
                         "32768 and 20000x12000.12000x28000; sharded: one n x n product with "
                         "its rows split over the ranks (torchrun), B broadcast")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- ranks

def aggregate(ms_local, ops_local):
    """Whole-job timing over the ranks of the default process group: the
    slowest rank's time, and the bit operations of all ranks over it.
    Returns (ms, ops_total, value).  One process (no group): the local ones."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ms_local, ops_local, ops_local / (ms_local * 1e-3)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    o = torch.tensor([float(ops_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(o, op=dist.ReduceOp.SUM)
    ms, ops = float(t.item()), float(o.item())
    return ms, ops, ops / (ms * 1e-3)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 20 ms, time-stamped) of SM clock and throttle
    reasons.  Started before the warm-up so that it is running when the timed
    region begins; summary(t0, t1) keeps the samples taken inside it."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self, t0=None, t1=None, pad=0.5):
        """Median SM clock, max clock and throttle reasons of the samples taken
        between host times t0 and t1; when none fall inside (a timed region
        shorter than the sampling period), the samples within `pad` seconds
        of it; else all samples."""
        import datetime
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            try:
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        window = "timed region"
        if t0 is not None and t1 is not None:
            inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
            near = [r for r in rows if r[0] is not None and t0 - pad <= r[0] <= t1 + pad]
            if inside:
                rows = inside
            elif near:
                rows = near
                window = "within %.1f s of the timed region (shorter than the sampling period)" % pad
            else:
                window = "whole run (no sample inside the timed region)"
        else:
            window = "whole run"
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, _, flags in rows:
            for nm, v in zip(names, flags):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "window": window}


# ---------------------------------------------------------------- our arm

def roofline_for(fam, leaves, M, L, N, k, ms_per_launch, peaks, peak_kind):
    """Roofline of the dominant kernel from its algorithmic work per launch."""
    if ms_per_launch <= 0:
        return None
    if fam in ("tc_fp8", "tc_fp4"):
        flops = 2.0 * M * L * N * leaves                    # dense 0/1 product, exact sums
        achieved = flops / (ms_per_launch * 1e-3) / 1e12
        ratio = 2.0 if fam == "tc_fp8" else 6.0              # nominal 4.5 / 13.5 vs 2.25 PFLOP/s bf16
        peak = ratio * peaks["bf16_tflops"]
        mma_only = MMA_ONLY_TFLOPS[fam]
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "frac_of_mma_only": achieved / mma_only,
                "traffic": ncu_traffic(fam, leaves, M, L, N),
                "peak_note": "%g x bf16 burst of %s peaks (nominal %s/bf16 ratio); an MMA-only loop of "
                             "this instruction on this GPU reaches %.0f TFLOP/s" % (
                                 ratio, peak_kind, fam[3:], mma_only)}
    if fam == "tc_b1":
        ops = 2.0 * M * L * N * leaves                      # AND + popcount per bit pair, int32 sums
        achieved = ops / (ms_per_launch * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": B1_MMA_SYNC_TOPS, "unit": "TOPS",
                "frac": achieved / B1_MMA_SYNC_TOPS, "traffic": None,
                "peak_note": "mma.sync m16n8k256 b1 and.popc rate measured on this GPU by a "
                             "register-only throughput loop (tcgen05 has no binary kind on sm_103a)"}
    if fam == "tc_s8":
        ops = 2.0 * M * L * N * leaves                      # dense 0/1 int8 product, int32 sums
        achieved = ops / (ms_per_launch * 1e-3) / 1e12
        peak = S8_MMA_SYNC_TOPS
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TOPS",
                "frac": achieved / peak, "traffic": None,
                "peak_note": "mma.sync m16n8k32 s8 rate measured on this GPU by a register-only "
                             "throughput loop (tcgen05 has no int8 kind on sm_103a)"}
    # packed M4RM: table-row reads from shared memory, M*L*N/(8k) bytes per product
    smem_bytes = M * L * N / (8.0 * k) * leaves
    achieved = smem_bytes / (ms_per_launch * 1e-3) / 1e9
    peak, note = smem_peak(peaks)
    nominal = 152 * 128 * peaks.get("sm_max_mhz", 2070.0) / 1e3
    return {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "frac_of_nominal": achieved / nominal,
            "traffic": ncu_traffic("m4rm", leaves, M, L, N),
            "traffic_note": "DRAM bytes per launch, scaled by leaf operand bytes from a 49-leaf ncu capture",
            "peak_note": note}


def strassen_stream_bytes(M, L, N, d, leaf_bytes_per_entry=0.125):
    """Algorithmic HBM bytes per product of the Strassen-Winograd additions
    (padded sizes M, L, N, depth d), following the launch schedule: splits
    go top-down two levels per launch (reading the parents of A, M x L, and
    of B, L x N, writing 49 or 7 children each; the last level's children at
    `leaf_bytes_per_entry`: 1/8 packed, 1/2 or 1 when they are written
    expanded for the FP4 or FP8 base case, by a single-level split of their
    own); combines go bottom-up two levels
    per launch (reading 7^j products of level j, writing level j-2 or j-1,
    C-sized at level 0)."""
    split = comb = 0.0
    fused = leaf_bytes_per_entry != 0.125
    j = 1
    while j <= d:
        step = 2 if d - j + 1 >= 2 else 1
        if fused and step == 2 and j + 1 == d:
            step = 1                      # the expanded leaves come from a single-level split
        jt = j + step - 1
        parents = 7 ** (j - 1)
        children = 7 ** jt
        out = leaf_bytes_per_entry if jt == d else 0.125
        split += parents * (M * L + L * N) / 4 ** (j - 1) / 8.0 + children * (M * L + L * N) / 4 ** jt * out
        j += step
    j = d
    while j >= 1:
        step = 2 if j >= 2 else 1
        jp = j - step
        comb += (7 ** j * M * N / 4 ** j + 7 ** jp * M * N / 4 ** jp) / 8.0
        j -= step
    return split, comb


L2_BYTES = 129 * 2**20


class L2Flush:
    """Writes a buffer larger than the 129 MB L2 on the timing stream, so that
    the next timed product starts from a cold cache."""

    def __init__(self, torch):
        self.buf = torch.empty(256 * 2**20, dtype=torch.uint8, device="cuda")
        self.k = 0

    def __call__(self):
        self.k = (self.k + 1) & 0xFF
        self.buf.fill_(self.k)


class _Held:
    """A running ClockSampler shared by several measurements (summaries are
    taken after it stops)."""

    def __init__(self, cs):
        self.cs = cs

    def __enter__(self):
        return self.cs

    def __exit__(self, *exc):
        return False


def measure_product(g, torch, MC, MA, MB, m, l, n, o, steps, warmup, peaks, peak_kind, local_rank,
                    dist=None, rank=0, flush=None, sampler=None):
    """One product configuration through gf2_mul: a first call (the autotuner's
    choice for automatic options), `warmup` untimed calls, then `steps` calls
    timed with CUDA events on the current stream, with the library's per-kernel
    device-time accounting on, nvidia-smi clock samples around the timed region
    and Freivalds' check of the result.  With `flush`, L2 is flushed before
    every timed call and only the calls themselves are timed."""
    stream = torch.cuda.current_stream()
    g.gf2_mul(MC, MA, MB, o)
    torch.cuda.synchronize()
    with (ClockSampler(local_rank) if sampler is None else _Held(sampler)) as cs:
        for _ in range(warmup):
            g.gf2_mul(MC, MA, MB, o)
        torch.cuda.synchronize()
        plan = g.gf2_describe_plan(m, l, n, o)
        if dist is not None:
            dist.barrier()
        launches0 = g.gf2_launch_count()
        g.gf2_profile_enable(True)
        torch.cuda.synchronize()
        t_start = time.time()
        if flush is None:
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(steps):
                g.gf2_mul(MC, MA, MB, o)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms_total = ev0.elapsed_time(ev1)
        else:
            pairs = []
            for _ in range(steps):
                flush()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.gf2_mul(MC, MA, MB, o)
                e1.record(stream)
                pairs.append((e0, e1))
            torch.cuda.synchronize()
            ms_total = sum(a.elapsed_time(b) for a, b in pairs)
        t_end = time.time()
    launches = g.gf2_launch_count() - launches0
    fam = {}
    for i, name in enumerate(g.PROFILE_FAMILIES):
        t, c = g.gf2_profile_read(i)
        if c:
            fam[name] = {"ms": t, "launches": c}
    g.gf2_profile_enable(False)
    ms, _, value = aggregate(ms_total / steps, 2.0 * m * l * n)
    bad = g.gf2_freivalds(MC, MA, MB, 1000 + rank)
    kv = dict(x.split("=", 1) for x in plan.split() if "=" in x)
    d = int(kv["depth"])
    M, L, N = (int(x) for x in kv["leaf"].split("x"))
    leaves = int(kv["leaves"])
    k = int(kv.get("m4rm_k", 8))
    dom = max(fam.items(), key=lambda kvp: kvp[1]["ms"])[0] if fam else None
    dom_ms = fam[dom]["ms"] / max(fam[dom]["launches"], 1) if fam else 0.0
    # leaves per launch of the dominant kernel: all of them, or one group of
    # them when the leaf products are pipelined with the last level's additions
    dom_leaves = leaves * steps / fam[dom]["launches"] if fam and fam[dom]["launches"] else leaves
    rl = roofline_for(dom, dom_leaves, M, L, N, k, dom_ms, peaks, peak_kind) \
        if dom in BASE_FAMILIES else None
    hbm = {}
    Mp, Lp, Np = (int(x) for x in kv["padded"].split("x"))
    fused = kv.get("fused_expand") == "1"
    leaf_bpe = {"tc_fp4": 0.5, "tc_fp8": 1.0}.get(kv.get("base"), 0.125) if fused else 0.125
    sb, cb = strassen_stream_bytes(Mp, Lp, Np, d, leaf_bpe)
    eb = 0.0 if fused else expand_bytes(kv.get("base"), leaves, M, L, N)
    for fam_name, nbytes in (("sw_split", sb), ("sw_combine", cb), ("expand", eb)):
        if fam_name in fam and nbytes > 0:
            per_step_ms = fam[fam_name]["ms"] / steps
            gbs = nbytes / (per_step_ms * 1e-3) / 1e9
            hbm[fam_name] = {"bound": "hbm", "bytes_per_step": nbytes, "ms_per_step": per_step_ms,
                             "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": gbs / peaks["hbm_gbs"]}
    return {
        "ms": ms, "value": value, "depth": d, "plan": plan, "hbm_kernels": hbm,
        "gpu_launches": launches, "kernels": fam, "dominant": dom,
        "dominant_ms_per_launch": dom_ms, "roofline": rl, "steps": steps, "warmup": warmup,
        "l2": "flushed (256 MiB written) before every timed call" if flush is not None else
              "inputs and output exceed the 129 MB L2",
        "freivalds_mismatched_rows": bad,
        "clocks": cs.summary(t_start, t_end) if sampler is None else None, "timed_window": (t_start, t_end),
    }


BASE_FAMILIES = ("m4rm", "tc_fp8", "tc_fp4", "tc_s8", "tc_b1")


def expand_bytes(base, leaves, M, L, N):
    """Algorithmic HBM bytes of the expansion of the leaf operands for the
    tcgen05 base cases: the packed A and B^T leaves read once (M x L and
    N x L bits), the expanded rows written once (L rounded up to 128 FP8 or
    256 FP4 entries, one byte or half a byte per entry)."""
    if base not in ("tc_fp8", "tc_fp4"):
        return 0.0
    epr, eb = (128, 1.0) if base == "tc_fp8" else (256, 0.5)
    kp = -(-L // epr) * epr
    return leaves * ((M + N) * L / 8.0 + (M + N) * kp * eb)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_0811_1714_gb300 as g

    torch.cuda.set_device(local_rank)
    g.build()
    g.lib()
    n = l = m = args.n
    dist = None
    if world > 1:
        import torch.distributed as dist

    A = g.empty(m, l)
    B = g.empty(l, n)
    C = g.empty(m, n)
    MA, MB, MC = g.mat(A, l), g.mat(B, n), g.mat(C, n)
    g.gf2_random(MA, 1 + 100 * rank, args.p)
    g.gf2_random(MB, 2 + 100 * rank, args.p)
    torch.cuda.synchronize()
    peaks, peak_kind = load_peaks()

    avail = [p.strip() for p in args.paths.split(",") if p.strip()]
    # the warp-level mma.sync forms are ~30x slower than the others: they are
    # measured after the end-to-end run, so that it follows the headline
    # path's own measurement directly
    slow = [p for p in avail if p in ("tc_s8", "tc_b1")]
    fast = [p for p in avail if p not in slow]
    results = {}

    def measure(path):
        o = g.opts(base=BASE_OF[path](g), depth=args.depth, k=args.k if path == "m4rm" else 0,
                   t=args.t if path == "m4rm" else 0)
        small = (m * l + l * n) / 8 < L2_BYTES
        try:
            results[path] = measure_product(g, torch, MC, MA, MB, m, l, n, o, args.steps, args.warmup,
                                            peaks, peak_kind, local_rank, dist, rank,
                                            L2Flush(torch) if small else None)
            results[path].pop("timed_window", None)
        except g.GF2Error as e:
            results[path] = {"unavailable": str(e)}

    def best():
        ok = {p: r for p, r in results.items() if "ms" in r}
        return (min(ok, key=lambda p: ok[p]["ms"]), ok) if ok else (None, ok)

    for path in fast:
        measure(path)
    e2e_path, _ = best()
    e2e = None
    if not args.no_e2e and e2e_path is not None:
        # leave C holding that path's product for the comparison
        g.gf2_mul(MC, MA, MB, g.opts(base=BASE_OF[e2e_path](g), depth=args.depth))
        torch.cuda.synchronize()
        # start from freshly sized scratch (the arena the other paths grew
        # stays allocated otherwise, and slows the host-buffer path measurably)
        g.gf2_release_scratch()
        # the same product through the public C ABI on pinned HOST buffers:
        # H2D of A and B, the product, D2H of C, every step
        hA = A.cpu().pin_memory()
        hB = B.cpu().pin_memory()
        hC = torch.zeros_like(C, device="cpu").pin_memory()
        o = g.opts(base=BASE_OF[e2e_path](g), depth=args.depth)
        hMA, hMB, hMC = g.mat(hA, l), g.mat(hB, n), g.mat(hC, n)
        # the clock sampler starts before the warm-up, so that its start-up
        # (NVML initialisation in another process) is over before the timed
        # region, whose host-side time this measurement is
        with ClockSampler(local_rank) as cs:
            for _ in range(max(1, args.warmup)):
                g.gf2_mul(hMC, hMA, hMB, o)
            time.sleep(1.0)
            for _ in range(2):
                g.gf2_mul(hMC, hMA, hMB, o)
            if dist is not None:
                dist.barrier()
            w0 = time.time()                         # wall clock of the sampler's timestamps
            t0 = time.perf_counter()
            for _ in range(args.steps):
                g.gf2_mul(hMC, hMA, hMB, o)         # returns after the D2H copy completed
            t1 = time.perf_counter()
            w1 = time.time()
        t_e2e = (t1 - t0) / args.steps
        ms_e2e, _, v_e2e = aggregate(t_e2e * 1e3, 2.0 * m * l * n)
        same = bool(torch.equal(hC.cuda(), C))
        e2e = {"value": v_e2e, "unit": UNIT,
               "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": (hA.numel() + hB.numel()) * 8,
               "d2h_bytes_per_step": hC.numel() * 8, "matches_device_result": same,
               "base": e2e_path, "clocks": cs.summary(w0, w1)}
        del hA, hB, hC
    for path in slow:
        measure(path)
    head, ok = best()
    if head is None:
        raise SystemExit("no base case ran: %s" % results)
    H = ok[head]
    del A, B, C
    torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": H["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": H["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_OF[head],
        "data": "synthetic: SplitMix64 Bernoulli(%g) bits, seeds 1/2 (+100*rank)" % args.p,
        "config": {"workload": "square C=A*B over GF(2), m=l=n=%d" % n, "m": m, "l": l, "n": n, "p": args.p,
                   "base": head, "depth": H["depth"], "plan": H["plan"],
                   "parallelism": "independent product per GPU" if world > 1 else "single GPU",
                   "l2": H["l2"]},
        "roofline": H["roofline"], "gpu_launches": H["gpu_launches"],
        "clocks": H["clocks"], "e2e": e2e,
        "verified": {"freivalds_64_vectors_mismatched_rows": H["freivalds_mismatched_rows"]},
        "paths": {p: {kk: vv for kk, vv in r.items() if kk not in ("plan",)} for p, r in results.items()},
        "cpu_baseline": None,
    }
    return line


BASE_OF = {"m4rm": lambda g: g.GF2_BASE_M4RM, "tc_fp8": lambda g: g.GF2_BASE_TC_FP8,
           "tc_fp4": lambda g: g.GF2_BASE_TC_FP4,
           "tc_s8": lambda g: g.GF2_BASE_TC_S8, "tc_b1": lambda g: g.GF2_BASE_TC_B1,
           "auto": lambda g: g.GF2_BASE_AUTO}
DTYPE_OF = {"m4rm": "u64-packed-bits", "tc_fp8": "fp8e4m3-0/1", "tc_fp4": "fp4e2m1-0/1",
            "tc_s8": "s8-0/1", "tc_b1": "b1-packed-bits"}


def config_list(args):
    """The other configurations of the workload, measured after the headline
    by the default run: (name, m, l, n, p, path, options)."""
    return [
        ("config1_n1024_k8_depth0", 1024, 1024, 1024, 0.5, "m4rm", dict(depth=0, k=8)),
        ("config2_n16384", 16384, 16384, 16384, 0.5, "auto", dict()),
        ("config2_rect_20000x12000x28000", 20000, 12000, 28000, 0.5, "auto", dict()),
        ("config3_n65536_p0.5_m4rm", 65536, 65536, 65536, 0.5, "m4rm", dict()),
        ("config3_n65536_p0.9_m4rm", 65536, 65536, 65536, 0.9, "m4rm", dict()),
        ("config3_n65536_p0.5_tc_fp8", 65536, 65536, 65536, 0.5, "tc_fp8", dict()),
        ("config3_n65536_p0.9_tc_fp8", 65536, 65536, 65536, 0.9, "tc_fp8", dict()),
        ("config3_n65536_p0.5_tc_fp4", 65536, 65536, 65536, 0.5, "tc_fp4", dict()),
        ("config3_n65536_p0.9_tc_fp4", 65536, 65536, 65536, 0.9, "tc_fp4", dict()),
    ]


def run_configs(args, rank, world, local_rank):
    """Every configuration besides the headline: config 1, config 2's other
    shapes, config 3 at n = 65536 (p = 0.5 and 0.9, both base cases), the
    4096-product batch (config 4) and the chain (config 5).  Fewer steps than
    the headline (at most 10, at least 3 warm-up calls) keep the whole run
    within a few minutes; products whose inputs fit in L2 are timed with L2
    flushed before every call."""
    import torch
    import paper_0811_1714_gb300 as g

    peaks, peak_kind = load_peaks()
    steps = max(3, min(args.steps, 10))
    warmup = max(3, min(args.warmup, 3))
    flush = L2Flush(torch)
    out = {}
    cs = ClockSampler(local_rank)
    cs.__enter__()
    time.sleep(0.5)                      # nvidia-smi is sampling before the first timed region
    for name, m, l, n, p, path, kw in config_list(args):
        t0 = time.time()
        A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
        MA, MB, MC = g.mat(A, l), g.mat(B, n), g.mat(C, n)
        g.gf2_random(MA, 1 + 100 * rank, p)
        g.gf2_random(MB, 2 + 100 * rank, p)
        o = g.opts(base=BASE_OF[path](g), **kw)
        small = (m * l + l * n) / 8 < L2_BYTES
        try:
            r = measure_product(g, torch, MC, MA, MB, m, l, n, o, steps, warmup, peaks, peak_kind, local_rank,
                                None, rank, flush if small else None, sampler=cs)
            r.update({"m": m, "l": l, "n": n, "p": p, "path": path, "wall_s": time.time() - t0})
        except g.GF2Error as e:
            r = {"unavailable": str(e)}
        out[name] = r
        del A, B, C, MA, MB, MC
        torch.cuda.empty_cache()
    time.sleep(0.3)
    cs.__exit__(None, None, None)
    for r in out.values():
        if "timed_window" in r:
            r["clocks"] = cs.summary(*r.pop("timed_window"))
    del flush
    torch.cuda.empty_cache()
    t0 = time.time()
    bargs = argparse.Namespace(**vars(args))
    bargs.steps, bargs.warmup = steps, warmup
    out["config4_batched_4096"] = run_batched(bargs, rank, 1, local_rank)
    out["config4_batched_4096"]["wall_s"] = time.time() - t0
    torch.cuda.empty_cache()
    t0 = time.time()
    cargs = argparse.Namespace(**vars(args))
    cargs.steps, cargs.warmup = max(3, min(args.steps, 5)), warmup
    out["config5_chain"] = run_chain(cargs, rank, 1, local_rank)
    out["config5_chain"]["wall_s"] = time.time() - t0
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(n, target_s, seed_a=1, seed_b=2):
    """Time the CPU oracle on rows 0..r-1 of C for the n x n workload; r is
    chosen so that one sample takes about target_s seconds."""
    import oracle
    import synth
    B = synth.random_packed(n, n, seed_b)
    r = 2
    while True:
        A = synth.random_packed(r, n, seed_a)
        t0 = time.perf_counter()
        oracle.mul_packed(A, B, r, n, n)
        dt = time.perf_counter() - t0
        if dt >= target_s or r >= n:
            return r, dt
        r = min(n, max(r * 2, int(r * target_s / max(dt, 1e-3) * 0.9)))


def cpu_baseline(n, target_s):
    import oracle
    r, dt = oracle_sample(n, target_s)
    return {"value": 2.0 * r * n * n / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "rows 0..%d of C = A B at n=%d (naive cubic on unpacked bytes, "
                      "unpacking included), %.1f s" % (r - 1, n, dt)}


def run_reference(args):
    """The CPU oracle timed on the host cores: each step one bounded sample."""
    import oracle
    import synth
    n = args.n
    # each step is one bounded sample: the whole warm-up + timed run stays
    # near 100 s of CPU work whatever --steps and --warmup are
    per_step = max(1.0, min(args.cpu_seconds, 20.0, 100.0 / max(1, args.steps + args.warmup)))
    r, _ = oracle_sample(n, per_step)
    B = synth.random_packed(n, n, 2)
    A = synth.random_packed(r, n, 1)
    for _ in range(args.warmup):
        oracle.mul_packed(A, B, r, n, n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.mul_packed(A, B, r, n, n)
    dt = (time.perf_counter() - t0) / args.steps
    v = 2.0 * r * n * n / dt
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8-unpacked",
        "data": "synthetic: SplitMix64 Bernoulli(1/2) bits, seeds 1/2",
        "config": {"workload": "square C=A*B over GF(2), m=l=n=%d" % n, "m": n, "l": n, "n": n,
                   "sample_rows": r},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "rows 0..%d of C per step (naive cubic oracle)" % (r - 1)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def batched_table_bytes(vname, dims):
    """Algorithmic table-row reads of a batched variant: m*l*n / (8k) bytes
    per product for k-bit tables.  A split variant "tall-k8t4-bm<b>-from<r>+
    slots-k<k>t<t>-..." runs each product's full b-row blocks, and its last
    block when that keeps at least r rows, with k = 8 and the other rows with
    the slot kernel's k."""
    import re
    if "+" in vname:
        tb = int(re.search(r"^tall-k\d+t\d+-bm(\d+)-from", vname).group(1))
        split = int(re.search(r"-from(\d+)\+", vname).group(1))
        k_rest = int(re.search(r"\+slots-k(\d+)t", vname).group(1))
        total = 0.0
        for m, l, n in dims:
            full = m // tb * tb
            tall = m if m - full >= split else full
            total += tall * l * n / 64.0 + (m - tall) * l * n / (8.0 * k_rest)
        return total, "k=8 on the tall row blocks (%d-row blocks, the last one from %d rows), k=%d on the rest" % (
            tb, split, k_rest)
    k = int(re.search(r"k(\d+)t", vname).group(1))
    return sum(m * l * n for m, l, n in dims) / (8.0 * k), "k=%d tables" % k


def run_batched(args, rank, world, local_rank):
    """4096 independent products, m, l, n log-uniform in [64, 2048] (seeded),
    one persistent launch replayed as a CUDA graph (autotuned variant)."""
    import torch
    import paper_0811_1714_gb300 as g
    import synth

    torch.cuda.set_device(local_rank)
    g.build()
    dims = synth.batch_dims(4096)
    MA, MB, MC, keep = [], [], [], []
    for i, (m, l, n) in enumerate(dims):
        A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
        MA.append(g.mat(A, l)); MB.append(g.mat(B, n)); MC.append(g.mat(C, n))
        g.gf2_random(MA[-1], 10_000 + 2 * i + 100_000 * rank)
        g.gf2_random(MB[-1], 10_001 + 2 * i + 100_000 * rank)
        keep.append((A, B, C))
    arrs = g.MatArrays(MC, MA, MB)
    ops = sum(2.0 * m * l * n for m, l, n in dims)
    variant = g.gf2_mul_batched_ex(arrs)          # first call: autotune + graph build
    stream = torch.cuda.current_stream()

    clocks = {}

    def timed(options, tag):
        g.gf2_mul_batched(arrs, options=options)      # first call for these options: tuning, graph
        with ClockSampler(local_rank) as cs:
            for _ in range(args.warmup):
                g.gf2_mul_batched(arrs, options=options)
            launches0 = g.gf2_launch_count()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.time()
            ev0.record(stream)
            for _ in range(args.steps):
                g.gf2_mul_batched(arrs, options=options)
            ev1.record(stream)
            torch.cuda.synchronize()
            t1 = time.time()
        clocks[tag] = cs.summary(t0, t1)
        return ev0.elapsed_time(ev1) / args.steps, g.gf2_launch_count() - launches0

    def sampled_bad(seed0):
        return sum(1 for i in range(0, len(dims), 64) if g.gf2_freivalds(MC[i], MA[i], MB[i], seed0 + i))

    g.gf2_profile_enable(True)
    ms_local, launches = timed(None, "m4rm")
    k_ms, k_n = g.gf2_profile_read(g.PROFILE_FAMILIES.index("batched"))
    g.gf2_profile_enable(False)
    bad = sampled_bad(5)
    peaks, peak_kind = load_peaks()
    vname = g.gf2_batched_variant_name(variant)
    rl = None
    if k_n:
        per_launch_ms = k_ms / k_n
        smem_bytes, note_k = batched_table_bytes(vname, dims)
        achieved = smem_bytes / (per_launch_ms * 1e-3) / 1e9
        peak, note = smem_peak(peaks)
        rl = {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
              "traffic": None, "kernel_ms_per_launch": per_launch_ms,
              "peak_note": note,
              "work_note": "table-row reads, sum of m*l*n/(8k) over the 4096 products (%s); "
                           "time of the whole graph" % note_k}
    ms, ops_all, value = aggregate(ms_local, ops)
    # the same batch on the tcgen05 base cases: one batched transpose, one
    # batched expansion and one persistent tensor-core launch per step
    tcs = {}
    for tname, tbase, ratio in (("tc_fp4", g.GF2_BASE_TC_FP4, 6.0), ("tc_fp8", g.GF2_BASE_TC_FP8, 2.0)):
        g.gf2_profile_enable(True)
        tc_ms_local, tc_launches = timed(g.opts(base=tbase, depth=0), tname)
        t_ms, t_n = g.gf2_profile_read(g.PROFILE_FAMILIES.index(tname))
        g.gf2_profile_enable(False)
        tc_ms, _, tc_value = aggregate(tc_ms_local, ops)
        tc_rl = None
        if t_n:
            flops = sum(2.0 * m * l * n for m, l, n in dims)
            ach = flops / (t_ms / t_n * 1e-3) / 1e12
            pk = ratio * peaks["bf16_tflops"]
            tc_rl = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                     "traffic": None, "kernel_ms_per_launch": t_ms / t_n,
                     "peak_note": "%g x bf16 burst of %s peaks (nominal ratio)" % (ratio, peak_kind),
                     "work_note": "2 m l n of the 4096 products over the time of the whole graph "
                                  "(expansion of A, transposed expansion of B, MMA kernel; tiles of "
                                  "128 x 256 entries of C pad small products)"}
        tcs[tname] = {"ms_per_step": tc_ms, "value": tc_value, "gpu_launches": tc_launches, "roofline": tc_rl,
                      "clocks": clocks.get(tname),
                      "graph": "batched expansion of every A and transposed expansion of every B + one "
                               "persistent tensor-core kernel",
                      "freivalds_sampled_products_failed": sampled_bad(9)}
    ops = ops_all
    return {
        "metric": "effective GF(2) bit-ops/s (2mnk/t), 4096 batched products", "value": value,
        "unit": "bit-ops/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64-packed-bits", "data": "synthetic: SplitMix64 bits, dims log-uniform [64, 2048] seed 42",
        "config": {"workload": "4096 batched products, m,l,n log-uniform in [64, 2048]",
                   "variant": g.gf2_batched_variant_name(variant), "total_bit_ops": ops},
        "gpu_launches": launches, "roofline": rl, "clocks": clocks.get("m4rm"),
        "l2": "operands of all products (about 0.5 GB) exceed the 129 MB L2",
        "graph": "each step replays one CUDA graph: counter reset + one persistent kernel (two for a split variant)",
        "verified": {"freivalds_sampled_products_failed": bad},
        "tensor_core_bases": tcs,
    }


def run_chain(args, rank, world, local_rank):
    """A (131072 x 65536) . B (65536 x 131072), then . C (131072 x 8192)."""
    import torch
    import paper_0811_1714_gb300 as g

    torch.cuda.set_device(local_rank)
    g.build()
    M, K1, N1, N2 = 131072, 65536, 131072, 8192
    A, B, AB = g.empty(M, K1), g.empty(K1, N1), g.empty(M, N1)
    C, ABC = g.empty(N1, N2), g.empty(M, N2)
    MA, MB, MAB, MC, MABC = g.mat(A, K1), g.mat(B, N1), g.mat(AB, N1), g.mat(C, N2), g.mat(ABC, N2)
    g.gf2_random(MA, 31 + 100 * rank)
    g.gf2_random(MB, 32 + 100 * rank)
    g.gf2_random(MC, 33 + 100 * rank)
    for _ in range(max(1, args.warmup)):
        g.gf2_mul(MAB, MA, MB)
        g.gf2_mul(MABC, MAB, MC)
    plans = [g.gf2_describe_plan(M, K1, N1), g.gf2_describe_plan(M, N1, N2)]
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    t1 = t2 = 0.0
    launches0 = g.gf2_launch_count()
    g.gf2_profile_enable(True)
    with ClockSampler(local_rank) as cs:
        ts0 = time.time()
        for _ in range(args.steps):
            ev[0].record(stream)
            g.gf2_mul(MAB, MA, MB)
            ev[1].record(stream)
            g.gf2_mul(MABC, MAB, MC)
            ev[2].record(stream)
            torch.cuda.synchronize()
            t1 += ev[0].elapsed_time(ev[1])
            t2 += ev[1].elapsed_time(ev[2])
        ts1 = time.time()
    launches = g.gf2_launch_count() - launches0
    fam = {}
    for i, name in enumerate(g.PROFILE_FAMILIES):
        t, c = g.gf2_profile_read(i)
        if c:
            fam[name] = {"ms_per_step": t / args.steps, "launches_per_step": c / args.steps}
    g.gf2_profile_enable(False)
    t1 /= args.steps
    t2 /= args.steps
    ops1, ops2 = 2.0 * M * K1 * N1, 2.0 * M * N1 * N2
    ok = (g.gf2_freivalds(MAB, MA, MB, 1000) == 0) and (g.gf2_freivalds(MABC, MAB, MC, 1001) == 0)
    _, _, value = aggregate(t1 + t2, ops1 + ops2)
    return {
        "metric": "effective GF(2) bit-ops/s (2mnk/t), chain A.B then .C", "value": value,
        "unit": "bit-ops/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t1 + t2, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "auto", "data": "synthetic: SplitMix64 Bernoulli(1/2) bits, seeds 31/32/33",
        "config": {"workload": "chain 131072x65536 . 65536x131072 . 131072x8192", "plans": plans,
                   "stage_ms": [t1, t2],
                   "l2": "operands (1 GiB and more each) exceed the 129 MB L2"},
        "gpu_launches": launches, "kernels": fam, "clocks": cs.summary(ts0, ts1),
        "verified": {"freivalds_both_stages": ok},
    }


def run_sharded(args, rank, world, local_rank):
    """One n x n product with the rows of A and C split over the ranks and B
    broadcast from rank 0 once per step (Section 3: C's rows are A's rows
    times B, so no reduction).  Timed per step: the broadcast of B and every
    rank's product of its rows; the stitching of C on rank 0 runs once
    afterwards and is checked by Freivalds' test on every block."""
    import torch
    import paper_0811_1714_gb300 as g
    from paper_0811_1714_gb300.sharded import gf2_mul_sharded, row_blocks

    torch.cuda.set_device(local_rank)
    g.build()
    n = args.n
    r0, r1 = row_blocks(n, world)[rank]
    rows = r1 - r0
    A = g.empty(rows, n)
    B = g.empty(n, n)
    if rows:
        g.gf2_random(g.mat(A, n), 1 + 100 * rank)
    if rank == 0:
        g.gf2_random(g.mat(B, n), 2)
    o = g.opts(base=BASE_OF[args.paths.split(",")[0]](g) if args.paths != DEFAULT_PATHS else g.GF2_BASE_AUTO,
               depth=args.depth)
    group = None
    import torch.distributed as dist
    for _ in range(max(3, args.warmup)):
        C_local, _ = gf2_mul_sharded(A, B, n, n, options=o, gather=False)
    torch.cuda.synchronize()
    dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as cs:
        t0 = time.time()
        e0.record(stream)
        for _ in range(args.steps):
            C_local, _ = gf2_mul_sharded(A, B, n, n, options=o, gather=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t1 = time.time()
    ms, ops, value = aggregate(e0.elapsed_time(e1) / args.steps, 2.0 * rows * n * n)
    bad = g.gf2_freivalds(g.mat(C_local, n), g.mat(A, n), g.mat(B, n), 1000 + rank) if rows else 0
    bad_t = torch.tensor([float(bad)], device="cuda")
    dist.all_reduce(bad_t)
    _, C = gf2_mul_sharded(A, B, n, n, options=o, gather=True)
    return {
        "metric": "effective GF(2) bit-ops/s (2mnk/t), one product sharded by rows", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "auto", "data": "synthetic: SplitMix64 bits, B seed 2, row blocks of A seeds 1+100*rank",
        "config": {"workload": "square C=A*B over GF(2), m=l=n=%d, rows of A and C split over %d ranks, "
                               "B broadcast once per step" % (n, world),
                   "rows_per_rank": [b1 - b0 for b0, b1 in row_blocks(n, world)],
                   "plan_rank0": g.gf2_describe_plan(rows, n, n, o) if rows else None},
        "clocks": cs.summary(t0, t1),
        "verified": {"freivalds_mismatched_rows_all_ranks": int(bad_t.item()),
                     "stitched_rows": int(C.shape[0]) if C is not None else None},
    }


def run_sweep(args, rank, world, local_rank):
    """Packed M4RM over Strassen-Winograd depth (the cutoff) x k (bits per
    table; t automatic) on the square 8192, 16384 and 32768 products and on
    20000x12000 . 12000x28000.  Every point is timed by CUDA events (one
    warm-up, `steps` timed calls) and Freivalds-checked."""
    import torch
    import paper_0811_1714_gb300 as g

    torch.cuda.set_device(local_rank)
    g.build()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    shapes = [(8192, 8192, 8192), (16384, 16384, 16384), (32768, 32768, 32768), (20000, 12000, 28000)]
    ks = [4, 5, 6, 7, 8, 9, 10]
    points, failed = [], 0
    for (m, l, n) in shapes:
        A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
        MA, MB, MC = g.mat(A, l), g.mat(B, n), g.mat(C, n)
        g.gf2_random(MA, 1 + 100 * rank)
        g.gf2_random(MB, 2 + 100 * rank)
        depth = 0
        while min(m, l, n) >> depth >= 1024:
            for k in ks:
                o = g.opts(base=g.GF2_BASE_M4RM, depth=depth, k=k, peel=0)
                g.gf2_mul(MC, MA, MB, o)
                torch.cuda.synchronize()
                ev[0].record(stream)
                for _ in range(max(1, args.steps)):
                    g.gf2_mul(MC, MA, MB, o)
                ev[1].record(stream)
                torch.cuda.synchronize()
                ms = ev[0].elapsed_time(ev[1]) / max(1, args.steps)
                ok = g.gf2_freivalds(MC, MA, MB, 4242) == 0
                failed += 0 if ok else 1
                points.append({"m": m, "l": l, "n": n, "depth": depth, "k": k, "ms": ms,
                               "bit_ops_per_s": 2.0 * m * l * n / (ms * 1e-3), "freivalds_ok": ok,
                               "plan": g.gf2_describe_plan(m, l, n, o)})
            depth += 1
        del A, B, C
        torch.cuda.empty_cache()
    best = max((p for p in points if p["n"] == 32768 and p["m"] == 32768), key=lambda p: p["bit_ops_per_s"])
    return {
        "metric": "effective GF(2) bit-ops/s (2mnk/t), packed M4RM over depth x k", "value": best["bit_ops_per_s"],
        "unit": "bit-ops/s", "n_gpus": world, "steps": args.steps, "warmup": 1,
        "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64-packed-bits", "data": "synthetic: SplitMix64 Bernoulli(1/2) bits, seeds 1/2",
        "config": {"workload": "sweep of Strassen-Winograd depth x M4RM k", "best_at_32768": best},
        "sweep": points, "verified": {"freivalds_failures": failed},
    }


def run_peaks(args, rank, world, local_rank):
    """The throughput probes behind the peaks that MEASURED_PEAKS.json does
    not hold (shared-memory lookups, L2, mma.sync, tcgen05 MMA-only), run as
    the package's probe executable, with the clocks sampled around it."""
    import subprocess
    import paper_0811_1714_gb300 as g
    from paper_0811_1714_gb300 import buildlib
    g.build()
    exe = buildlib.probe_path("peaks")
    with ClockSampler(local_rank) as cs:
        t0 = time.time()
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
        t1 = time.time()
    if r.returncode != 0:
        raise RuntimeError("peak probes failed (%d): %s %s" % (r.returncode, r.stdout[-2000:], r.stderr[-2000:]))
    probes = json.loads(r.stdout.strip().splitlines()[-1])
    return {"workload": "peaks", "probes": probes, "clocks": cs.summary(t0, t1),
            "note": "CUDA-event time of the second of two identical launches per probe"}


def emit(line):
    """Print the JSON line as the last line of stdout: output that native
    libraries buffered in C stdio (NCCL prints its version there) is
    flushed first, so it cannot follow the line at exit."""
    try:
        import ctypes
        ctypes.CDLL(None).fflush(None)
    except (OSError, AttributeError):
        pass
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            emit(run_reference(args))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == "sharded" and world == 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % int(os.environ.get("MASTER_PORT", "29533")),
                                rank=0, world_size=1)
    def finish(line):
        # the process group (and whatever its library prints on the way out)
        # is closed before rank 0 prints the one JSON line
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            dist.barrier()
            dist.destroy_process_group()
        if rank == 0:
            emit(line)

    if args.workload in ("batched", "chain", "sweep", "sharded", "peaks"):
        run = {"batched": run_batched, "chain": run_chain, "sweep": run_sweep, "sharded": run_sharded,
               "peaks": run_peaks}[args.workload]
        finish(run(args, rank, world, local_rank))
        return
    line = run_ours(args, rank, world, local_rank)
    if world == 1 and not args.no_configs:
        line["configs"] = run_configs(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.n, args.cpu_seconds)
    finish(line)


if __name__ == "__main__":
    main()
