#!/usr/bin/env python3
"""Benchmark: batched FP64 panel-major routines on one GB300 (or N, as replicas).

Workload (one "step"): the FP64 routine sweep -- dgemm_nt, dsyrk_ln, dpotrf_l,
dtrsm_rltn and the fused dsyrk_dpotrf_ln at square n in
{4, 8, 16, 24, 32, 48, 64, 96, 128, 192, 256}, k = n, each point with a batch
sized so that its inputs fill about 1 GiB of HBM (far larger than the 129 MB
L2, so no L2 flush is needed between steps).  Entries iid N(0, 1); SPD
inputs M M^T + n I; the trsm factor is the Cholesky factor of such an input;
syrk_potrf computes chol(n I + M M^T).  All data synthetic and seeded.

Metric: GFLOP/s of the whole step (sum of the routines' flop counts over the
step time), with per-point GFLOP/s and roofline fraction.  Flop counts:
gemm 2mnk, syrk k m(m+1), potrf n^3/3 + n^2/2 + n/6, trsm m n^2,
syrk_potrf = syrk + potrf.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(independent problems, no collective: replicas, weak scaling); rank 0 prints
one JSON line.  --impl reference times the CPU oracle on a bounded sample.
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

SWEEP_N = (4, 8, 16, 24, 32, 48, 64, 96, 128, 192, 256)
# (m, n, k) of a sweep point at order n, as bf_layout_get takes them
SIZES = {"dgemm_nt": lambda n: (n, n, n), "dsyrk_ln": lambda n: (n, 0, n), "dpotrf_l": lambda n: (n, 0, 0),
         "dtrsm_rltn": lambda n: (n, n, 0), "dsyrk_dpotrf_ln": lambda n: (n, 0, n)}
ROUTINES = ("dgemm_nt", "dsyrk_ln", "dpotrf_l", "dtrsm_rltn", "dsyrk_dpotrf_ln")

# FP64 ALU peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA
# lanes per SM and clock x 2 flop x 2.07 GHz.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070


def flops(routine: str, n: int) -> float:
    m = k = n
    if routine == "dgemm_nt":
        return 2.0 * m * n * k
    if routine == "dsyrk_ln":
        return float(k * m * (m + 1))
    if routine == "dpotrf_l":
        return n ** 3 / 3.0 + n ** 2 / 2.0 + n / 6.0
    if routine == "dtrsm_rltn":
        return float(m * n * n)
    if routine == "dsyrk_dpotrf_ln":
        return float(k * m * (m + 1)) + n ** 3 / 3.0 + n ** 2 / 2.0 + n / 6.0
    raise ValueError(routine)


def alg_bytes(routine: str, n: int) -> float:
    """Bytes the method must move per problem: inputs read once, output written
    once, triangles only for symmetric/triangular operands."""
    m = k = n
    if routine == "dgemm_nt":
        return 8.0 * (m * k + n * k + 2 * m * n)
    if routine == "dsyrk_ln":
        return 8.0 * (2 * m * k + m * (m + 1))
    if routine == "dpotrf_l":
        return 8.0 * n * (n + 1)
    if routine == "dtrsm_rltn":
        return 8.0 * (n * (n + 1) / 2 + 2 * m * n)
    if routine == "dsyrk_dpotrf_ln":
        return 8.0 * (2 * n * k + n * (n + 1))
    raise ValueError(routine)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def roofline_gflops(routine, n, hbm_gbs):
    return min(FP64_PEAK_GFLOPS, hbm_gbs * flops(routine, n) / alg_bytes(routine, n))


# ncu measurements of DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum)
# per launch, keyed by kernel and sweep point, with the git blob hash of the
# kernel's source file when the counters were taken: the bench reports the
# traffic only while that file is unchanged.
TRAFFIC = {
    ("k_gemm_nt<0,1,1>", "dgemm_nt", 256): {
        "bytes": 1076203776 + 334554880,
        "src": "paper_1704_02457_gb300/csrc/bf_gemm.cu",
        "blob": "832d67af2617fb7fd4a53f8274acb08d6ac53bb9",
        "profile": "profiles/k_gemm_nt_n256.md",
    },
}


def _git_blob_hash(path):
    import hashlib
    try:
        data = open(os.path.join(ROOT, path), "rb").read()
    except OSError:
        return None
    return hashlib.sha1(b"blob %d\0" % len(data) + data).hexdigest()


def small_g(n):
    """Lanes per problem the small Cholesky kernel uses at order n (at least 2:
    one lane per problem is the register kernel's, up to n = 8)."""
    ne = n * (n + 1) // 2
    g = 2
    while g <= 16:
        if ne * (32 // g) * 8 <= 26 * 1024:
            return g
        g *= 2
    return 16 if ne * 2 * 8 <= 48 * 1024 else 0


def potrf_block_layout(h, batch, sms=152):
    """The layout the library's rule picks for a diagonal block of order h of
    the blocked Cholesky (the non-fused rule for the block's order and the
    batch): "blocked" again for a large block, "rows8", "latency", or None
    for the order's default kernel."""
    if h <= 32 and batch <= 4 * sms:
        return "latency"
    if 21 <= h <= 56 and batch >= 32 * sms:
        return "rows8"
    if h >= 128 and batch >= 2 * sms:
        return "blocked"
    return None


def kernel_of(routine, n, layout=None, batch=None, sms=152):
    """Name of the kernel the library launches for (routine, n) at this sweep
    in `layout` (a tune.LAYOUT_NAMES name; None: the row kernels of the
    Cholesky, the built-in choice of the other routines).  Layouts made of
    several launches are named by their parts; with `batch` given, the
    blocked layout's diagonal blocks are named by the layout the rule picks
    for them."""
    fused = int(routine == "dsyrk_dpotrf_ln")
    if layout in ("ks2", "ks4"):
        return f"k_gemm_nt<{int(routine == 'dsyrk_ln')},1,1>/{layout}"
    if layout and layout.startswith("latency"):
        if routine == "dtrsm_rltn":
            return f"k_trsm_lat<{max(8, (n + 7) // 8 * 8)},{layout[-1]}>"
        return f"k_chol_lat<{fused},{max(8, (n + 7) // 8 * 8)}>"
    if layout and layout.startswith("small_g"):
        return f"k_chol_small<{layout[7:]},{fused},1>"
    if layout == "tiny":
        return f"k_chol_tiny<{n},{fused},1>"
    if layout == "rows8":
        t, b = (256, 4) if n <= 32 else ((384, 3) if n <= 48 else (512, 2))
        return f"k_chol_rows8<{fused},1,double,{t},{b}>"
    if layout == "split":
        return ("k_gemm_nt<1,1,1>+" if fused else "") + kernel_of("dpotrf_l", n, "rows")
    if layout == "blocked":
        h = (n // 2) & ~3

        def block(o):
            if batch is None:
                return kernel_of("dpotrf_l", o, "rows")
            return kernel_of("dpotrf_l", o, potrf_block_layout(o, batch, sms), batch, sms)
        return (("k_gemm_nt<1,1,1>+" if fused else "") + "blocked[" + block(h) + "+" +
                kernel_of("dtrsm_rltn", h) + "+k_gemm_nt<1,1,1>+" + block(n - h) + "]")
    if routine == "dgemm_nt":
        return "k_gemm_nt<0,1,1>"
    if routine == "dsyrk_ln":
        return "k_gemm_nt<1,1,1>"
    if routine == "dtrsm_rltn":
        if n <= 32:
            return f"k_trsm_rltn_w<{4 if n <= 4 else (n + 7) // 8 * 8}>"
        return "k_trsm_rltn"
    if n <= 8 and layout is None:  # the sweep's batches give one lane per problem
        return f"k_chol_tiny<{n},{fused},1>"
    if n <= 31 and small_g(n) and not (fused and n >= 24 and n % 8 == 0) and layout is None:
        return f"k_chol_small<{small_g(n)},{fused},1>"
    if n <= 64:
        return f"k_chol_rows4<{fused},1,double,256,4>"
    if n <= 96:
        return f"k_chol_rows4<{fused},1,double,384,3>"
    if n <= 128:
        return f"k_chol_rows2<16,{fused},1,double,256,4>"
    if n <= 192:
        return f"k_chol_rows2<16,{fused},1,double,384,3>"
    if n <= 256:
        return f"k_chol_rows2<16,{fused},1,double,512,2>"
    return f"k_chol_rows<16,{fused},1,double>"


def launches_of(routine, n, batch, sms=152, layout=None):
    """Kernel launches of one call at this sweep.  The Cholesky of orders
    193..256 splits a batch whose last wave of two-problem CTAs (two per SM)
    holds more pairs than SMs but at most 80% of its slots: the pairs of the
    full waves, then the rest one problem per CTA.  The split layout adds
    the syrk launch; the blocked layout is potrf, trsm, syrk, potrf and the
    launch that rebuilds info from the diagonal (plus the syrk of the fused
    routine's sum)."""
    fused = routine == "dsyrk_dpotrf_ln"
    if layout == "split":
        return int(fused) + launches_of("dpotrf_l", n, batch, sms)
    if layout == "blocked":
        # each diagonal block in the layout the rule picks for its order (a
        # nested blocked block adds no info launch of its own)
        h = (n // 2) & ~3

        def block(o):
            lay = potrf_block_layout(o, batch, sms)
            return launches_of("dpotrf_l", o, batch, sms, lay) - (lay == "blocked")
        return int(fused) + block(h) + 2 + block(n - h) + 1
    if routine in ("dpotrf_l", "dsyrk_dpotrf_ln") and 192 < n <= 256:
        slots, pairs = 2 * sms, (batch + 1) // 2
        rest = pairs % slots
        if pairs > slots and sms < rest and rest * 100 <= slots * 80:
            return 2
    return 1


WORKLOAD = ("FP64 routine sweep: dgemm_nt, dsyrk_ln, dpotrf_l, dtrsm_rltn, dsyrk_dpotrf_ln "
            "at square n in {4,8,16,24,32,48,64,96,128,192,256}, k=n, batch sized so the "
            "inputs of each point fill ~1 GiB; iid N(0,1), SPD inputs M M^T + n I")


def config_dict(points):
    return {
        "workload": WORKLOAD,
        "routines": list(ROUTINES),
        "n": sorted({n for _, n in points}),
        "batch_per_point_inputs_bytes": 1 << 30,
        "layout": "panel-major, ps=4",
        "l2": "inputs larger than L2 (1 GiB per point), no flush",
    }


# ------------------------------------------------------------- multi-rank --

def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(flops_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job GFLOP/s: every rank runs the same workload on its own GPU
    (independent problems, weak scaling), timed by the slowest rank."""
    return flops_per_rank * world / seconds / 1e9


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons),
            "samples": len(sm),
        }


# --------------------------------------------------------------- GPU arm ---

class Point:
    """One (routine, n) sweep point: resident panel-major inputs and outputs."""

    def __init__(self, routine, n, dev, seed, batch=None):
        import torch

        import paper_1704_02457_gb300 as bf
        from paper_1704_02457_gb300 import inputs

        self.routine, self.n = routine, n
        self.batch = bt = inputs.sweep_batch(routine, n) if batch is None else batch
        self.flops = flops(routine, n) * bt
        self.roof = None
        mk = lambda X: bf.DMatBatch.from_colmajor(X, tight=True)  # noqa: E731
        if routine == "dgemm_nt":
            self.A = mk(inputs.normal((bt, n, n), seed, dev))
            self.B = mk(inputs.normal((bt, n, n), seed + 1, dev))
            self.C = mk(inputs.normal((bt, n, n), seed + 2, dev))
            self.D = bf.DMatBatch(bt, n, n, tight=True)
        elif routine == "dsyrk_ln":
            self.A = mk(inputs.normal((bt, n, n), seed, dev))
            self.C = mk(inputs.normal((bt, n, n), seed + 2, dev))
            self.D = bf.DMatBatch(bt, n, n, tight=True)
        elif routine == "dpotrf_l":
            self.C = mk(inputs.spd(bt, n, seed, dev))
            self.D = bf.DMatBatch(bt, n, n, tight=True)
            self.info = torch.zeros(bt, dtype=torch.int32, device=dev)
        elif routine == "dtrsm_rltn":
            # the factor of an SPD input, computed (untimed) by this library's potrf
            S = mk(inputs.spd(bt, n, seed, dev))
            self.L = bf.DMatBatch(bt, n, n, tight=True, fill=0.0)
            bf.dpotrf_l(n, S, 0, 0, self.L, 0, 0, dinv=False)
            del S
            self.B = mk(inputs.normal((bt, n, n), seed + 1, dev))
            self.D = bf.DMatBatch(bt, n, n, tight=True)
        elif routine == "dsyrk_dpotrf_ln":
            self.A = mk(inputs.normal((bt, n, n), seed, dev))
            Q = torch.zeros(bt, n, n, dtype=torch.float64, device=dev)
            Q.diagonal(dim1=1, dim2=2).fill_(float(n))
            self.C = mk(Q)
            del Q
            self.D = bf.DMatBatch(bt, n, n, tight=True)
            self.info = torch.zeros(bt, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()

    def run(self, stream=None):
        import paper_1704_02457_gb300 as bf
        n = self.n
        r = self.routine
        if r == "dgemm_nt":
            bf.dgemm_nt(n, n, n, 1.0, self.A, 0, 0, self.B, 0, 0, 1.0, self.C, 0, 0, self.D, 0, 0, stream=stream)
        elif r == "dsyrk_ln":
            bf.dsyrk_ln(n, n, 1.0, self.A, 0, 0, self.A, 0, 0, 1.0, self.C, 0, 0, self.D, 0, 0, stream=stream)
        elif r == "dpotrf_l":
            bf.dpotrf_l(n, self.C, 0, 0, self.D, 0, 0, dinv=False, info=self.info, stream=stream)
        elif r == "dtrsm_rltn":
            bf.dtrsm_rltn(n, n, 1.0, self.L, 0, 0, self.B, 0, 0, self.D, 0, 0, stream=stream)
        elif r == "dsyrk_dpotrf_ln":
            bf.dsyrk_dpotrf_ln(n, n, self.A, 0, 0, self.A, 0, 0, self.C, 0, 0, self.D, 0, 0, dinv=False,
                               info=self.info, stream=stream)


class OracleSampler:
    """The CPU oracle timed on a bounded sample of every sweep point.

    Calibration picks, per point, a sample of problems that takes about
    budget_s seconds (at most the point's full batch) and keeps its inputs;
    each timed pass then runs the oracle on those cached inputs and returns
    GFLOP/s per point.  The oracle runs its problems on every host core
    (OpenMP)."""

    def __init__(self, points_spec, budget_s=0.25):
        import oracle
        from paper_1704_02457_gb300 import inputs

        oracle.build()
        self.spec = list(points_spec)
        self.cores = oracle.num_threads()
        self.cache = {}
        for routine, n in self.spec:
            full = inputs.sweep_batch(routine, n)
            # probe with ~20 MFLOP, then size the sample to the budget
            count = max(1, min(full, int(2e7 / max(flops(routine, n), 1.0))))
            data = _oracle_inputs(routine, n, count)
            t = _oracle_time(routine, n, data)
            if t < 0.5 * budget_s and count < full:
                count = min(full, int(count * min(256.0, budget_s / max(t, 1e-6))) + 1)
                data = _oracle_inputs(routine, n, count)
            self.cache[(routine, n)] = (count, data)

    def rates(self):
        out = {}
        for (routine, n), (count, data) in self.cache.items():
            out[(routine, n)] = flops(routine, n) * count / _oracle_time(routine, n, data) / 1e9
        return out

    def describe(self):
        first = ", ".join(f"{r}@{n}:{self.cache[(r, n)][0]}" for r, n in self.spec[:3])
        return ("oracle (plain C loops, -O2 -ffp-contract=off, OpenMP over problems) on a bounded sample "
                f"of problems per point ({first}, ...); step time = sum over points of full-batch "
                "flops / sample rate")


def _oracle_inputs(routine, n, count):
    """Sample inputs, already in the oracle's column-major layout, with output
    buffers: the timed call runs the C routine only."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(7 + n)
    A = rng.standard_normal((count, n, n))
    cm = oracle._colmajor
    if routine == "dpotrf_l":
        ins = (cm(A @ A.transpose(0, 2, 1) + n * np.eye(n)),)
    elif routine == "dtrsm_rltn":
        ins = (cm(np.linalg.cholesky(A @ A.transpose(0, 2, 1) + n * np.eye(n))), cm(rng.standard_normal((count, n, n))))
    elif routine == "dsyrk_dpotrf_ln":
        ins = (cm(A), cm(np.broadcast_to(n * np.eye(n), (count, n, n))))
    else:
        ins = (cm(A), cm(rng.standard_normal((count, n, n))), cm(rng.standard_normal((count, n, n))))
    out = np.zeros((count, n, n))
    return ins + (out, np.zeros((count, n)), np.zeros(count, dtype=np.int32), count)


def _oracle_time(routine, n, data):
    import ctypes

    import oracle
    lib, P = oracle._lib(), oracle._ptr
    *ins, out, dinv, info, bt = data
    nn = n * n
    ip = info.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    t0 = time.perf_counter()
    if routine == "dpotrf_l":
        lib.or_dpotrf_l_batch(bt, n, P(ins[0]), n, nn, P(out), n, nn, P(dinv), n, ip)
    elif routine == "dtrsm_rltn":
        lib.or_dtrsm_rltn_batch(bt, n, n, 1.0, P(ins[0]), n, nn, P(ins[1]), n, nn, P(out), n, nn)
    elif routine == "dsyrk_dpotrf_ln":
        lib.or_dsyrk_dpotrf_ln_batch(bt, n, n, P(ins[0]), n, nn, P(ins[0]), n, nn, P(ins[1]), n, nn,
                                     P(out), n, nn, P(dinv), n, ip)
    elif routine == "dgemm_nt":
        lib.or_dgemm_nt_batch(bt, n, n, n, 1.0, P(ins[0]), n, nn, P(ins[1]), n, nn, 1.0, P(ins[2]), n, nn,
                              P(out), n, nn)
    else:
        lib.or_dsyrk_ln_batch(bt, n, n, 1.0, P(ins[0]), n, nn, P(ins[0]), n, nn, 1.0, P(ins[2]), n, nn,
                              P(out), n, nn)
    return time.perf_counter() - t0


# Error bounds of the check below: the gemm/syrk bound of the routines'
# acceptance (max |D - D_oracle| <= 1e-15 k ||A||_F ||B||_F), the
# factorization residual ||L L^T - S||_F / ||S||_F <= 1e-13 and, for trsm,
# ||X L^T - B||_F / (||X||_F ||L||_F) <= 1e-13; the factors are also compared
# with the oracle's (relative Frobenius distance <= 1e-12; 1e-11 for trsm).
ORACLE_BOUNDS = {"dgemm_nt": 1e-15, "dsyrk_ln": 1e-15, "dpotrf_l": 1e-13, "dtrsm_rltn": 1e-13,
                 "dsyrk_dpotrf_ln": 1e-13}


def oracle_check(pts, samples=4, seed=11):
    """Errors of the GPU results against the FP64 oracle on sampled problems
    of every point (the first, the last and seeded random ones), read back
    from the outputs the timed steps wrote.  Runs in the cpu_baseline leg."""
    import numpy as np

    import oracle

    def fro(x):
        return float(np.sqrt(np.sum(x * x)))

    rng = np.random.default_rng(seed)
    out, worst = [], {}
    for p in pts:
        bt, n = p.batch, p.n
        idx = sorted({0, bt - 1, *[int(i) for i in rng.integers(0, bt, size=max(0, samples - 2))]})

        def g(X):
            return X.to_colmajor()[idx].cpu().numpy()

        D = g(p.D)
        names = {"dgemm_nt": ("A", "B", "C"), "dsyrk_ln": ("A", "C"), "dpotrf_l": ("C",),
                 "dtrsm_rltn": ("L", "B"), "dsyrk_dpotrf_ln": ("A", "C")}[p.routine]
        X = {k: g(getattr(p, k)) for k in names}
        err = oerr = 0.0
        for s in range(len(idx)):
            if p.routine == "dgemm_nt":
                A, B, C = X["A"][s], X["B"][s], X["C"][s]
                e = np.abs(D[s] - oracle.dgemm_nt(1.0, A, B, 1.0, C)).max() / (n * fro(A) * fro(B))
                err, oerr = max(err, e), max(oerr, e)
            elif p.routine == "dsyrk_ln":
                A, C = X["A"][s], X["C"][s]
                Do = oracle.dsyrk_ln(1.0, A, A, 1.0, C, D0=np.zeros((n, n)))
                e = np.abs(np.tril(D[s] - Do)).max() / (n * fro(A) ** 2)
                err, oerr = max(err, e), max(oerr, e)
            elif p.routine in ("dpotrf_l", "dsyrk_dpotrf_ln"):
                if p.routine == "dpotrf_l":
                    S = X["C"][s]
                    Lo = oracle.dpotrf_l(S)[0]
                else:
                    A, C = X["A"][s], X["C"][s]
                    S = C + A @ A.T
                    Lo = oracle.dsyrk_dpotrf_ln(A, A, C)[0]
                L = np.tril(D[s])
                err = max(err, fro(L @ L.T - S) / fro(S))
                oerr = max(oerr, fro(L - np.tril(Lo)) / fro(np.tril(Lo)))
            else:
                Lf, B = np.tril(X["L"][s]), X["B"][s]
                err = max(err, fro(D[s] @ Lf.T - B) / (fro(D[s]) * fro(Lf)))
                Xo = oracle.dtrsm_rltn(1.0, Lf, B)
                oerr = max(oerr, fro(D[s] - Xo) / fro(Xo))
        out.append({"routine": p.routine, "n": n, "problems": len(idx), "err": float(f"{err:.3e}"),
                    "rel_to_oracle": float(f"{oerr:.3e}")})
        w = worst.setdefault(p.routine, [0.0, 0.0])
        w[0], w[1] = max(w[0], err), max(w[1], oerr)
    ok = all(o["err"] <= ORACLE_BOUNDS[o["routine"]] and
             o["rel_to_oracle"] <= (1e-11 if o["routine"] == "dtrsm_rltn" else 1e-12) for o in out)
    return {"all_within_bounds": ok,
            "max_by_routine": {r: {"err": float(f"{w[0]:.3e}"), "bound": ORACLE_BOUNDS[r],
                                   "rel_to_oracle": float(f"{w[1]:.3e}")} for r, w in worst.items()},
            "sample": f"{samples} problems per point (first, last, seeded random), outputs of the timed steps",
            "per_point": out}


def oracle_single_core(points=(("dgemm_nt", 24), ("dsyrk_dpotrf_ln", 24), ("dgemm_nt", 128),
                               ("dsyrk_dpotrf_ln", 128)), budget_s=0.2):
    """The oracle on one host core, for comparison with the paper's
    single-core figures (context only: the oracle is plain loops)."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        out = {}
        for routine, n in points:
            count = max(1, int(2e6 / flops(routine, n)))
            data = _oracle_inputs(routine, n, count)
            t = _oracle_time(routine, n, data)
            if t < budget_s:
                count = max(1, int(count * budget_s / max(t, 1e-6)))
                data = _oracle_inputs(routine, n, count)
                t = _oracle_time(routine, n, data)
            out[f"{routine}@{n}"] = round(flops(routine, n) * count / t / 1e9, 3)
    finally:
        oracle.set_num_threads(cores)
    return out


def host_cpu():
    """One-line description of the host CPU (model name where the kernel
    reports one, else the implementer/part codes of an Arm core)."""
    import platform
    info = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    info.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    name = info.get("model name") or (
        f"Arm implementer {info.get('CPU implementer', '?')} part {info.get('CPU part', '?')}"
        if "CPU part" in info else platform.processor())
    return f"{name}, {os.cpu_count()} logical cores, {platform.machine()}"


def run_config1(args, dev, bt=128, n=24, graph_launches=100):
    """The small parity configuration as a latency workload: 128 problems of
    order 24 (gemm_nt with alpha = beta = 1; syrk_potrf of M, M with Q = 24 I;
    trsm against that factor).  Per routine: the median of >= 20 single
    launches after 5 warm-up launches (CUDA events, one stream), and the
    per-launch time inside one captured CUDA graph of 100 launches."""
    import statistics

    import torch

    import paper_1704_02457_gb300 as bf
    from paper_1704_02457_gb300 import inputs, tune

    mk = lambda X: bf.DMatBatch.from_colmajor(X, tight=True)  # noqa: E731
    A = mk(inputs.normal((bt, n, n), 20170508, dev))
    B = mk(inputs.normal((bt, n, n), 20170509, dev))
    C = mk(inputs.normal((bt, n, n), 20170510, dev))
    Q = torch.zeros(bt, n, n, dtype=torch.float64, device=dev)
    Q.diagonal(dim1=1, dim2=2).fill_(float(n))
    Qd = mk(Q)
    D = bf.DMatBatch(bt, n, n, device=dev, tight=True)
    L = bf.DMatBatch(bt, n, n, device=dev, fill=0.0)
    X = bf.DMatBatch(bt, n, n, device=dev, tight=True)
    info = torch.zeros(bt, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream()
    calls = {
        "dgemm_nt": lambda: bf.dgemm_nt(n, n, n, 1.0, A, 0, 0, B, 0, 0, 1.0, C, 0, 0, D, 0, 0, stream=stream),
        "dsyrk_dpotrf_ln": lambda: bf.dsyrk_dpotrf_ln(n, n, A, 0, 0, A, 0, 0, Qd, 0, 0, L, 0, 0, info=info,
                                                      stream=stream),
        "dtrsm_rltn": lambda: bf.dtrsm_rltn(n, n, 1.0, L, 0, 0, B, 0, 0, X, 0, 0, use_dinv=True, stream=stream),
    }
    out = {}
    with torch.cuda.stream(stream):
        calls["dsyrk_dpotrf_ln"]()  # the factor trsm uses
        for name, fn in calls.items():
            for _ in range(5):
                fn()
            stream.synchronize()
            ts = []
            for _ in range(max(20, args.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for _ in range(graph_launches):
                    fn()
            g.replay()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            med = statistics.median(ts)
            per = e0.elapsed_time(e1) / graph_launches
            fl = flops(name, n) * bt
            out[name] = {"launch_us": round(med * 1e3, 2), "graph_us_per_launch": round(per * 1e3, 2),
                         "gflops_single": round(fl / (med * 1e-3) / 1e9, 2),
                         "gflops_graph": round(fl / (per * 1e-3) / 1e9, 2)}
    # the floor of a launch inside a captured graph on this machine: the same
    # measurement for the library's smallest kernel (a one-element pack)
    one = torch.zeros(1, dtype=torch.float64, device=dev)
    P1 = bf.DMatBatch(1, 1, 1, device=dev)
    floor_call = lambda: bf.pack(one.view(1, 1, 1), P1, stream=stream)  # noqa: E731
    with torch.cuda.stream(stream):
        for _ in range(5):
            floor_call()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(graph_launches):
                floor_call()
        g.replay()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        e1.synchronize()
    floor_us = e0.elapsed_time(e1) / graph_launches * 1e3
    return {"workload": "128 problems, n = k = 24 (A, B, C iid N(0,1); Q = 24 I)", "routines": out,
            "graph_floor_us_per_launch": round(floor_us, 2),
            "layouts": {r: tune.LAYOUT_NAMES[r][tune.current_layout(r, bt, *SIZES[r](n))] for r in calls}}


def run_gpu(args):
    import torch

    import paper_1704_02457_gb300 as bf
    from paper_1704_02457_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or world == 1:
        build()
    if world > 1:
        torch.distributed.barrier()
    build()
    bf.load()

    spec = [(r, n) for n in SWEEP_N for r in ROUTINES]
    if args.points:
        keep = set(args.points.split(","))
        spec = [(r, n) for r, n in spec if f"{r}@{n}" in keep or r in keep or str(n) in keep]
    hbm, hbm_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pts = []
    for i, (r, n) in enumerate(spec):
        pts.append(Point(r, n, dev, seed=5000 + 97 * i))
        torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    # the kernel layout of every point: timed by the autotuner on the point's
    # own operands (untimed here), or the built-in rule with --no-tune
    from paper_1704_02457_gb300 import tune
    tuned = {}
    t_tune = time.perf_counter()
    for p in pts:
        sizes = SIZES[p.routine](p.n)
        if args.no_tune:
            lay = tune.rule_layout(p.routine, p.batch, *sizes)
            p.layout = tune.LAYOUT_NAMES[p.routine][lay]
        else:
            c = tune.tune(p.routine, p.batch, *sizes, run=lambda p=p: p.run(stream), stream=stream)
            p.layout = tune.LAYOUT_NAMES[p.routine][c.layout]
            tuned[(p.routine, p.n)] = c.as_dict()
    t_tune = time.perf_counter() - t_tune

    def step(ev=None):
        for j, p in enumerate(pts):
            if ev is not None:
                ev[j][0].record(stream)
            p.run(stream)
            if ev is not None:
                ev[j][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in pts]
           for _ in range(K)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    time.sleep(0.3)
    t0.record(stream)
    for s in range(K):
        step(evs[s])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    ms_per_step = total_ms / K
    step_flops = sum(p.flops for p in pts)
    value = job_rate(step_flops, ms_per_step * 1e-3, world)

    per_point = []
    per_routine = {}
    for j, p in enumerate(pts):
        times = [evs[s][j][0].elapsed_time(evs[s][j][1]) for s in range(K)]
        med = statistics.median(times)
        mean = sum(times) / len(times)
        g = p.flops / (med * 1e-3) / 1e9
        roof = roofline_gflops(p.routine, p.n, hbm)
        row = {"routine": p.routine, "n": p.n, "batch": p.batch, "ms": round(med, 4),
               "gflops": round(g, 2), "roofline_frac": round(g / roof, 4), "layout": p.layout}
        if (p.routine, p.n) in tuned:
            t = tuned[(p.routine, p.n)]
            row["rule_layout"] = t["rule_layout"]
            row["layout_ms"] = t["layout_ms"]
        per_point.append(row)
        acc = per_routine.setdefault(p.routine, [0.0, 0.0, 0, 0.0])
        acc[0] += p.flops
        acc[1] += mean
        acc[2] += 1
        acc[3] += alg_bytes(p.routine, p.n) * p.batch

    # dominant kernel: the kernel function with the largest share of step time;
    # its roofline is reported for its largest launch of the step
    by_kernel = {}
    for j, p in enumerate(pts):
        times = [evs[s][j][0].elapsed_time(evs[s][j][1]) for s in range(K)]
        by_kernel.setdefault(kernel_of(p.routine, p.n, p.layout, p.batch, sms), []).append((statistics.mean(times), p))
    step_ms = sum(t for v in by_kernel.values() for t, _ in v)
    dom = max(by_kernel, key=lambda kname: sum(t for t, _ in by_kernel[kname]))
    t_big, p_big = max(by_kernel[dom], key=lambda x: x[0])
    achieved_tflops = p_big.flops / (t_big * 1e-3) / 1e12
    tr = TRAFFIC.get((dom, p_big.routine, p_big.n))
    traffic = tr["bytes"] if tr and _git_blob_hash(tr["src"]) == tr["blob"] else None
    roof_obj = {
        "kernel": dom,
        "launch": f"{p_big.routine} n={p_big.n} batch={p_big.batch}",
        "bound": "alu",
        "achieved": round(achieved_tflops, 4),
        "peak": round(FP64_PEAK_GFLOPS / 1e3, 4),
        "unit": "TFLOP/s",
        "frac": round(achieved_tflops / (FP64_PEAK_GFLOPS / 1e3), 4),
        "traffic": traffic,
        "algorithmic_bytes_per_launch": round(alg_bytes(p_big.routine, p_big.n) * p_big.batch),
        "kernel_time_share": round(sum(t for t, _ in by_kernel[dom]) / step_ms, 4),
        "peak_source": "FP64 ALU peak from unit counts and clock (152 SMs x 2 FMA/clk x 2 flop x "
                       "2.07 GHz); HBM roof of the per-point fractions uses %s %.0f GB/s" % (hbm_src, hbm),
        "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this launch (%s)" % tr["profile"])
                          if traffic else None,
    }

    result = {
        "metric": "batched dsyrk_dpotrf/dgemm_nt GFLOP/s & roofline % vs n; mixed vs FP64 at 1e-12",
        "value": round(value, 2),
        "unit": "GFLOP/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded iid N(0,1), SPD M M^T + n I)",
        "config": config_dict(spec),
        "gpu_launches": sum(launches_of(p.routine, p.n, p.batch, sms, p.layout) for p in pts) * K,
        "layouts": ("autotuned per point before the timed steps (%.1f s, untimed); per_point gives each "
                    "layout's time" % t_tune) if not args.no_tune else "built-in rule (--no-tune)",
        "clocks": clocks,
        "roofline": roof_obj,
        "per_point": per_point,
    }
    result["per_routine_gflops"] = {r: round(v[0] / (v[1] * 1e-3) / 1e9, 2) for r, v in per_routine.items()}

    # The end-to-end leg first: it pins about 60 GB of host memory, and host
    # DMA runs slower once the other legs have fragmented the host's memory
    # (measured on one box: 843 GFLOP/s right after the sweep, 500-700 after
    # the other legs).
    if not args.no_e2e:
        result["e2e"] = run_e2e(pts, args, dev, world)
    if not args.no_mixed:
        result["mixed_vs_fp64"] = run_mixed(args, dev)
    if not args.no_riccati:
        result["riccati"] = run_riccati(args, dev)
    if not args.no_adjoint:
        result["adjoint"] = run_adjoint(args, dev)
    if not args.no_next4:
        result["next4"] = run_next4(args, dev)
    if not args.no_config1:
        result["config1"] = run_config1(args, dev)
    if not args.no_vbatched:
        result["vbatched"] = run_vbatched(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu:
        sampler = OracleSampler(spec, budget_s=args.cpu_budget)
        rates = sampler.rates()
        t_cpu = sum(p.flops / (rates[(p.routine, p.n)] * 1e9) for p in pts)
        result["cpu_baseline"] = {"value": round(step_flops / t_cpu / 1e9, 3), "unit": "GFLOP/s",
                                  "cores": sampler.cores, "kind": "oracle", "sample": sampler.describe(),
                                  "host_cpu": host_cpu(), "single_core_gflops": oracle_single_core()}
        result["oracle_check"] = oracle_check(pts)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


# Host output buffers of the end-to-end pipeline (a ring; nothing reads
# them back during the timed steps).
E2E_OUT_SLOTS = 3


class E2EPipeline:
    """The sweep through the public C ABI with host buffers.  Every step, for
    every point: pack its inputs from pinned host memory (column-major, as a
    user holds them) into its panel-major operands with bf_pack_dmat_batched,
    run the routine, and unpack the result into pinned host memory with
    bf_unpack_dmat_batched.  The library reaches the pinned host memory
    directly (mapped), so these two calls are the host-to-device and
    device-to-host transfers: nothing else copies.

    Host inputs are kept in per-n pinned pools that the routines of that n
    share: a pool of N(0,1) data (gemm A, B, C; syrk A, C; trsm B; syrk_potrf
    M), a pool of SPD matrices (potrf), one of Cholesky factors (trsm) and one
    of n*I (syrk_potrf).  `plan` lists (point, [(operand, pinned host
    input)]) in issue order.

    Issue order: alternately from the small-n end (transfer-bound: ~1 GiB of
    inputs for little arithmetic) and the large-n end (compute-bound) of the
    sweep, so that the transfers of one kind overlap the kernels of the other.
    The points are independent; the work per step is unchanged.

    Three streams joined by events: packs (host -> device), routines, unpacks
    (device -> host), the transfer streams at high priority.  A point's pack
    waits only for the previous step's unpack of the same point (its
    operands and result are then free)."""

    def __init__(self, pts, dev):
        import torch

        from paper_1704_02457_gb300 import inputs

        by_n = {}
        for p in pts:
            by_n.setdefault(p.n, []).append(p)
        pools = {}
        for n, group in by_n.items():
            pool = {}
            need_norm = max(p.batch * n * n * {"dgemm_nt": 3, "dsyrk_ln": 2, "dtrsm_rltn": 1,
                                                 "dsyrk_dpotrf_ln": 1}.get(p.routine, 0) for p in group)
            if need_norm:
                h = torch.empty(need_norm, dtype=torch.float64, pin_memory=True)
                h.copy_(inputs.normal((need_norm,), 7000 + n, dev))
                pool["norm"] = h
            for p in group:
                bt = p.batch
                if p.routine == "dpotrf_l":
                    h = torch.empty((bt, n, n), dtype=torch.float64, pin_memory=True)
                    h.copy_(inputs.spd(bt, n, 7100 + n, dev))
                    pool["spd"] = h
                elif p.routine == "dtrsm_rltn":
                    h = torch.empty((bt, n, n), dtype=torch.float64, pin_memory=True)
                    h.copy_(p.L.to_colmajor().transpose(1, 2))
                    pool["fac"] = h
                elif p.routine == "dsyrk_dpotrf_ln":
                    h = torch.zeros((bt, n, n), dtype=torch.float64, pin_memory=True)
                    h.diagonal(dim1=1, dim2=2).fill_(float(n))
                    pool["q"] = h
            pools[n] = pool
        plan = []
        self.h2d = self.d2h = 0
        for p in pts:
            n, bt, pool = p.n, p.batch, pools[p.n]
            sz = bt * n * n
            norm = lambda i: pool["norm"][i * sz:(i + 1) * sz].view(bt, n, n)  # noqa: E731
            if p.routine == "dgemm_nt":
                ins = [("A", norm(0)), ("B", norm(1)), ("C", norm(2))]
            elif p.routine == "dsyrk_ln":
                ins = [("A", norm(0)), ("C", norm(1))]
            elif p.routine == "dpotrf_l":
                ins = [("C", pool["spd"])]
            elif p.routine == "dtrsm_rltn":
                ins = [("L", pool["fac"]), ("B", norm(0))]
            else:
                ins = [("A", norm(0)), ("C", pool["q"])]
            self.h2d += sum(h.numel() * 8 for _, h in ins)
            self.d2h += sz * 8
            plan.append((p, ins))
        lo, hi, order = 0, len(plan) - 1, []
        while lo <= hi:
            order.append(plan[lo])
            if hi != lo:
                order.append(plan[hi])
            lo, hi = lo + 1, hi - 1
        self.plan = order
        self.NO = E2E_OUT_SLOTS
        max_sz = max(p.batch * p.n * p.n for p in pts)
        # the transfer streams at the highest priority: their CTAs (one per SM,
        # waiting on the host link) start as soon as a compute CTA retires
        # instead of queueing behind the compute grid (measured: 580 -> 401 ms
        # per step)
        self.s_in = torch.cuda.Stream(priority=-1)
        self.s_run = torch.cuda.Stream()
        self.s_out = torch.cuda.Stream(priority=-1)
        self.out_host = [torch.empty(max_sz, dtype=torch.float64, pin_memory=True) for _ in range(self.NO)]
        self.in_ready = [torch.cuda.Event() for _ in self.plan]
        self.run_done = [torch.cuda.Event() for _ in self.plan]
        self.out_done = [torch.cuda.Event() for _ in self.plan]
        self.started = False
        self.count = 0
        torch.cuda.synchronize()

    def step(self, out_targets=None):
        """Issue one step.  out_targets: optional pinned host tensors, one per
        entry of `plan`, that receive the points' results instead of the
        output ring's host buffers (for checking)."""
        import torch

        import paper_1704_02457_gb300 as bf

        for jp, (p, ins) in enumerate(self.plan):
            oi = self.count % self.NO
            self.count += 1
            sz = p.batch * p.n * p.n
            with torch.cuda.stream(self.s_in):
                if self.started:
                    self.s_in.wait_event(self.out_done[jp])
                for name, h in ins:
                    bf.pack(h, getattr(p, name), stream=self.s_in)
                self.in_ready[jp].record(self.s_in)
            with torch.cuda.stream(self.s_run):
                self.s_run.wait_event(self.in_ready[jp])
                p.run(self.s_run)
                self.run_done[jp].record(self.s_run)
            with torch.cuda.stream(self.s_out):
                self.s_out.wait_event(self.run_done[jp])
                dst = out_targets[jp].view(-1)[:sz] if out_targets is not None else self.out_host[oi][:sz]
                bf.unpack(p.D, dst.view(p.batch, p.n, p.n), stream=self.s_out)
                self.out_done[jp].record(self.s_out)
        self.started = True


def link_probe(dev, nbytes=1 << 30, reps=3):
    """Host-link bandwidth in this run, for reading e2e against its bound:
    copy-engine H2D / D2H (torch copies between pinned host and device
    memory), both directions at once, and the library's own transfers
    (bf_pack_dmat_batched from / bf_unpack_dmat_batched to pinned host
    memory) alone and at once.  GB/s, best of `reps`."""
    import torch

    import paper_1704_02457_gb300 as bf

    n = 64
    bt = nbytes // (8 * n * n)
    h_in = torch.empty((bt, n, n), dtype=torch.float64, pin_memory=True).fill_(1.0)
    h_out = torch.empty((bt, n, n), dtype=torch.float64, pin_memory=True)
    d_a = torch.empty((bt, n, n), dtype=torch.float64, device=dev)
    d_b = torch.empty((bt, n, n), dtype=torch.float64, device=dev)
    P = bf.DMatBatch(bt, n, n, tight=True)
    Q = bf.DMatBatch(bt, n, n, tight=True)
    Q.storage.fill_(2.0)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nb = bt * n * n * 8

    def best(fn, nbytes_moved):
        out = 0.0
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            out = max(out, nbytes_moved / (time.perf_counter() - t0) / 1e9)
        return round(out, 1)

    def both(f_in, f_out):
        def go():
            with torch.cuda.stream(s1):
                f_in()
            with torch.cuda.stream(s2):
                f_out()
        return go

    ce_in = lambda: d_a.copy_(h_in, non_blocking=True)  # noqa: E731
    ce_out = lambda: h_out.copy_(d_b, non_blocking=True)  # noqa: E731
    bf_in = lambda: bf.pack(h_in, P, stream=torch.cuda.current_stream())  # noqa: E731
    bf_out = lambda: bf.unpack(Q, h_out, stream=torch.cuda.current_stream())  # noqa: E731
    res = {"copy_engine_h2d_gbs": best(ce_in, nb), "copy_engine_d2h_gbs": best(ce_out, nb),
           "copy_engine_both_gbs_each": best(both(ce_in, ce_out), nb),
           "bf_pack_from_host_gbs": best(bf_in, nb), "bf_unpack_to_host_gbs": best(bf_out, nb),
           "bf_both_gbs_each": best(both(bf_in, bf_out), nb), "bytes": nb}
    del h_in, h_out, d_a, d_b, P, Q
    torch.cuda.empty_cache()
    return res


def run_e2e(pts, args, dev, world):
    """The end-to-end leg: E2EPipeline steps timed on the host clock, plus a
    probe of the host link in the same run."""
    import torch

    pipe = E2EPipeline(pts, dev)
    steps = max(1, min(args.steps, 5))  # the mean over up to five steps: the host link is shared
    pipe.step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        pipe.step()
    torch.cuda.synchronize()
    dt = max_over_ranks((time.perf_counter() - t0) / steps, world, dev)
    step_flops = sum(p.flops for p in pts)
    h2d, d2h = pipe.h2d, pipe.d2h
    del pipe
    torch.cuda.empty_cache()
    link = link_probe(dev)
    # the time the host link alone needs for the step's transfers: a lower
    # bound with each direction at the library's one-way rate (full duplex),
    # and the time at its measured rate with both directions at once
    r_in, r_out = link["bf_pack_from_host_gbs"] * 1e9, link["bf_unpack_to_host_gbs"] * 1e9
    each = link["bf_both_gbs_each"] * 1e9
    bound_ms = max(h2d / r_in, d2h / r_out) * 1e3 if r_in > 0 and r_out > 0 else None
    shared_ms = max(h2d, d2h) / each * 1e3 if each > 0 else None
    return {"value": round(job_rate(step_flops, dt, world), 2), "unit": "GFLOP/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": steps, "ms_per_step": round(dt * 1e3, 2), "link": link,
            "link_bound_ms": round(bound_ms, 2) if bound_ms else None,
            "link_both_directions_ms": round(shared_ms, 2) if shared_ms else None,
            "path": "pinned host column-major -> bf_pack_dmat_batched (reads the host directly) -> routine "
                    "-> bf_unpack_dmat_batched (writes the host directly), points issued small-n/large-n "
                    "alternately on three streams (pack, compute, unpack)"}


def run_mixed(args, dev, bt=8192, n=128, nrhs=4):
    """Mixed precision vs plain FP64 on SPD solves to a 1e-12 relative
    residual: 8192 systems of order 128 with cond(A) log-uniform in
    [1e2, 1e6] and 4 right-hand sides each.  Arms:
      fp64    potrf + potrs in FP64;
      ffma    FP32 factor on the FP32 FMA pipe + FP64 iterative refinement;
      bf16_tc, tf32_tc, 3xtf32_tc   blocked factor: FP64 diagonal blocks and
              panels, trailing updates on the tensor cores (tcgen05) in BF16,
              TF32 or split TF32, + the same FP64 refinement.
    Per arm: time on the whole batch, and per cond band (1e2-1e3 ... 1e5-1e6)
    the share of systems that reach 1e-12, their mean corrections, the
    systems not converged within 30 corrections (iters -1) and those whose
    factorization failed (iters -2), and the time of a batch of that band
    alone."""
    import numpy as np
    import torch

    import paper_1704_02457_gb300 as bf
    from paper_1704_02457_gb300 import inputs

    A, cond = inputs.spd_cond(bt, n, 9000, dev)
    B = inputs.normal((bt, n, nrhs), 9001, dev)
    stream = torch.cuda.current_stream()
    reps = max(3, args.steps)

    def timeit(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def arms_for(Ab, Bb):
        """Callables of every arm on one batch, and their outputs."""
        m = Ab.shape[0]
        dA, dB = bf.DMatBatch.from_colmajor(Ab, tight=True), bf.DMatBatch.from_colmajor(Bb, tight=True)
        dL = bf.DMatBatch(m, n, n, tight=True, fill=0.0)
        out = {}
        info = torch.zeros(m, dtype=torch.int32, device=dev)

        def fp64(X=bf.DMatBatch(m, n, nrhs, tight=True)):
            bf.dpotrf_l(n, dA, 0, 0, dL, 0, 0, dinv=False, info=info, stream=stream)
            bf.dpotrs_l(n, nrhs, dL, 0, 0, dB, 0, 0, X, 0, 0, stream=stream)
            return X, None

        out["fp64"] = fp64
        for name, prec in [("ffma", None), ("bf16_tc", "bf16"), ("tf32_tc", "tf32"), ("3xtf32_tc", "3xtf32")]:
            X = bf.DMatBatch(m, n, nrhs, tight=True)
            it = torch.zeros(m, dtype=torch.int32, device=dev)
            res = torch.zeros(m, dtype=torch.float64, device=dev)
            box = {"work": None}

            def call(X=X, it=it, res=res, box=box, prec=prec):
                if prec is None:
                    box["work"] = bf.dposv_mixed(n, nrhs, dA, 0, 0, dB, 0, 0, X, 0, 0, tol=1e-12, max_iter=30,
                                                 iters=it, resid=res, work=box["work"], stream=stream)
                else:
                    box["work"] = bf.dposv_mixed_tc(n, nrhs, dA, 0, 0, dB, 0, 0, X, 0, 0, prec=prec, tol=1e-12,
                                                    max_iter=30, iters=it, resid=res, work=box["work"],
                                                    stream=stream)
                return X, it

            out[name] = call
        return out

    def rel(X):
        R = B - torch.bmm(A, X)
        return (torch.linalg.matrix_norm(R) / (torch.linalg.matrix_norm(A) * torch.linalg.matrix_norm(X))).cpu().numpy()

    arms = arms_for(A, B)
    times, iters, resids = {}, {}, {}
    for name, fn in arms.items():
        times[name] = timeit(fn)
        X, it = fn()
        torch.cuda.synchronize()
        iters[name] = it.cpu().numpy() if it is not None else None
        resids[name] = rel(X.to_colmajor())
    lc = np.log10(cond.cpu().numpy())
    bands = [(2, 3), (3, 4), (4, 5), (5, 6)]
    per_arm = {}
    for name in arms:
        it = iters[name]
        entry = {"ms": round(times[name], 4), "speedup_vs_fp64": round(times["fp64"] / times[name], 3)}
        if it is not None:
            ok = it >= 1
            entry["converged"] = int(ok.sum())
            entry["not_converged_iters_-1"] = int((it == -1).sum())
            entry["factorization_failed_iters_-2"] = int((it == -2).sum())
            entry["max_rel_resid_converged"] = float(resids[name][ok].max()) if ok.any() else None
            entry["mean_iters"] = round(float(it[ok].mean()), 3) if ok.any() else None
            by_band = {}
            for lo, hi in bands:
                sel = (lc >= lo) & (lc < hi)
                s_ok = ok[sel]
                by_band[f"1e{lo}-1e{hi}"] = {
                    "systems": int(sel.sum()), "converged_frac": round(float(s_ok.mean()), 4) if sel.any() else None,
                    "mean_iters": round(float(it[sel][s_ok].mean()), 3) if s_ok.any() else None,
                    "iters_-1": int((it[sel] == -1).sum()), "iters_-2": int((it[sel] == -2).sum())}
            entry["by_cond"] = by_band
        else:
            entry["max_rel_resid"] = float(resids[name].max())
        per_arm[name] = entry
    # each band alone: the time of every arm on a batch of that band's systems
    for lo, hi in bands:
        idx = torch.from_numpy(np.nonzero((lc >= lo) & (lc < hi))[0]).to(dev)
        if idx.numel() == 0:
            continue
        band_arms = arms_for(A.index_select(0, idx).contiguous(), B.index_select(0, idx).contiguous())
        for name, fn in band_arms.items():
            per_arm[name].setdefault("band_ms", {})[f"1e{lo}-1e{hi}"] = round(timeit(fn), 4)
        del band_arms
        torch.cuda.empty_cache()
    fl = bt * (n ** 3 / 3.0 + n ** 2 / 2.0 + n / 6.0 + 2.0 * n * n * nrhs)
    t64, tmx = times["fp64"], times["ffma"]
    it = iters["ffma"]
    hist = {int(k): int(v) for k, v in zip(*np.unique(it, return_counts=True))}
    return {
        "workload": "8192 SPD systems, n=128, cond log-uniform in [1e2,1e6] (Q diag(lam) Q^T), 4 RHS",
        "fp64_path": "potrf_l + potrs_l (FP64)",
        "mixed_path": "FP32 potrf (FFMA) + FP32 triangular solves + FP64 residuals, stop at 1e-12",
        "fp64_ms": round(t64, 4), "mixed_ms": round(tmx, 4), "speedup": round(t64 / tmx, 3),
        "fp64_gflops": round(fl / (t64 * 1e-3) / 1e9, 2),
        "mixed_gflops_equiv": round(fl / (tmx * 1e-3) / 1e9, 2),
        "max_rel_resid_fp64": float(resids["fp64"].max()),
        "max_rel_resid_mixed": float(resids["ffma"][it >= 1].max()),
        "all_converged": bool((it >= 1).all()), "iters_hist": hist,
        "mean_iters": round(float(it[it >= 1].mean()), 3) if (it >= 1).any() else None,
        "arms": per_arm,
    }


def run_riccati(args, dev, batch=4096, N=20):
    """Uneven batched backward Riccati recursion (square-root form, Sec. 5.3):
    4096 MPC instances, horizon 20, nx ~ U{8..64}, nu ~ U{2..16}, A and B iid
    N(0, 1/nx), Q = R = I, P_N = I.  The bucket launches are captured in a
    CUDA graph and replayed; CTA widths come from the autotuner."""
    import numpy as np
    import torch

    from paper_1704_02457_gb300 import inputs
    from paper_1704_02457_gb300.riccati import RiccatiBatch

    rng = np.random.default_rng(20170508)
    nx = rng.integers(8, 65, size=batch)
    nu = rng.integers(2, 17, size=batch)
    rb = RiccatiBatch(nx, nu, N, device=dev)
    counter = [0]

    def gen(a, b, count):
        counter[0] += 1
        A = inputs.normal((count, a, a), 11000 + 2 * counter[0], dev) / np.sqrt(a)
        B = inputs.normal((count, a, b), 11001 + 2 * counter[0], dev) / np.sqrt(a)
        return A, B

    rb.set_inputs(gen, None)
    tune = rb.autotune()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        rb.run()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rb.run()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    reps = max(3, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    info = rb.infos()
    gf = rb.flops / (ms * 1e-3) / 1e9
    return {
        "workload": "4096 MPC instances, N=20, nx~U{8..64}, nu~U{2..16}, A,B~N(0,1/nx), Q=R=I, P_N=I; "
                    "square-root Riccati (trmm_rlnn + syrk_potrf_ln + trsm_rlnn per stage)",
        "ms": round(ms, 4), "gflops": round(gf, 2), "frac_fp64_peak": round(gf / FP64_PEAK_GFLOPS, 4),
        "flops": rb.flops, "launches_per_recursion": len(rb.buckets), "cuda_graph": True,
        "autotune": tune, "all_info_zero": bool((info == 0).all()),
    }


def run_adjoint(args, dev, bt=2048, n=64, nrhs=1):
    """Factor-and-solve x = A^{-1} b and its hand-written adjoint
    (db = A^{-1} xbar, dA = -sym(db x^T)) on 2048 SPD systems
    M M^T + 64 I of order 64 with one right-hand side.  The gradient is
    cross-checked against torch.linalg.solve's autograd (symmetrized)."""
    import torch

    import paper_1704_02457_gb300 as bf
    from paper_1704_02457_gb300 import inputs

    S = inputs.spd(bt, n, 12000, dev)
    B = inputs.normal((bt, n, nrhs), 12001, dev)
    W = inputs.normal((bt, n, nrhs), 12002, dev)
    dS, dB, dW = (bf.DMatBatch.from_colmajor(X, tight=True) for X in (S, B, W))
    dL = bf.DMatBatch(bt, n, n, tight=True, fill=0.0)
    dX = bf.DMatBatch(bt, n, nrhs, tight=True)
    dBb, dAb = bf.DMatBatch(bt, n, nrhs, tight=True), bf.DMatBatch(bt, n, n, tight=True)
    lib = bf.load()
    stream = torch.cuda.current_stream()

    def fwd():
        bf.dpotrf_l(n, dS, 0, 0, dL, 0, 0, dinv=False, stream=stream)
        bf.dpotrs_l(n, nrhs, dL, 0, 0, dB, 0, 0, dX, 0, 0, stream=stream)

    def bwd():
        bf._check("adjoint", lib.bf_dposv_adjoint_batched(bt, n, nrhs, *bf._op(dL), *bf._op(dX), *bf._op(dW),
                                                          *bf._op(dBb), *bf._op(dAb), bf._stream(stream)))

    def timeit(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(3, args.steps)
    tf, tb = timeit(fwd, reps), timeit(bwd, reps)
    # cross-check on a sample against torch's autograd of a general solve
    k = 64
    A_ = S[:k].clone().requires_grad_(True)
    B_ = B[:k].clone().requires_grad_(True)
    (torch.linalg.solve(A_, B_) * W[:k]).sum().backward()
    gA_ref = 0.5 * (A_.grad + A_.grad.transpose(1, 2))
    gA, gB = dAb.to_colmajor()[:k], dBb.to_colmajor()[:k]
    relA = float(((gA - gA_ref).norm(dim=(1, 2)) / gA_ref.norm(dim=(1, 2))).max())
    relB = float(((gB - B_.grad).norm(dim=(1, 2)) / B_.grad.norm(dim=(1, 2))).max())
    fl_f = bt * (n ** 3 / 3.0 + n ** 2 / 2.0 + n / 6.0 + 2.0 * n * n * nrhs)
    fl_b = bt * (2.0 * n * n * nrhs + 4.0 * n * n * nrhs)
    return {
        "workload": "2048 SPD systems M M^T + 64 I, n=64, 1 RHS; forward potrf+potrs, backward adjoint kernel",
        "forward_ms": round(tf, 4), "backward_ms": round(tb, 4),
        "forward_gflops": round(fl_f / (tf * 1e-3) / 1e9, 2), "backward_gflops": round(fl_b / (tb * 1e-3) / 1e9, 2),
        "max_rel_err_dA_vs_torch": relA, "max_rel_err_db_vs_torch": relB,
    }


def next4_flops(routine: str, n: int) -> float:
    """Flops of one n x n problem, counted from the algorithm's own steps:
    gemm_nn 2n^3; trmm_rlnn one FMA per nonzero of L per row of B; getrf per
    column j a reciprocal-scaled column of k = n-j-1 multipliers and a k x k
    rank-1 update; gelqf per row i a norm (2k) and scaling (k) of the
    k = n-i-1 tail entries, then for each of the k rows below a dot product
    (2k), tau * w and the update of k+1 entries (2k + 1)."""
    if routine == "dgemm_nn":
        return 2.0 * n ** 3
    if routine == "dtrmm_rlnn":
        return float(n * n * (n + 1))
    if routine == "dgetrf":
        return float(sum(k + 2 * k * k for k in range(n)))
    if routine == "dgelqf":
        return float(sum(3 * k + k * (4 * k + 2) for k in range(n)))
    raise ValueError(routine)


NEXT4_POINTS = [("dgemm_nn", 64, 4096), ("dtrmm_rlnn", 64, 4096), ("dgetrf", 16, 65536), ("dgetrf", 64, 8192),
                ("dgetrf", 128, 2048), ("dgetrf", 192, 1024), ("dgetrf", 256, 512), ("dgelqf", 16, 65536),
                ("dgelqf", 64, 8192), ("dgelqf", 128, 2048), ("dgelqf", 192, 1024), ("dgelqf", 256, 512)]


def run_next4(args, dev):
    """The remaining routines of the paper's list on square problems, each
    batch's inputs larger than L2 (at least 128 MiB read per launch): CUDA
    events around `reps` back-to-back launches on the current stream after
    three warm-up launches."""
    import torch

    import paper_1704_02457_gb300 as bf
    from paper_1704_02457_gb300 import inputs, tune

    stream = torch.cuda.current_stream()
    out = {}
    for i, (r, n, bt) in enumerate(NEXT4_POINTS):
        A = bf.DMatBatch.from_colmajor(inputs.normal((bt, n, n), 13000 + 7 * i, dev), tight=True)
        D = bf.DMatBatch(bt, n, n, device=dev, tight=True)
        if r in ("dgemm_nn", "dtrmm_rlnn"):
            B = bf.DMatBatch.from_colmajor(inputs.normal((bt, n, n), 13001 + 7 * i, dev), tight=True)
        if r == "dgemm_nn":
            C = bf.DMatBatch.from_colmajor(inputs.normal((bt, n, n), 13002 + 7 * i, dev), tight=True)
            fn = lambda: bf.dgemm_nn(n, n, n, 1.0, A, 0, 0, B, 0, 0, 1.0, C, 0, 0, D, 0, 0, stream=stream)  # noqa: E731
        elif r == "dtrmm_rlnn":
            fn = lambda: bf.dtrmm_rlnn(n, n, 1.0, A, 0, 0, B, 0, 0, D, 0, 0, stream=stream)  # noqa: E731
        elif r == "dgetrf":
            ipiv = torch.empty((bt, n), dtype=torch.int32, device=dev)
            info = torch.empty((bt,), dtype=torch.int32, device=dev)
            fn = lambda: bf.dgetrf(n, A, 0, 0, D, 0, 0, ipiv, info=info, stream=stream)  # noqa: E731
        else:
            tau = torch.empty((bt, n), dtype=torch.float64, device=dev)
            fn = lambda: bf.dgelqf(n, n, A, 0, 0, D, 0, 0, tau, stream=stream)  # noqa: E731
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        reps = max(3, args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        g = bt * next4_flops(r, n) / (ms * 1e-3) / 1e9
        out[f"{r}@{n}"] = {"batch": bt, "ms": round(ms, 4), "gflops": round(g, 2),
                           "frac_of_fp64_alu_peak": round(g / FP64_PEAK_GFLOPS, 4)}
        if r in tune.ROUTINE_IDS:
            out[f"{r}@{n}"]["layout"] = tune.LAYOUT_NAMES[r][tune.current_layout(r, bt, n, n, 0)]
        del A, D
        torch.cuda.empty_cache()
    return out


def run_vbatched(args, dev, batch=4096, nmin=8, nmax=128):
    """The descriptor-array forms on uneven sizes: 4096 problems of order
    n ~ U{8..128} (k = n), each in the top-left corner of a 128 x 128 slot,
    through gemm_nt and syrk_potrf (SPD: M M^T + n I).  CUDA events around
    `reps` launches after three warm-up launches."""
    import numpy as np
    import torch

    import paper_1704_02457_gb300 as bf
    from paper_1704_02457_gb300 import inputs

    rng = np.random.default_rng(14000)
    ns0 = rng.integers(nmin, nmax + 1, size=batch)
    mk = lambda seed: bf.DMatBatch.from_colmajor(inputs.normal((batch, nmax, nmax), seed, dev), tight=True)  # noqa: E731
    A, B, C = mk(14001), mk(14002), mk(14003)
    Q = torch.zeros(batch, nmax, nmax, dtype=torch.float64, device=dev)
    Q.diagonal(dim1=1, dim2=2).copy_(torch.from_numpy(np.repeat(ns0[:, None], nmax, 1)).to(dev).double())
    Qd = bf.DMatBatch.from_colmajor(Q, tight=True)
    del Q
    D = bf.DMatBatch(batch, nmax, nmax, device=dev, tight=True)
    info = torch.zeros(batch, dtype=torch.int32, device=dev)
    status = torch.zeros(batch, dtype=torch.int32, device=dev)
    vorder = torch.zeros(batch, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    calls = {}
    # the records in generation order, and sorted by decreasing order (a
    # caller that knows its sizes passes the longest problems first, as the
    # Riccati leg does; the CTAs then start longest-first)
    for tag, order in (("", np.arange(batch)), ("_sorted", np.argsort(-ns0, kind="stable"))):
        ns = ns0[order]
        sizes = bf.dsize_records([(int(n), int(n), int(n)) for n in ns], device=dev)
        rec = lambda M, order=order: bf.dsub_records([(M, int(b), 0, 0) for b in order], device=dev)  # noqa: E731
        rA, rB, rC, rQ, rD = rec(A), rec(B), rec(C), rec(Qd), rec(D)
        calls["dgemm_nt" + tag] = (
            lambda sizes=sizes, rA=rA, rB=rB, rC=rC, rD=rD: bf.dgemm_nt_vbatched(
                batch, sizes, 1.0, rA, rB, 1.0, rC, rD, nmax, nmax, status=status, stream=stream),
            float(sum(flops("dgemm_nt", int(n)) for n in ns)))
        calls["dsyrk_dpotrf_ln" + tag] = (
            lambda sizes=sizes, rA=rA, rQ=rQ, rD=rD: bf.dsyrk_dpotrf_ln_vbatched(
                batch, sizes, rA, rA, rQ, rD, nmax, info=info, status=status, stream=stream),
            float(sum(flops("dsyrk_dpotrf_ln", int(n)) for n in ns)))
        # the ordered form: the records sorted by size on the device (inside
        # the timed call), then problems of one size class sharing a CTA
        calls["dsyrk_dpotrf_ln_ordered" + tag] = (
            lambda sizes=sizes, rA=rA, rQ=rQ, rD=rD: (
                bf.vbatched_order(batch, sizes, nmax, vorder, stream=stream),
                bf.dsyrk_dpotrf_ln_vbatched_ordered(batch, sizes, vorder, rA, rA, rQ, rD, nmax, info=info,
                                                    status=status, stream=stream)),
            float(sum(flops("dsyrk_dpotrf_ln", int(n)) for n in ns)))
    out = {}
    for name, (fn, fl) in calls.items():
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        reps = max(3, args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        g = fl / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 4), "gflops": round(g, 2), "frac_of_fp64_alu_peak": round(g / FP64_PEAK_GFLOPS, 4)}
    out["status_all_zero"] = bool((status == 0).all())
    out["info_all_zero"] = bool((info == 0).all())
    out["workload"] = ("4096 problems, n ~ U{8..128}, k = n, descriptor-array forms (one launch per routine); "
                       "_sorted: the same problems, records sorted by decreasing order; _ordered: the records "
                       "sorted by size on the device (bf_vbatched_order, inside the timed call), then the ordered "
                       "form (two problems of neighbouring sizes per CTA, one launch)")
    return out


# ---------------------------------------------------------- reference arm --

def run_reference(args):
    """The reference arm: the CPU oracle, timed on the host cores on a bounded
    sample of every sweep point (cached after one calibration), reported as
    the same whole-step GFLOP/s metric."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    from paper_1704_02457_gb300 import inputs
    spec = [(r, n) for n in SWEEP_N for r in ROUTINES]
    sampler = OracleSampler(spec, budget_s=args.ref_budget)
    for _ in range(args.warmup):
        sampler.rates()
    step_times = []
    for _ in range(args.steps):
        rates = sampler.rates()
        step_times.append(sum(flops(r, n) * inputs.sweep_batch(r, n) / (rates[(r, n)] * 1e9) for r, n in spec))
    step_flops = sum(flops(r, n) * inputs.sweep_batch(r, n) for r, n in spec)
    t = statistics.median(step_times)
    value = step_flops / t / 1e9
    print(json.dumps({
        "impl": "reference",
        "metric": "batched dsyrk_dpotrf/dgemm_nt GFLOP/s & roofline % vs n; mixed vs FP64 at 1e-12",
        "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded iid N(0,1), SPD M M^T + n I)", "config": config_dict(spec),
        "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": sampler.cores, "kind": "oracle",
                         "sample": sampler.describe()},
        "e2e": {"value": round(value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", default="", help="comma list of routine@n, routine or n (debug subsets)")
    ap.add_argument("--no-tune", action="store_true", help="built-in kernel layouts instead of the autotuner's")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-riccati", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-next4", action="store_true")
    ap.add_argument("--no-config1", action="store_true")
    ap.add_argument("--no-vbatched", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=0.15, help="seconds of oracle time per point")
    ap.add_argument("--ref-budget", type=float, default=0.06,
                    help="seconds of oracle time per point and step of the reference arm")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
