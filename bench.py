#!/usr/bin/env python
"""Throughput of FP64 sCholQR3 (cholqr_factor) on GB300.

One step = one cholqr_factor call on a resident m x n FP64 matrix
A = U diag(s) V^T (the paper's test-matrix recipe, Sec. 4.1), default
m = 1,000,000, n = 64, kappa = 1e12.  Metric: rows*cols/s = m n / t_step,
summed over ranks (each rank factors its own matrix: replicas, weak scaling).

Prints ONE JSON line (rank 0) with the contract keys plus:
  roofline      dominant kernel by total time in the timed region: at
                17 <= n <= 128 the tensor-core digit Gramian or digit solve
                (bf16 digit FLOP against the sustained bf16 peak, with the
                FP64-equivalent rate and HBM rate beside it, and the other
                kernel nested); at n <= 16 the FP64 row solve, and without
                the tensor-core path the fused FP64 row sweep (against the
                FP64 peak); achieved rates from CUDA events on each launch's
                stream, DRAM traffic from the committed ncu capture;
  cpu_baseline  the CPU oracle on a bounded sample of the same matrix;
  e2e           the same metric through cholqr_factor_host (host buffers,
                copies inside the timed region);
  clocks        nvidia-smi samples taken during the timed region;
  sweep         a short n x kappa sweep at the same m;
  update / mixed / pn / serve   the basis-growth, mixed-precision, pnCholQR
                and serving legs (each skippable with --no-<leg>).
``--impl reference`` times the CPU oracle instead (rank 0 only).
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

METRIC = ("sCholQR3 rows·cols/s & %HBM roofline at ‖QᵀQ−I‖≤1e-13; "
          "serve p50/p99 latency")
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9   # SMs x DFMA/clk/SM x 2 FLOP x max SM clock
OZGRAM_PAIRS = 16  # symmetric digit pairs of the tensor-core Gramian (orders 0..6 of 7 digits)
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1700.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=1_000_000)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--kappa", type=float, default=1e12)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--emulation", default="auto", choices=["auto", "tcgen05", "off"],
                    help="digit kernels: auto = the tcgen05 Gramian for 33 <= n <= 64 and mma.sync elsewhere, "
                         "tcgen05 = the tcgen05 Gramian and solve for 17 <= n <= 64, off = FP64 CUDA cores")
    ap.add_argument("--no-tcgen05-leg", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=600_000)
    ap.add_argument("--cpu-rows-all-cores", type=int, default=200_000)
    ap.add_argument("--no-update", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--update-m", type=int, default=2_000_000)
    ap.add_argument("--mixed-m", type=int, default=4_000_000)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-wide", action="store_true")
    ap.add_argument("--no-pn", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=512)
    return ap.parse_args()


def peaks():
    """(HBM GB/s, source, bf16 TFLOP/s sustained, source)."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return (float(d["hbm_gbs"]), "measured", float(d["bf16_tflops_sustained"]),
                "measured (cuBLAS bf16 GEMM, sustained: the kernel runs inside a multi-kernel step)")
    except Exception:
        return FALLBACK_HBM_GBS, "fallback", FALLBACK_BF16_TFLOPS, "fallback"


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def has_sample(self) -> bool:
        try:
            return self.f is not None and os.path.getsize(self.f.name) > 0
        except OSError:
            return False

    @staticmethod
    def _stamp(parts):
        # nvidia-smi's timestamp (local time) as seconds since the epoch
        if len(parts) < 10:
            return None
        import datetime
        try:
            return datetime.datetime.strptime(parts[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, window=None):
        """Median SM clock, max clock and throttle reasons of the samples
        taken inside `window` = (t0, t1) in time.time() seconds (all samples
        when none carries a timestamp inside it)."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        in_window = None
        if window is not None:
            t0, t1 = window
            inside = [r for r in rows if (ts := self._stamp(r)) is not None and t0 - 0.05 <= ts <= t1 + 0.05]
            in_window = len(inside)
            if inside:
                rows = inside
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(rows)}
        if in_window is not None:
            out["samples_in_timed_region"] = in_window
        return out


KERNEL_FILES = {"rowsweep": ("rowsweep.cu",), "trsm_rows": ("trsm.cu",),
                "ozgram": ("ozgram.cu", "ozdigits.cuh"), "ozgemm": ("ozgemm.cu", "ozdigits.cuh"),
                "tcgram": ("tcgram.cu", "tc05.cuh", "ozdigits.cuh"), "tcgemm": ("tcgemm.cu", "tc05.cuh", "ozdigits.cuh")}
TC05_MIN_N, TC05_MAX_N = 17, 64  # widths of the tcgen05 Gramian and solve
TC05_AUTO_GRAM_MIN_N = 33        # the Gramian runs on tcgen05 by default from this width


def tc05_kernels(emulation: str, n: int):
    """(Gramian, solve) on the tcgen05 kernels for this emulation mode and
    width, the library's rule: the Gramian for 33 <= n <= 64 by default and
    for 17 <= n <= 64 under tcgen05, the solve under tcgen05 only."""
    gram = n <= TC05_MAX_N and ((emulation == "tcgen05" and n >= TC05_MIN_N) or
                                (emulation == "auto" and n >= TC05_AUTO_GRAM_MIN_N))
    solve = emulation == "tcgen05" and TC05_MIN_N <= n <= TC05_MAX_N
    return gram, solve


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and blank lines, each line
    right-stripped (string literals in the kernels hold no comment
    markers)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_hash(name: str) -> str:
    """Hash of one kernel's source files with their comments removed: the
    DRAM counters of a kernel stay valid while its code does not change."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_07788_gb300", "csrc")
    for f in KERNEL_FILES[name]:
        h.update(strip_comments(open(os.path.join(csrc, f)).read()).encode())
    return h.hexdigest()[:16]


def traffic_per_launch(rows: int, name: str, cols: int = 0):
    """DRAM bytes per launch of a kernel from its committed ncu summary
    (profiles/traffic_<name>.txt), scaled to `rows` rows (and `cols`
    columns, when the capture names its width) per launch, or None when the
    kernel sources changed since the counters were taken."""
    d = {}
    try:
        for line in open(os.path.join(ROOT, "profiles", f"traffic_{name}.txt")):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    except Exception:
        return None, None
    if d.get("source_hash") != kernel_source_hash(name):
        return None, d
    try:
        scale = rows / float(d["capture_rows"])
        if cols and "capture_cols" in d:
            scale *= cols / float(d["capture_cols"])
        return float(d["capture_bytes_per_launch"]) * scale, d
    except Exception:
        return None, d


def _oracle_factor_seconds(S):
    """One oracle sCholQR3 of S in this (spawned) process: seconds."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.cholqr(S)
    return time.perf_counter() - t0


def _oracle_ready(_):
    import oracle
    oracle.build()
    return os.getpid()


def cpu_baseline(A, rows, n, all_core_rows=None):
    """The oracle as it stands on the host cores, on bounded samples of the
    benchmark matrix: one factorisation of the first `rows` rows on one core,
    and, on every core at once, one process per core each factoring the
    first `all_core_rows` rows (the unmodified single-threaded oracle, so the
    all-core figure is the host's aggregate throughput of independent
    factorisations).  Processes are spawned, never forked from a process
    that has used the GPU."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    host_cores = os.cpu_count() or 1
    S = A[:rows]
    t0 = time.perf_counter()
    Q, R, st, info = oracle.cholqr(S)
    dt = time.perf_counter() - t0
    out = {"value": rows * n / dt, "unit": "rows*cols/s", "cores": 1, "kind": "oracle",
           "host_cores": host_cores,
           "sample": f"first {rows} of {A.shape[0]} rows of the benchmark matrix, one factorisation "
                     f"({dt:.1f} s, {info.iters} passes, single-threaded plain C)",
           "seconds": dt}
    rp = all_core_rows or max(n, rows // 4)
    try:
        Sp = A[:rp].copy(order="F")
        ctx = mp.get_context("spawn")
        with ctx.Pool(host_cores) as pool:
            pool.map(_oracle_ready, range(host_cores))
            t0 = time.perf_counter()
            secs = pool.map(_oracle_factor_seconds, [Sp] * host_cores)
            wall = time.perf_counter() - t0
        out["all_cores"] = {"value": host_cores * rp * n / wall, "unit": "rows*cols/s", "cores": host_cores,
                            "kind": "oracle",
                            "sample": f"{host_cores} processes, each one factorisation of the first {rp} rows "
                                      f"(single-threaded plain C oracle, unmodified); wall {wall:.1f} s, "
                                      f"per process {min(secs):.1f}-{max(secs):.1f} s",
                            "seconds": wall}
    except Exception as exc:  # the single-core figure stands alone
        out["all_cores"] = {"unavailable": f"{type(exc).__name__}: {exc}"}
    return out


def replica_throughput(ms_local: float, ws: int, m: int, n: int, device: str):
    """Whole-job throughput of ws independent replicas, each factoring its own
    m x n matrix: the slowest rank's time per step (max over ranks) and the
    rows*cols all ranks processed per second."""
    ms = ms_local
    if ws > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ws * m * n / (ms * 1e-3)


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return 0
    from paper_2507_07788_gb300 import synth
    import oracle
    oracle.build()
    rows = min(args.m, 250_000)
    A = synth.test_matrix(args.m if args.m <= 250_000 else rows, args.n, args.kappa, rep=0)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        Q, R, st, info = oracle.cholqr(A)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    val = rows * args.n / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "rows*cols/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"sCholQR3 FP64 n={args.n} kappa={args.kappa:g} (A=U diag(s) V^T), "
                                   f"bounded CPU sample m={rows} of m={args.m}",
                       "m": args.m, "n": args.n, "kappa": args.kappa, "sample_rows": rows},
            "cpu_baseline": {"value": val, "unit": "rows*cols/s", "cores": 1, "kind": "oracle",
                             "host_cores": os.cpu_count(),
                             "sample": f"{rows} x {args.n} matrix per step"},
            "e2e": {"value": val, "unit": "rows*cols/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_factor(cq, torch, dA, dQ, dR, opts, steps, warmup):
    for _ in range(warmup):
        cq.factor(dA, Q=dQ, R=dR, opts=opts)
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    res = None
    for _ in range(steps):
        res = cq.factor(dA, Q=dQ, R=dR, opts=opts)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, res


def roofline_from(tm, m, n, hbm_peak, hbm_src, tc_peak, tc_src, emulation="auto"):
    """Roofline of the dominant kernel from the library's per-launch events.

    The roofline of this path is HBM bytes: the top level reports the
    dominant kernel's algorithmic bytes per launch (8 per entry read, 8 per
    entry written) over its mean launch time against the measured HBM copy
    peak.  What the kernel spends besides bytes is nested: for the
    tensor-core digit kernels (17 <= n <= 128) their bf16 digit FLOP against
    the sustained bf16 tensor peak and their FP64-equivalent rate, for the
    FP64 CUDA-core kernels their FLOP against the FP64 peak.  The pass
    pipeline runs a solve kernel and the digit Gramian per row chunk; the
    one with the larger total time in the timed region is the dominant
    kernel and the other is nested under its own key."""
    def per(k):
        nl = max(tm[f"{k}_launches"], 1)
        ms = tm[f"{k}_ms"] / nl
        fl = tm[f"{k}_flops"] / nl
        by = tm[f"{k}_bytes"] / nl
        return ms, fl, by, (fl / (ms * 1e-3) if ms > 0 else 0.0), (by / (ms * 1e-3) / 1e9 if ms > 0 else 0.0)

    fp64_src = "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (FP64 CUDA cores)"

    def record(kernel, ms, fl, by, af, ag, traffic, total_ms, extra):
        r = {"bound": "hbm", "achieved": ag, "peak": hbm_peak, "unit": "GB/s",
             "frac": ag / hbm_peak if hbm_peak else 0.0, "traffic": traffic, "kernel": kernel,
             "peak_source": f"{hbm_src} (HBM copy, MEASURED_PEAKS.json hbm_gbs)",
             "per_launch": {"ms": ms, "algorithmic_bytes": by, "algorithmic_fp64_flops": fl},
             "total_ms": total_ms}
        r.update(extra)
        return r

    def fp64_alu(af):
        return {"achieved": af / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": af / FP64_PEAK_FLOPS, "peak_source": fp64_src}

    gram_tc05, solve_tc05 = tc05_kernels(emulation, n)
    gname = "tcgram" if gram_tc05 else "ozgram"
    sname = "tcgemm" if solve_tc05 else "ozgemm"
    gram = None
    if tm["gram_launches"] > 0:
        gms, gfl, gby, gaf, gag = per("gram")
        grows = gby / (8.0 * n)
        gtraffic, _ = traffic_per_launch(int(round(grows)), gname, n)
        # 16 symmetric digit pairs, each a full NT x NT block per row
        nt = 16 if n <= 16 else (32 if n <= 32 else (64 if n <= 64 else 128))
        gtcf = grows * 2.0 * OZGRAM_PAIRS * nt * nt
        gtca = gtcf / (gms * 1e-3) if gms > 0 else 0.0
        gram = record(("tcgram64_kernel (exact FP64 Gramian from bf16 digits, tcgen05 with TMEM "
                       "accumulators and TMA tiles, one launch per row chunk)") if gram_tc05 else
                      ("ozgram_kernel (exact FP64 Gramian from bf16 digits on the tensor cores, mma.sync, "
                       "one launch per row chunk)"), gms, gfl, gby, gaf, gag, gtraffic, tm["gram_ms"],
                      {"tensor": {"achieved": gtca / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
                                  "frac": gtca / 1e12 / tc_peak, "bf16_digit_flops_per_launch": gtcf,
                                  "peak_source": tc_src},
                       "fp64_equiv": fp64_alu(gaf)})
    if tm["tsolve_launches"] > 0:
        ms, fl, by, af, ag = per("tsolve")
        tcf = tm["tsolve_tc_flops"] / max(tm["tsolve_launches"], 1)
        tca = tcf / (ms * 1e-3) if ms > 0 else 0.0
        traffic, _ = traffic_per_launch(int(round(by / (16.0 * n))), sname, n)
        solve = record(("tcgemm64_kernel (Q = Y R~^-1 as an exact bf16 digit product, tcgen05 with TMEM "
                        "accumulators, one launch per row chunk)") if solve_tc05 else
                       ("ozgemm_kernel (Q = Y R~^-1 as an exact bf16 digit product on the tensor cores, "
                        "mma.sync, one launch per row chunk)"), ms, fl, by, af, ag, traffic, tm["tsolve_ms"],
                       {"tensor": {"achieved": tca / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
                                   "frac": tca / 1e12 / tc_peak, "bf16_digit_flops_per_launch": tcf,
                                   "peak_source": tc_src},
                        "fp64_equiv": fp64_alu(af)})
        if gram and gram["total_ms"] > solve["total_ms"]:
            roof = dict(gram)
            roof["solve"] = solve
        else:
            roof = dict(solve)
            if gram:
                roof["gram"] = gram
        roof["dominant_by"] = "total kernel time in the timed region (CUDA events on each launch's stream)"
        return roof
    if tm["solve_launches"] > 0:
        ms, fl, by, af, ag = per("solve")
        traffic, _ = traffic_per_launch(int(round(by / (16.0 * n))), "trsm_rows", n)  # 16 B per row entry
        roof = record("trsm_rows_kernel (FP64 row solve of the pass pipeline, one launch per row chunk)",
                      ms, fl, by, af, ag, traffic, tm["solve_ms"], {"alu": fp64_alu(af)})
        if gram:
            roof["gram"] = gram
        return roof
    ms, fl, by, af, ag = per("fused")
    traffic, _ = traffic_per_launch(int(round(m)), "rowsweep", n)
    return record("rowsweep_kernel (fused triangular solve + Gramian sweep, FP64 CUDA cores)",
                  ms, fl, by, af, ag, traffic, tm["fused_ms"], {"alu": fp64_alu(af)})


def factorisation_hbm(m, n, passes, ms, hbm_peak):
    """The whole factorisation against the HBM roofline: the first Gramian
    reads the block once (8 m n bytes) and every pass reads it once and
    writes it once (16 m n bytes; its Gramian comes with the solve), so
    3 passes move 56 m n bytes."""
    by = 8.0 * m * n + 16.0 * m * n * passes
    gbs = by / (ms * 1e-3) / 1e9
    return {"bytes": by, "passes": passes, "achieved_gbs": gbs, "peak_gbs": hbm_peak,
            "frac": gbs / hbm_peak if hbm_peak else 0.0,
            "formula": "(8 m n + 16 m n x passes) / ms_per_step"}


def append_hbm_bytes(m: int, q: int, p: int, iters: int) -> float:
    """Algorithmic HBM bytes of one append (Alg. 2) with `iters` outer
    iterations: the first sweep reads [Q_in A_in] (8 m (q + p)), every
    iteration reads [Q_in Y] and writes the new block (8 m (q + p) + 8 m p)."""
    return 8.0 * m * (q + p) + iters * (8.0 * m * (q + p) + 8.0 * m * p)


def leg_update(cq, torch, m, p=8, count=32, seed=0, cache=True, hbm_peak=0.0):
    """Basis growth (Alg. 2): 32 appends of 8 columns up to n = 256 at m rows.
    block_k = Q_prev G 0.1 + N eta (eta log-uniform in [1e-12, 1]); the first
    block is N.  Inputs are drawn on the device from a seeded generator; the
    orthogonality of every new block against the whole basis is checked
    right after its append.  With `cache` the basis keeps the digits of its
    columns (basis_enable_digit_cache), so the appends' cross Gramian and
    projection run on the tensor cores."""
    import numpy as np
    from paper_2507_07788_gb300.synth import seed_for
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed_for(m, p, count, seed) & 0x7FFFFFFFFFFFFFFF)
    rng = np.random.default_rng(seed_for(m, p, count, seed, 1))
    # warm-up: two appends to a throwaway basis of the same shape (first-use
    # costs of the kernels and of the cache's memory stay out of the timing)
    w = cq.Basis(m, 2 * p)
    if cache:
        w.enable_digit_cache()
    wgen = torch.Generator(device="cuda")
    wgen.manual_seed(seed_for(m, p, count, seed, 2) & 0x7FFFFFFFFFFFFFFF)
    for _ in range(2):
        w.append(cq.to_colmajor(torch.randn((m, p), generator=wgen, device="cuda", dtype=torch.float64)))
    w.close()
    torch.cuda.synchronize()
    b = cq.Basis(m, p * count)
    if cache:
        b.enable_digit_cache()
    blk = cq.colmajor(m, p)
    times, worst, iters, shifts, statuses = [], 0.0, [], [], []
    bytes_alg = 0.0
    torch.cuda.synchronize()
    for k in range(count):
        N = torch.randn((p, m), generator=gen, device="cuda", dtype=torch.float64).t()
        if k == 0:
            blk.copy_(N)
        else:
            Qp = b.Q()
            G = torch.randn((Qp.shape[1], p), generator=gen, device="cuda", dtype=torch.float64)
            eta = 10.0 ** rng.uniform(-12.0, 0.0)
            blk.copy_(Qp @ G * 0.1 + N * eta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = b.append(blk)
        times.append(time.perf_counter() - t0)
        bytes_alg += append_hbm_bytes(m, k * p, p, info["iters"])
        statuses.append(st)
        iters.append(info["iters"])
        shifts.append(info["shifts"])
        Qa = b.Q()
        Qn = Qa[:, -p:]
        Gm = Qa.t() @ Qn
        Gm[-p:, :] -= torch.eye(p, dtype=Gm.dtype, device=Gm.device)
        worst = max(worst, float(torch.linalg.norm(Gm)))
    q_end = b.cols
    b.close()
    tot = sum(times)
    gbs = bytes_alg / tot / 1e9
    return {"workload": f"basis growth m={m}: {count} appends of p={p} to n={q_end}, blocks Q_prev G 0.1 + N eta"
                        + (", basis digit cache" if cache else ", FP64 projection and cross Gramian"),
            "appends_per_s": count / tot, "ms_per_append_mean": 1e3 * tot / count,
            "ms_per_append_median": 1e3 * statistics.median(times), "ms_first_append": 1e3 * times[0],
            "ms_per_append_last": 1e3 * times[-1], "rows_cols_per_s": m * q_end / tot,
            "max_block_orth_frob": worst, "iters": iters, "shifts": shifts,
            "status": sorted(set(statuses)),
            "hbm": {"bytes": bytes_alg, "achieved_gbs": gbs, "peak_gbs": hbm_peak,
                    "frac": gbs / hbm_peak if hbm_peak else 0.0,
                    "formula": "sum over appends of 8 m (q + p) + iters (8 m (q + p) + 8 m p), over the summed append times"}}


def leg_mixed(cq, torch, synth, m, n=128, kappas=(1e6, 1e10, 1e14), steps=3, hbm_peak=0.0):
    """Mixed precision vs plain FP64 at m x 128 on the same matrices; beside
    each factorisation, its first-pass Gramian alone (cholqr_gram with the
    same options: the exact digit Gramian for FP64, the reduced-digit one for
    mixed)."""
    out = []
    for kap in kappas:
        A = synth.test_matrix(m, n, kap, rep=21)
        dA = cq.to_colmajor(A)
        del A
        dQ, dR = cq.colmajor(m, n), cq.colmajor(n, n)
        row = {"kappa": kap}
        for prec, name in ((cq.PREC_FP64, "fp64"), (cq.PREC_MIXED, "mixed")):
            o = cq.default_opts(precision=prec)
            ms, res = time_factor(cq, torch, dA, dQ, dR, o, steps, 1)
            Gm = dQ.t() @ dQ
            loo = float(torch.linalg.norm(Gm - torch.eye(n, dtype=Gm.dtype, device=Gm.device)))
            rrr = float(torch.linalg.norm(dA - dQ @ torch.triu(dR)) / torch.linalg.norm(dA))
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            cq.gram(dA, opts=o)
            torch.cuda.synchronize()
            g0.record()
            for _ in range(steps):
                cq.gram(dA, opts=o)
            g1.record()
            torch.cuda.synchronize()
            row[name] = {"ms": ms, "rows_cols_per_s": m * n / (ms * 1e-3), "iters": res.info["iters"],
                         "status": res.status, "loo_frob": loo, "rrr_frob": rrr,
                         "sigma_first": res.info["sigma_first"],
                         "first_gram_ms": g0.elapsed_time(g1) / steps,
                         "hbm_frac": factorisation_hbm(m, n, res.info["iters"], ms, hbm_peak)["frac"]}
        row["speedup_mixed_vs_fp64"] = row["fp64"]["ms"] / row["mixed"]["ms"]
        out.append(row)
        del dA, dQ, dR
        torch.cuda.empty_cache()
    return {"workload": f"mixed vs FP64 sCholQR3, m={m} n={n}, A=U diag(s) V^T", "rows": out}


def leg_wide(cq, torch, synth, m=200000, ns=(192, 256, 384, 512), off_ns=(256, 512), kappa=1e12, steps=2,
             hbm_peak=0.0):
    """Widths above 128: the Gramian by 64 x 64 block pairs on the tensor
    cores, the tensor-core solve with its
    contraction in blocks of 64 and the cooperative control step, beside
    n = 128 (tensor-core pipeline) and, at the widths in off_ns, the FP64
    row sweeps (emulation off)."""
    rows = []
    cases = [(n, "auto") for n in (128,) + tuple(ns)] + [(n, "off") for n in off_ns]
    cases.sort()
    for n, emu in cases:
        A = synth.test_matrix(m, n, kappa, rep=41)
        dA = cq.to_colmajor(A)
        del A
        dQ, dR = cq.colmajor(m, n), cq.colmajor(n, n)
        opts = cq.default_opts(emulation=cq.EMU_OFF if emu == "off" else cq.EMU_AUTO)
        ms, res = time_factor(cq, torch, dA, dQ, dR, opts, steps, 1)
        if n <= 128:
            path = "tensor-core digit kernels"
        elif emu == "off":
            path = "FP64 CUDA cores (Gramian and solve), cooperative control step"
        else:
            path = "tensor-core Gramian (64 x 64 block pairs) and solve (blocks of 64), cooperative control step"
        rows.append({"n": n, "emulation": emu, "ms": ms, "rows_cols_per_s": m * n / (ms * 1e-3),
                     "iters": res.info["iters"], "status": res.status, "orth_frob": res.info["orth_frob"],
                     "hbm_frac": factorisation_hbm(m, n, res.info["iters"], ms, hbm_peak)["frac"], "path": path})
        del dA, dQ, dR
        torch.cuda.empty_cache()
    return {"workload": f"sCholQR3 at m={m}, kappa={kappa:g}, n = 128 and above", "rows": rows}


def leg_pn(cq, torch, synth, m, n=64, kappa=1e12, rs=(1, 2, 4, 8), steps=2):
    """pnCholQR (Alg. 3) with r panels against sCholQR3 on the same matrix.
    The paper's flop model puts pnCholQR at G(r) = 1/2 + 1/(2r) of the
    one-shot method's flops (its flop comparison of Alg. 3)."""
    A = synth.test_matrix(m, n, kappa, rep=41)
    dA = cq.to_colmajor(A)
    del A
    dQ, dR = cq.colmajor(m, n), cq.colmajor(n, n)
    ms_f, rf = time_factor(cq, torch, dA, dQ, dR, None, steps, 1)
    rows = []
    for r in rs:
        cq.pn(dA, r, Q=dQ, R=dR)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            res = cq.pn(dA, r, Q=dQ, R=dR)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        G = dQ.t() @ dQ
        loo = float(torch.linalg.norm(G - torch.eye(n, dtype=G.dtype, device=G.device)))
        rows.append({"r": r, "ms": ms, "rows_cols_per_s": m * n / (ms * 1e-3), "status": res.status,
                     "iters_total": res.info["iters"], "loo_frob": loo, "time_vs_scholqr3": ms / ms_f,
                     "paper_flop_ratio": 0.5 + 0.5 / r})
    del dA, dQ, dR
    torch.cuda.empty_cache()
    return {"workload": f"pnCholQR vs sCholQR3, m={m} n={n} kappa={kappa:g}, A=U diag(s) V^T",
            "scholqr3_ms": ms_f, "scholqr3_iters": rf.info["iters"], "rows": rows}


def leg_serve(cq, torch, n_requests=512, utilization=0.7):
    """Serving: Poisson arrivals (seed 0) of factor / append requests over 64
    device-resident bases (m log-uniform in [1e4, 2e6], capacity 256);
    factors n in [8, 128], kappa log-uniform in [1e2, 1e14]; appends of 4..32
    columns; 50/50 mix.  The requests are first served one at a time (each
    submitted when the previous completed) to measure their mean service
    time S; the arrival process is then scaled to mean gap S / utilization
    and replayed in real time on fresh bases.  Latency = completion -
    submission.  Then the same stream is submitted all at once, for the
    runtime's capacity (rows*cols/s at saturation)."""
    import numpy as np
    from paper_2507_07788_gb300 import serve_driver as sd
    t0 = time.perf_counter()
    wl = sd.make_workload(n_bases=64, n_requests=n_requests, mean_gap_s=1.0, seed=0)
    sd.make_payloads(wl, seed=0)
    gen_s = time.perf_counter() - t0

    def server():
        return cq.Server(slots=4, batch_max=16, hbm_budget_bytes=16 << 30, small_rows=262144)

    bases = sd.make_bases(cq, wl)
    srv = server()
    sd.run_alone(cq, srv, bases, wl)
    srv.close()
    for b in bases:
        b.close()
    alone = sd.service_times(wl)
    s_mean = float(alone.mean())
    gap = s_mean / utilization
    sd.scale_arrivals(wl, gap)
    bases = sd.make_bases(cq, wl)
    srv = server()
    info = sd.replay(cq, srv, bases, wl, realtime=True)
    srv.close()
    st = sd.latency_stats(wl)
    st.update(info)
    for b in bases:
        b.close()
    # capacity: the same stream submitted all at once (no arrival gaps)
    bases = sd.make_bases(cq, wl)
    srv = server()
    sd.replay(cq, srv, bases, wl, realtime=False)
    srv.close()
    sat = sd.latency_stats(wl)
    st["saturated"] = {"rows_cols_per_s": sat["rows_cols_per_s"], "makespan_s": sat["makespan_s"],
                       "batched": sat["batched"], "max_batch": sat["max_batch"]}
    st["utilization"] = utilization
    st["alone"] = {"mean_ms": s_mean * 1e3, "p50_ms": float(np.percentile(alone, 50) * 1e3),
                   "p99_ms": float(np.percentile(alone, 99) * 1e3)}
    st["mean_gap_ms"] = gap * 1e3
    st["workload"] = (f"{n_requests} requests, Poisson arrivals at mean gap = mean service time alone / "
                      f"{utilization}, 64 bases m log-uniform [1e4, 2e6], factor n U[8,128] kappa "
                      "logU[1e2,1e14] / append p U[4,32], 50/50, FP64")
    st["arrival_span_s"] = wl.reqs[-1].arrival
    st["setup_s"] = gen_s
    st["factors"] = sum(1 for r in wl.reqs if r.kind == "factor")
    for b in bases:
        b.close()
    for r in wl.reqs:
        r.payload = None
    torch.cuda.empty_cache()
    return st


def run_ours(args):
    import numpy as np
    import torch

    import paper_2507_07788_gb300 as cq
    from paper_2507_07788_gb300 import _build, synth

    ws, rank, local = dist()
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    _build.build()
    m, n, kappa = args.m, args.n, args.kappa
    emu = {"auto": cq.EMU_AUTO, "tcgen05": cq.EMU_TCGEN05, "off": cq.EMU_OFF}[args.emulation]
    opts = cq.default_opts(precision=cq.PREC_MIXED if args.precision == "mixed" else cq.PREC_FP64,
                           emulation=emu)

    A = synth.test_matrix(m, n, kappa, rep=rank)
    dA = cq.to_colmajor(A)
    dQ = cq.colmajor(m, n)
    dR = cq.colmajor(n, n)

    for _ in range(args.warmup):
        cq.factor(dA, Q=dQ, R=dR, opts=opts)
    cq.cqr_timing_reset()
    cq.cqr_timing_enable(True)
    clocks = Clocks(local)
    clocks.start()
    # keep the GPU busy (untimed) until the sampler has written its first
    # line, so that samples cover the timed region
    t_wait = time.time()
    while not clocks.has_sample() and time.time() - t_wait < 5.0:
        cq.factor(dA, Q=dQ, R=dR, opts=opts)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start = time.time()
    e0.record(s)
    res = None
    for _ in range(args.steps):
        res = cq.factor(dA, Q=dQ, R=dR, opts=opts)
    e1.record(s)
    torch.cuda.synchronize()
    t_end = time.time()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop(window=(t_start, t_end))
    cq.cqr_timing_enable(False)
    tm = cq.cqr_timing_read()
    ms, value = replica_throughput(e0.elapsed_time(e1) / args.steps, ws, m, n, "cuda")

    # quality of the timed result (outside the timed region)
    G = dQ.t() @ dQ
    loo_f = float(torch.linalg.norm(G - torch.eye(n, dtype=G.dtype, device=G.device)))

    hbm_peak, hbm_src, tc_peak, tc_src = peaks()
    roof = roofline_from(tm, m, n, hbm_peak, hbm_src, tc_peak, tc_src, emulation=args.emulation)

    hbm = factorisation_hbm(m, n, res.info["iters"], ms, hbm_peak)
    line = {"metric": METRIC, "value": value, "unit": "rows*cols/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"sCholQR3 FP64 m={m} n={n} kappa={kappa:g} (A=U diag(s) V^T, Sec. 4.1)",
                       "m": m, "n": n, "kappa": kappa, "precision": args.precision,
                       "emulation": args.emulation,
                       "l2": f"inputs larger than L2 ({8 * m * n / 2**20:.0f} MiB per matrix)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": roof, "hbm_frac": hbm["frac"], "factorisation_hbm": hbm,
            "gpu_launches": int(tm["kernel_launches"]),
            "quality": {"status": res.status, "iters": res.info["iters"], "loo_frob": loo_f,
                        "orth_frob_last_gram": res.info["orth_frob"], "shifts": res.info["shifts"]},
            "clocks": clk}

    if rank == 0 and not args.no_e2e:
        Ah = torch.from_numpy(np.asfortranarray(A)).t().contiguous().pin_memory().t()
        Qh = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
        Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        for _ in range(2):
            cq.factor_host(Ah, Q=Qh, R=Rh, opts=opts)
        t0 = time.perf_counter()
        k = max(2, args.steps // 2)
        for _ in range(k):
            r2 = cq.factor_host(Ah, Q=Qh, R=Rh, opts=opts)
        dt = (time.perf_counter() - t0) / k
        line["e2e"] = {"value": m * n / dt, "unit": "rows*cols/s", "h2d_bytes_per_step": 8 * m * n,
                       "d2h_bytes_per_step": 8 * (m * n + n * n), "ms_per_step": dt * 1e3,
                       "api": "cholqr_factor_host (pinned host A, Q, R allocated once; H2D + factor + D2H in the timed region)"}

    if rank == 0 and not args.no_tcgen05_leg and args.emulation != "tcgen05":
        # the same factorisation with the tcgen05 Gramian and solve
        o5 = cq.default_opts(precision=opts.precision, emulation=cq.EMU_TCGEN05)
        t5, r5 = time_factor(cq, torch, dA, dQ, dR, o5, 10, 3)
        line["tcgen05_leg"] = {"workload": f"the headline factorisation with emulation TCGEN05 (tcgen05 Gramian "
                                           f"and solve for 17 <= n <= 64)", "ms": t5,
                               "rows_cols_per_s": m * n / (t5 * 1e-3), "iters": r5.info["iters"],
                               "status": r5.status, "vs_default": ms / t5}

    if rank == 0 and not args.no_sweep:
        sweep = []
        for nn in (16, 32, 64):
            for kap in (1e4, 1e8, 1e12, 1e15):
                As = synth.test_matrix(m, nn, kap, rep=11)
                dAs, dQs, dRs = cq.to_colmajor(As), cq.colmajor(m, nn), cq.colmajor(nn, nn)
                tms, rs = time_factor(cq, torch, dAs, dQs, dRs, opts, 3, 1)
                sweep.append({"n": nn, "kappa": kap, "ms": tms, "rows_cols_per_s": m * nn / (tms * 1e-3),
                              "iters": rs.info["iters"], "status": rs.status,
                              "orth_frob": rs.info["orth_frob"]})
                del dAs, dQs, dRs
        line["sweep"] = sweep

    if rank == 0 and not args.no_update:
        line["update"] = leg_update(cq, torch, args.update_m, hbm_peak=hbm_peak)
        fp64 = leg_update(cq, torch, args.update_m, cache=False, hbm_peak=hbm_peak)
        line["update"]["without_cache"] = {k: fp64[k] for k in ("ms_per_append_mean", "ms_per_append_last",
                                                                 "rows_cols_per_s", "max_block_orth_frob", "hbm")}

    if rank == 0 and not args.no_mixed:
        line["mixed"] = leg_mixed(cq, torch, synth, args.mixed_m, hbm_peak=hbm_peak)

    if rank == 0 and not args.no_pn:
        line["pn"] = leg_pn(cq, torch, synth, m)

    if rank == 0 and not args.no_wide:
        line["wide"] = leg_wide(cq, torch, synth, hbm_peak=hbm_peak)

    if rank == 0 and not args.no_serve:
        line["serve"] = leg_serve(cq, torch, args.serve_requests)

    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(A, min(args.cpu_rows, m), n, min(args.cpu_rows_all_cores, m))

    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
