"""The roofline arithmetic of bench.py on CPU, from synthetic per-launch
timings: the dominant kernel is the one with the larger total time, its
achieved HBM rate is the algorithmic bytes of one launch over the mean launch
time against the measured HBM peak (its tensor or FP64 rate nested), its DRAM
traffic is the committed ncu capture scaled by rows, and the whole
factorisation moves 8 m n + 16 m n bytes per pass."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")

KEYS = ("sweep", "fused", "solve", "gram", "tsolve")


def _timing(**kw):
    tm = {}
    for k in KEYS:
        tm[f"{k}_launches"] = 0
        for f in ("ms", "flops", "bytes"):
            tm[f"{k}_{f}"] = 0.0
    tm["tsolve_tc_flops"] = 0.0
    tm.update(kw)
    return tm


def _capture(name):
    d = {}
    for line in open(os.path.join(ROOT, "profiles", f"traffic_{name}.txt")):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            d[k.strip()] = v.strip()
    return float(d["capture_bytes_per_launch"]), float(d["capture_rows"]), float(d.get("capture_cols", 0))


def _check_traffic(traffic, name, rows, n=None):
    # the committed capture scaled by rows (and columns, when the capture
    # names its width), or None while the kernel's sources differ from the
    # captured ones (or no capture exists)
    if traffic is None:
        return
    b, cr, cc = _capture(name)
    want = b * rows / cr * ((n / cc) if (n and cc) else 1.0)
    assert traffic == pytest.approx(want, rel=1e-12)


def test_tensor_pipeline_dominant_kernel():
    # 24 launches each of the digit Gramian and the digit solve on row chunks
    # of 125000 rows at n = 64; the Gramian takes longer in total
    n, rows, L = 64, 125000, 24
    g_ms, s_ms = 0.20, 0.18
    tc_solve_per_launch = 3.0e10
    tm = _timing(gram_launches=L, gram_ms=L * g_ms, gram_flops=L * rows * n * (n + 1.0),
                 gram_bytes=L * 8.0 * rows * n,
                 tsolve_launches=L, tsolve_ms=L * s_ms, tsolve_flops=L * rows * n * n,
                 tsolve_bytes=L * 16.0 * rows * n, tsolve_tc_flops=L * tc_solve_per_launch)
    r = bench.roofline_from(tm, 1_000_000, n, 6686.8, "measured", 1730.8, "measured", emulation="tcgen05")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6686.8
    assert r["kernel"].startswith("tcgram64_kernel") and r["solve"]["kernel"].startswith("tcgemm64_kernel")
    # by default the Gramian runs on tcgen05 from n = 33, the solve on mma.sync
    r0 = bench.roofline_from(tm, 1_000_000, n, 6686.8, "measured", 1730.8, "measured")
    assert r0["kernel"].startswith("tcgram64_kernel") and r0["solve"]["kernel"].startswith("ozgemm_kernel")
    r32 = bench.roofline_from(tm, 1_000_000, 32, 6686.8, "measured", 1730.8, "measured")
    assert r32["kernel"].startswith("ozgram_kernel")
    assert bench.tc05_kernels("auto", 33) == (True, False) and bench.tc05_kernels("auto", 32) == (False, False)
    assert bench.tc05_kernels("tcgen05", 17) == (True, True) and bench.tc05_kernels("tcgen05", 65) == (False, False)
    assert bench.tc05_kernels("off", 64) == (False, False)
    # 8 bytes per entry read, in 0.2 ms
    gbs = 8.0 * rows * n / (g_ms * 1e-3) / 1e9
    assert r["achieved"] == pytest.approx(gbs, rel=1e-12)
    assert r["frac"] == pytest.approx(gbs / 6686.8, rel=1e-12)
    # 16 symmetric digit pairs, each a 64 x 64 block per row, in 0.2 ms
    want = rows * 2 * 16 * 64 * 64 / (g_ms * 1e-3) / 1e12
    assert r["tensor"]["achieved"] == pytest.approx(want, rel=1e-12)
    assert r["tensor"]["frac"] == pytest.approx(want / 1730.8, rel=1e-12)
    _check_traffic(r["traffic"], "tcgram", rows, n)
    s = r["solve"]
    assert s["achieved"] == pytest.approx(16.0 * rows * n / (s_ms * 1e-3) / 1e9, rel=1e-12)
    assert s["tensor"]["achieved"] == pytest.approx(tc_solve_per_launch / (s_ms * 1e-3) / 1e12, rel=1e-12)
    _check_traffic(s["traffic"], "tcgemm", rows, n)


def test_solve_dominates_when_it_takes_longer():
    n, rows, L = 128, 62500, 16
    tm = _timing(gram_launches=L, gram_ms=L * 0.1, gram_flops=L * rows * n * (n + 1.0),
                 gram_bytes=L * 8.0 * rows * n,
                 tsolve_launches=L, tsolve_ms=L * 0.3, tsolve_flops=L * rows * n * n,
                 tsolve_bytes=L * 16.0 * rows * n, tsolve_tc_flops=L * 5.0e10)
    r = bench.roofline_from(tm, 1_000_000, n, 6686.8, "measured", 1730.8, "measured")
    assert r["kernel"].startswith("ozgemm_kernel") and "gram" in r
    assert r["achieved"] == pytest.approx(16.0 * rows * n / 0.3e-3 / 1e9, rel=1e-12)
    assert r["tensor"]["achieved"] == pytest.approx(5.0e10 / 0.3e-3 / 1e12, rel=1e-12)
    # the Gramian at n = 128: 16 pairs of 128 x 128 blocks per row
    assert r["gram"]["tensor"]["achieved"] == pytest.approx(rows * 2 * 16 * 128 * 128 / 0.1e-3 / 1e12,
                                                            rel=1e-12)


def test_narrow_blocks_report_the_fp64_solve():
    n, rows, L = 16, 125000, 8
    tm = _timing(gram_launches=L, gram_ms=L * 0.05, gram_flops=L * rows * n * (n + 1.0),
                 gram_bytes=L * 8.0 * rows * n,
                 solve_launches=L, solve_ms=L * 0.04, solve_flops=L * rows * n * n,
                 solve_bytes=L * 16.0 * rows * n)
    r = bench.roofline_from(tm, 1_000_000, n, 6686.8, "measured", 1730.8, "measured")
    assert r["bound"] == "hbm" and r["kernel"].startswith("trsm_rows_kernel")
    assert r["achieved"] == pytest.approx(16.0 * rows * n / 0.04e-3 / 1e9, rel=1e-12)
    assert r["alu"]["achieved"] == pytest.approx(rows * n * n / 0.04e-3 / 1e12, rel=1e-12)
    assert r["alu"]["frac"] == pytest.approx(r["alu"]["achieved"] * 1e12 / bench.FP64_PEAK_FLOPS, rel=1e-12)
    assert "gram" in r


def test_fp64_sweep_without_tensor_kernels():
    n, m = 64, 200000
    tm = _timing(fused_launches=3, fused_ms=3 * 2.0, fused_flops=3 * 4.0 * m * n * n,
                 fused_bytes=3 * 16.0 * m * n)
    r = bench.roofline_from(tm, m, n, 6686.8, "measured", 1730.8, "measured")
    assert r["bound"] == "hbm" and r["kernel"].startswith("rowsweep_kernel")
    assert r["achieved"] == pytest.approx(16.0 * m * n / 2.0e-3 / 1e9, rel=1e-12)
    assert r["alu"]["achieved"] == pytest.approx(4.0 * m * n * n / 2.0e-3 / 1e12, rel=1e-12)


def test_whole_factorisation_bytes():
    # 3 passes at m = 1e6, n = 64: 56 m n bytes
    h = bench.factorisation_hbm(1_000_000, 64, 3, 6.5, 6686.8)
    assert h["bytes"] == 56.0 * 1_000_000 * 64
    assert h["frac"] == pytest.approx(56.0 * 64e6 / 6.5e-3 / 1e9 / 6686.8, rel=1e-12)


def test_append_bytes_follow_alg2_sweeps():
    # the first sweep reads [Q_in A_in]; each outer iteration reads [Q_in Y]
    # and writes the new block
    m, q, p = 1000, 16, 8
    assert bench.append_hbm_bytes(m, q, p, 0) == 8.0 * m * (q + p)
    assert bench.append_hbm_bytes(m, q, p, 2) == 8.0 * m * (q + p) + 2 * (8.0 * m * (q + p) + 8.0 * m * p)
    assert bench.append_hbm_bytes(m, 0, p, 1) == 8.0 * m * p + 16.0 * m * p


def test_kernel_hash_ignores_comments_only():
    # a comment or blank-line change keeps a capture's counters valid; a
    # change of code does not
    a = "int x; // old note\n/* a block\n   comment */\nint y;\n"
    b = "int x;   // new note\n\nint y;  /* another */\n"
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments("int x = 1;") != bench.strip_comments("int x = 2;")

