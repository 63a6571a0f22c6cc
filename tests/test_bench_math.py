"""The bench's algorithmic byte counts, checked on the CPU against closed forms.

The Strassen-Winograd additions (Algorithm 4) write 7 operands of a quarter
of the parent's size per level and per side.  The library fuses two levels
per launch where it can: splits top-down (levels 1-2, then 3-4, ...; a single
last level when the depth is odd), combines bottom-up (levels d..d-1, ...; a
single level 1 when the depth is odd).  The expected totals below are those
schedules written out by hand in units of a whole operand, (M L + L N) / 8
bytes for the splits and M N / 8 for the combines.
"""
import pytest

import bench

M = L = N = 32768
SPLIT_UNIT = (M * L + L * N) / 8.0
COMB_UNIT = M * N / 8.0

# depth: (split traffic, combine traffic) in units of one operand
CLOSED = {
    0: (0.0, 0.0),
    1: (1 + 7 / 4, 7 / 4 + 1),
    2: (1 + 49 / 16, 49 / 16 + 1),
    3: ((1 + 49 / 16) + (49 / 16 + 343 / 64), (343 / 64 + 7 / 4) + (7 / 4 + 1)),
    4: ((1 + 49 / 16) + (49 / 16 + 2401 / 256), (2401 / 256 + 49 / 16) + (49 / 16 + 1)),
    5: ((1 + 49 / 16) + (49 / 16 + 2401 / 256) + (2401 / 256 + 16807 / 1024),
        (16807 / 1024 + 343 / 64) + (343 / 64 + 7 / 4) + (7 / 4 + 1)),
}


@pytest.mark.parametrize("depth", sorted(CLOSED))
def test_strassen_stream_bytes_closed_forms(depth):
    split, comb = bench.strassen_stream_bytes(M, L, N, depth)
    es, ec = CLOSED[depth]
    assert split == pytest.approx(es * SPLIT_UNIT, rel=1e-12)
    assert comb == pytest.approx(ec * COMB_UNIT, rel=1e-12)


def test_depth4_totals_at_n32768():
    """4.43 GB of split traffic and 2.22 GB of combine traffic per product."""
    split, comb = bench.strassen_stream_bytes(M, L, N, 4)
    assert round(split / 1e9, 2) == 4.43
    assert round(comb / 1e9, 2) == 2.22


def test_rectangular_shapes_scale_per_side():
    """A side's traffic scales with that side's operand only."""
    s1, c1 = bench.strassen_stream_bytes(4096, 8192, 2048, 2)
    assert s1 == pytest.approx((1 + 49 / 16) * (4096 * 8192 + 8192 * 2048) / 8.0)
    assert c1 == pytest.approx((49 / 16 + 1) * 4096 * 2048 / 8.0)


PEAKS = {"hbm_gbs": 6780.7, "bf16_tflops": 1896.1, "sm_max_mhz": 2070.0}


def test_m4rm_roofline_counts_table_row_reads():
    """n = 32768 at depth 4: 2401 leaves of 2048^3, k = 8, so one launch
    reads 2401 * 2048^3 / 64 = 3.22e11 table bytes; at 11.47 ms that is
    28.1 TB/s of the 39.69 TB/s measured with the lookup pattern (the nominal
    152 x 128 B x 2070 MHz is 40.27 TB/s)."""
    r = bench.roofline_for("m4rm", 2401, 2048, 2048, 2048, 8, 11.47, PEAKS, "measured")
    assert r["bound"] == "smem" and r["unit"] == "GB/s"
    assert 2401 * 2048 ** 3 / 64 == pytest.approx(3.2226e11, rel=1e-4)
    assert r["peak"] == pytest.approx(39690.0)
    assert "40.3 TB/s" in r["peak_note"]
    assert r["achieved"] == pytest.approx(3.2226e11 / 11.47e-3 / 1e9, rel=1e-4)
    assert round(r["frac"], 3) == 0.708
    assert round(r["frac_of_nominal"], 3) == 0.698


def test_tc_roofline_counts_dense_flops_against_twice_bf16():
    """n = 32768 at depth 3: 343 leaves of 4096^3, 2 M L N flops each, against
    2 x the measured bf16 rate (the nominal FP8 / BF16 ratio)."""
    r = bench.roofline_for("tc_fp8", 343, 4096, 4096, 4096, 0, 21.5, PEAKS, "measured")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(3792.2)
    assert r["achieved"] == pytest.approx(2.0 * 4096 ** 3 * 343 / 21.5e-3 / 1e12)
    assert round(r["frac"], 2) == 0.58


def test_fp4_roofline_is_six_times_bf16():
    """FP4 against 6 x the measured bf16 rate (nominal 13.5 vs 2.25 PFLOP/s)."""
    r = bench.roofline_for("tc_fp4", 49, 8192, 8192, 8192, 0, 10.0, PEAKS, "measured")
    assert r["peak"] == pytest.approx(6 * 1896.1)
    assert r["achieved"] == pytest.approx(2.0 * 8192 ** 3 * 49 / 10.0e-3 / 1e12)


def test_expansion_bytes():
    """FP8: one byte per entry (K rounded up to 128); FP4: half a byte (K
    rounded up to 256); plus the packed leaves read once."""
    assert bench.expand_bytes("tc_fp8", 1, 128, 100, 256) == pytest.approx((384 * 100) / 8 + 384 * 128)
    assert bench.expand_bytes("tc_fp4", 2, 128, 300, 256) == pytest.approx(2 * ((384 * 300) / 8 + 384 * 512 * 0.5))
    assert bench.expand_bytes("m4rm", 1, 128, 100, 256) == 0.0


def test_code_sha_ignores_comments_but_not_code(tmp_path):
    """The key that keeps a DRAM-traffic capture valid follows the kernel's
    code only: comment and blank-line edits keep it, code edits change it."""
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// header\nint f(int x) { return x ^ 1; }  // tail\n")
    b.write_text("/* another\n   header */\n\nint f(int x) { return x ^ 1; }\n")
    c.write_text("// header\nint f(int x) { return x ^ 3; }  // tail\n")
    assert bench.code_sha([str(a)]) == bench.code_sha([str(b)])
    assert bench.code_sha([str(a)]) != bench.code_sha([str(c)])


def test_recorded_traffic_key_matches_the_kernel_sources():
    ent = bench.NCU_TRAFFIC["m4rm"]
    assert bench.code_sha(ent["sources"]) == ent["sha"]


def test_clock_summary_keeps_the_timed_region():
    """Samples outside [t0, t1] (the warm-up, the tail) are left out; a
    throttle reason seen inside the region is reported."""
    import datetime
    base = datetime.datetime(2026, 12, 4, 3, 0, 0)

    def line(dt_ms, mhz, pwr_cap="Not Active", hw="Not Active"):
        ts = (base + datetime.timedelta(milliseconds=dt_ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return "%s, 0, %d, 2070, 900.0, 0x0, %s, Not Active, Not Active, %s" % (ts, mhz, hw, pwr_cap)

    cs = bench.ClockSampler(0)
    cs.lines = [line(0, 1200), line(20, 1300, hw="Active"),               # warm-up
                line(100, 2070), line(120, 2055, pwr_cap="Active"), line(140, 2070),
                line(300, 1000)]                                        # after the region
    t0 = (base + datetime.timedelta(milliseconds=90)).timestamp()
    t1 = (base + datetime.timedelta(milliseconds=150)).timestamp()
    s = cs.summary(t0, t1)
    assert s["samples"] == 3 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    whole = cs.summary()
    assert whole["samples"] == 6 and "hw_slowdown" in whole["reasons"]


def test_batched_table_bytes_follow_each_row_block_k():
    """m*l*n/(8k) per product; split variants count the tall row blocks
    (full 1024-row blocks, and the last one when it keeps the threshold's
    rows) at k = 8 and the rest at the slot kernel's k."""
    dims = [(1100, 64, 128), (1300, 64, 128), (200, 64, 128)]
    b, _ = bench.batched_table_bytes("slots-k4t8-bm256", dims)
    assert b == pytest.approx(sum(m * l * n for m, l, n in dims) / 32.0)
    b, _ = bench.batched_table_bytes("tall-k8t4-bm512-from256+slots-k4t8-bm128", dims)
    # 1100: 1024 tall + 76 rest; 1300: all tall (276 >= 256); 200: all rest
    want = (1024 * 64 * 128 / 64 + 76 * 64 * 128 / 32 + 1300 * 64 * 128 / 64 + 200 * 64 * 128 / 32)
    assert b == pytest.approx(want)
    b, _ = bench.batched_table_bytes("tall-k8t4-bm512-from512+slots-k4t8-bm256", dims)
    want = (1024 * 64 * 128 / 64 + 76 * 64 * 128 / 32 + 1024 * 64 * 128 / 64 + 276 * 64 * 128 / 32
            + 200 * 64 * 128 / 32)
    assert b == pytest.approx(want)


def test_strassen_bytes_with_leaves_written_expanded():
    """When the last level of additions writes the leaves expanded (FP4: half
    a byte per entry instead of an eighth), only that level's writes grow,
    by 4x; the parents read and the other levels stay packed."""
    M = L = N = 32768
    packed, comb = bench.strassen_stream_bytes(M, L, N, 2)
    fused, comb2 = bench.strassen_stream_bytes(M, L, N, 2, 0.5)
    leaves_packed = 49 * (M * L + L * N) / 16 / 8.0
    level1 = 7 * (M * L + L * N) / 4 / 8.0
    assert comb2 == comb
    # depth 2 fused: level 1 is written and read back packed, then the
    # leaves are written expanded (4x their packed bytes)
    assert fused - packed == pytest.approx(2 * level1 + leaves_packed * 3)
    # depth 3: levels 1-2 fused in one launch, level 3 alone writes the leaves
    p3, _ = bench.strassen_stream_bytes(M, L, N, 3)
    f3, _ = bench.strassen_stream_bytes(M, L, N, 3, 1.0)
    assert f3 - p3 == pytest.approx(343 * (M * L + L * N) / 64 / 8.0 * 7)
