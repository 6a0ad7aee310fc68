"""Host-side checks of bench.py's accounting (no GPU): the flop count of the
radix plan, the algorithmic bytes per pass and the roofline object built from
per-pass timings."""
import math

import pytest

import bench


def test_fft_flop_count_of_the_radix_plan():
    # N = 512 = 8^3: first stage 56 / 8, the two twiddled stages (56 + 7 * 6) / 8
    assert bench.fft_flops_per_point(512) == pytest.approx(7.0 + 2 * 12.25, rel=0, abs=1e-12)
    # N = 1024 = 8^3 * 2: a radix-2 stage with one twiddle product per pair
    assert bench.fft_flops_per_point(1024) == pytest.approx(31.5 + (4 + 6) / 2, abs=1e-12)
    for n in (64, 256, 512, 1024):
        # below the radix-2 count 5 log2 N (fewer twiddle products)
        assert bench.fft_flops_per_point(n) < 5 * math.log2(n)


def test_pass_bytes_match_the_lattices_each_pass_touches():
    b = bench.PASS_BYTES
    # pass A: W and psi in, psi and W out, plus the per-site update input:
    # {A, B dtau} (complex128, 16 B), V as a double-float pair (8 B), V in FP32 (4 B)
    assert b["c128"]["update_x"] == 4 * 16 + 16
    assert b["df64"]["update_x"] == 4 * 16 + 8
    assert b["c64"]["update_x"] == 4 * 8 + 4
    for p in ("fwd_y", "z_kinetic", "inv_y"):
        assert b["c128"][p] == b["df64"][p] == 2 * 16 and b["c64"][p] == 2 * 8
    step = {k: sum(b[k][p] for p in ("update_x", "fwd_y", "z_kinetic", "inv_y")) for k in b}
    assert step == {"c128": 176.0, "df64": 168.0, "c64": 84.0}


@pytest.mark.parametrize("prec", ["c128", "df64", "c64"])
def test_roofline_object(prec):
    per_pass = {"update_x": {"launches": 10, "total_ms": 150.0}, "fwd_y": {"launches": 10, "total_ms": 66.0},
                "z_kinetic": {"launches": 10, "total_ms": 143.0}, "inv_y": {"launches": 10, "total_ms": 66.0}}
    peaks = {"hbm_gbs": 6800.0}
    alu = {"fp64_tflops": 1.2, "fp32_tflops": 70.0, "source": "test"}
    r = bench.roofline_for(prec, per_pass, peaks, alu)
    assert r["kernel"] == "update_x"
    sites = float(bench.N) ** 3
    assert r["avg_launch_ms"] == pytest.approx(15.0)
    assert r["algorithmic_bytes_per_launch"] == bench.PASS_BYTES[prec]["update_x"] * sites
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    if prec == "c128":
        assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == 1.2
        assert r["achieved"] == pytest.approx(bench.pass_flops(bench.N)["update_x"] * sites / 15e-3 / 1e12)
    else:
        assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6800.0
        assert r["achieved"] == pytest.approx(bench.PASS_BYTES[prec]["update_x"] * sites / 15e-3 / 1e9)
    per_site = bench.DRAM_BYTES_PER_SITE.get((prec, "update_x"))
    assert r["traffic"] == (pytest.approx(per_site * sites) if per_site else None)
    assert r["share_of_step"] == pytest.approx(150.0 / 425.0)
    mb = bench.PASS_A_MIN_BYTES[prec]
    assert r["hbm_frac_at_min_bytes"]["frac"] == pytest.approx(mb * sites / 15e-3 / 1e9 / 6800.0)


def test_step_hbm_fraction():
    # arithmetic only: a synthetic step time in, the design bytes over it out
    peaks = {"hbm_gbs": 6800.0}
    sites = float(bench.N) ** 3
    t_ms = 2.5  # synthetic input, not a measurement
    r = bench.step_hbm("c64", t_ms, peaks)
    per_site = sum(bench.PASS_BYTES["c64"][p] for p in ("update_x", "fwd_y", "z_kinetic", "inv_y"))
    assert r["bytes_per_site"] == per_site
    assert r["achieved_gbs"] == pytest.approx(per_site * sites / (t_ms * 1e-3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved_gbs"] / 6800.0)
