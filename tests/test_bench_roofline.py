"""The algorithmic work per launch that bench.py divides by the measured
launch time: the per-unit figures must be those the measurement states.
For 512 stations x 10 timeslots x 4 channels:
  - factorisation: P^3 / 3 flops at P = 8N;
  - statistics pass: 40 B per visibility in float32, 80 B in float64;
  - running-residual update: 72 B per visibility in float32;
  - triangular solves: the padded factor read once;
and the FP32 FMA figure is SMs x 128 lanes x 2 flops x clock.
No GPU: the launch time is set to one second and the SM count is fixed."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402
from paper_1910_13908_gb300 import synth  # noqa: E402

PK = {"hbm_gbs": 6793.4, "sm_max_mhz": 2070.0}


@pytest.fixture
def ska512(monkeypatch):
    monkeypatch.setattr(bench, "sm_count", lambda: 152)
    spec = synth.config("c4")
    assert (spec.N, spec.T, spec.F, spec.B) == (512, 10, 4, 130816)
    return spec


def one_second(kind, spec, prec):
    # one launch of 1000 ms: `achieved` is then the work in the line's unit
    return bench.roofline_for(kind, spec, prec, 5, 10, 1, 1000.0, PK, "measured")


def test_fp32_fma_figure(ska512):
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(80.54784)


def test_factorisation_counts_p_cubed_over_three(ska512):
    r = one_second("cholesky", ska512, sc.SC_MIXED)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] * 1e12 == pytest.approx(4096 ** 3 / 3)
    assert r["peak"] == pytest.approx(80.54784)


def test_statistics_pass_reads_forty_bytes_a_visibility(ska512):
    vis = 130816 * 10 * 4
    r = one_second("lm_stats", ska512, sc.SC_MIXED)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] * 1e9 == pytest.approx(40 * vis)
    assert one_second("lm_stats", ska512, sc.SC_FP64)["achieved"] * 1e9 == pytest.approx(80 * vis)


def test_running_residual_moves_seventy_two_bytes_a_visibility(ska512):
    vis = 130816 * 10 * 4
    r = one_second("vis_pass", ska512, sc.SC_MIXED)
    assert r["achieved"] * 1e9 == pytest.approx(72 * vis)
    assert r["peak"] == PK["hbm_gbs"]


def test_triangular_solve_reads_the_padded_factor(ska512):
    r = one_second("tri_solve", ska512, sc.SC_MIXED)
    assert r["achieved"] * 1e9 == pytest.approx(4096 * 4096 * 4)

