"""Host logic of bench.py's roofline objects (no GPU): each ceiling is the
measured probe rate divided by the work per sample, the fraction is the
achieved rate over that ceiling, and every timed kernel class has a DRAM
bytes-per-sample figure for its traffic."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

RATES = {"smem_atomic_conflict_free": 9.6e12, "smem_atomic_random": 2.8e12,
         "tex_gather_coherent_l1": 6.0e11, "tex_gather_coherent_l2": 5.9e11, "l2_sector_gather_gbs": 5000.0}


def test_matched_transpose_ceilings():
    r = bench.roofline_bp(2.0e11, 1.0, RATES)            # 2e11 samples in 1 s
    assert r["peak_samples_per_s"] == pytest.approx(9.6e12 / 8)
    assert r["frac"] == pytest.approx(2.0e11 / (9.6e12 / 8))
    assert r["random_scatter_peak"] == pytest.approx(2.8e12 / 8 / 1e9)
    s = bench.roofline_bp_split(2.0e11, 2.0, RATES)      # two words per product: 16 atomics per sample
    assert s["peak_samples_per_s"] == pytest.approx(9.6e12 / 16)
    assert s["frac"] == pytest.approx(1.0e11 / (9.6e12 / 16))


def test_projector_ceiling_is_two_gathers_per_sample():
    r = bench.roofline_fp(3.0e11, 1.0, RATES)
    assert r["peak_samples_per_s"] == pytest.approx(3.0e11)
    assert r["frac"] == pytest.approx(1.0)
    assert r["l2_random_gather_peak"] == pytest.approx(5000.0e9 / 32 / 1e9)


def test_every_timed_class_has_a_traffic_figure():
    assert set(bench.DRAM_BYTES_PER_SAMPLE) == {"fp_interp", "bp_matched", "bp_matched_split"}
    # the projector moves the volume and the projections once: well under a byte per sample;
    # the transposes read their rays' set-up table from every brick a ray passes near
    assert bench.DRAM_BYTES_PER_SAMPLE["fp_interp"] < 0.05
    assert 0.1 < bench.DRAM_BYTES_PER_SAMPLE["bp_matched"] < 5.0
