"""Stage-level algorithmic-byte efficiency in the benchmark line (host logic)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_stage_rooflines_groups_kernels_and_applies_the_byte_model():
    b = bench()
    km = {"ls_lg_ext": 0.5, "ls_finish_cta": 0.25, "dist": 0.25, "pd_hash": 0.4, "pd_retire": 0.1,
          "c_bounds": 0.05, "d2_cta": 0.2, "d_scan": 0.05, "d2_records": 0.25, "sum_tlen": 0.01}
    n, D, Da, sl = 1000, 400_000, 500_000, 380_000
    st = b.stage_rooflines(km, n, D, Da, sl, 1000.0)
    assert st["A"]["ms"] == pytest.approx(1.0)
    assert st["B"]["ms"] == pytest.approx(0.5)
    assert st["C"]["ms"] == pytest.approx(0.05)
    assert st["D"]["ms"] == pytest.approx(0.5)
    assert st["other"]["ms"] == pytest.approx(0.01)
    assert st["A"]["algorithmic_bytes"] == D + 32 * n
    assert st["B"]["algorithmic_bytes"] == Da + 16 * n
    assert st["D"]["algorithmic_bytes"] == 3 * ((Da - sl) + 8 * n) + 8 * n
    assert st["C"]["algorithmic_bytes"] is None and st["C"]["frac"] is None
    # A: 432,000 bytes in 1 ms = 0.432 GB/s against a 1000 GB/s peak
    assert st["A"]["achieved_gbs"] == pytest.approx(0.432)
    assert st["A"]["frac"] == pytest.approx(0.432 / 1000.0)
