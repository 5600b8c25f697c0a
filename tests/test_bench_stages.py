"""Stage-level algorithmic-byte efficiency in the benchmark line, and the DRAM
traffic it reports only for the library source the capture was taken on (host
logic)."""
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


def test_known_traffic_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    b = bench()
    csrc = tmp_path / "paper_2404_16517_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    h = b.lib_source_hash()
    t = tmp_path / "profiles" / "traffic.json"
    t.write_text('{"source_hash": "%s", "kernels": {"ls_lg_ext": 1234}}' % h)
    assert b.known_traffic("ls_lg_ext") == 1234
    assert b.known_traffic("pd_hash") is None  # not captured
    (csrc / "k.cu").write_text("__global__ void k() { }\n")  # the source changed since the capture
    assert b.lib_source_hash() != h
    assert b.known_traffic("ls_lg_ext") is None
    t.write_text("not json")
    assert b.known_traffic("ls_lg_ext") is None
