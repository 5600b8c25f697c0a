"""Autotuner host logic (no GPU): candidate grid validity, instance sampling,
workload signatures and the JSON cache."""
import os

from paper_2404_16517_gb300 import autotune


def test_candidates_valid_and_complete():
    c = autotune.candidates()
    assert c and all(x["direct_cap"] >= x["cta_cap"] for x in c)
    assert len(c) == len({tuple(sorted(x.items())) for x in c})
    assert {"cta_cap": 2048, "direct_cap": 8192, "bucket_target": 2048, "warp_cap": 32} in c
    small = autotune.candidates({"cta_cap": [512, 2048], "direct_cap": [1024, 8192]})
    assert sorted((x["cta_cap"], x["direct_cap"]) for x in small) == [(512, 1024), (512, 8192), (2048, 8192)]


def test_sample_instances_keeps_mix():
    sizes = [64, 65536, 100, 4000] * 50
    first = [sum(sizes[:i]) for i in range(len(sizes))]
    f, n = autotune.sample_instances(first, sizes, max_strings=sum(sizes) // 4)
    assert sum(n) <= sum(sizes) // 4
    assert set(n) == set(sizes)
    assert f == sorted(f)
    assert all(sizes[first.index(a)] == b for a, b in zip(f, n))


def test_signature_and_cache(tmp_path):
    k = autotune.signature("batch", 37478670, 5772285035, 4096)
    assert k == "batch:n2^25:N2^32:m2^12"
    p = os.path.join(tmp_path, "tune.json")
    assert autotune.cached(p, k, device_name="GPU X") is None
    autotune.store(p, k, {"cta_cap": 1024}, device_name="GPU X")
    autotune.store(p, "other", {"warp_cap": 16}, device_name="GPU Y")
    assert autotune.cached(p, k, device_name="GPU X") == {"cta_cap": 1024}
    assert autotune.cached(p, k, device_name="GPU Y") is None
