"""The host generators follow the input recipes the benchmarks state (no GPU):
config 1 and 2 template sets (lengths, alphabet, the shared template prefix,
uniform picks), a bounded sample equal to the same strings of the full set,
config 3 suffix views (distinct offsets, truncation to 256, views into one
text over 64 symbols), config 4 instance sizes and lengths, and config 5
request sizes."""
import numpy as np

import datagen


def _rows(ss):
    return ss.chars.reshape(ss.n, -1)


def test_config2_template_recipe_on_a_sample():
    ss = datagen.config2(count=4096)
    assert ss.n == 4096 and set(ss.lens.tolist()) == {500}
    assert np.array_equal(ss.offs, np.arange(4096, dtype=np.uint64) * 500)
    rows = _rows(ss)
    assert rows.min() >= ord("A") and rows.max() <= ord("Z")
    heads = {bytes(r[:242]) for r in rows}
    assert len(heads) == 64  # chars 0-241 come from one of 64 templates (4096 picks hit all 64)
    # the rest is uniform: character frequencies past the prefix near 1/26
    tail = rows[:, 242:].ravel()
    freq = np.bincount(tail - ord("A"), minlength=26) / tail.size
    assert np.all(np.abs(freq - 1 / 26) < 0.01)
    # strings sharing a template agree exactly on the 242 characters and, past
    # them, match the template no more often than chance
    by_head = {}
    for r in rows:
        by_head.setdefault(bytes(r[:242]), []).append(r)
    same = [g for g in by_head.values() if len(g) > 1][0]
    assert bytes(same[0][:242]) == bytes(same[1][:242]) and bytes(same[0][242:]) != bytes(same[1][242:])


def test_bounded_sample_equals_the_full_set_strings():
    a = datagen.config2(n=50000, first=1000, count=300)
    b = datagen.config2(n=50000, count=1300)
    assert np.array_equal(_rows(a), _rows(b)[1000:])


def test_config1_recipe():
    ss = datagen.config1()
    assert ss.n == 65536 and set(ss.lens.tolist()) == {100}
    rows = _rows(ss)
    assert len({bytes(r[:42]) for r in rows}) == 4
    assert rows.min() >= ord("A") and rows.max() <= ord("Z")


def test_config3_suffix_views_scaled():
    ss = datagen.config3(scale=6)  # 2^16-byte text, 2^15 suffixes
    assert ss.chars.size == 1 << 16 and ss.n == 1 << 15
    assert np.unique(ss.offs).size == ss.n  # distinct offsets
    assert not np.all(np.diff(ss.offs.astype(np.int64)) > 0)  # not in offset order
    assert np.array_equal(ss.lens, np.minimum(256, (1 << 16) - ss.offs.astype(np.int64)).astype(np.uint32))
    assert ss.chars.min() >= 0x21 and ss.chars.max() < 0x21 + 64


def test_config4_sizes_and_config5_requests():
    sizes, ratios = datagen.config4_sizes()
    assert sizes.size == 4096 and sizes.min() >= 1 << 6 and sizes.max() <= 1 << 16
    assert np.all((ratios >= 0.1) & (ratios <= 0.9))
    # sizes log-uniform: the median near 2^11
    assert 2 ** 10 < np.median(sizes) < 2 ** 12
    n, r, gaps, _ = datagen.config5_requests(count=4000)
    assert n.min() >= 1 and n.max() <= 1 << 24
    assert 2 ** 13 < np.median(n) < 2 ** 15  # lognormal sizes, median 2^14
    assert np.all((r >= 0.1) & (r <= 0.9))
    assert np.all(gaps >= 0) and abs(gaps.mean() - 1.0) < 0.06  # unit-rate exponential gaps
