"""sss_sort_host: the whole path for a string set in host memory, the upload
overlapped with the local sorts, equals the oracle's order and LCP array on
contiguous sets, overlapping suffix views with unordered offsets, one partition
and many; the host copies of the outputs equal the device outputs."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _host(ss):
    h_chars = torch.from_numpy(ss.chars if ss.chars.size else np.zeros(1, np.uint8)).pin_memory()
    h_offs = torch.from_numpy(ss.offs.view(np.int64)).pin_memory()
    h_lens = torch.from_numpy(ss.lens.view(np.int32)).pin_memory()
    return h_chars, h_offs, h_lens


@pytest.mark.parametrize("case", ["config2", "suffixes", "dna"])
@pytest.mark.parametrize("p", [1, 4, 16])
def test_sort_host_matches_oracle(case, p):
    import paper_2404_16517_gb300 as m
    if case == "config2":
        ss = datagen.config2(n=65536 * 4, count=40000)
    elif case == "suffixes":
        ss = datagen.config3(scale=7)
    else:
        rng = np.random.default_rng(3)
        alpha = np.frombuffer(b"ACGT", dtype=np.uint8)
        strs = [rng.choice(alpha, size=int(rng.integers(0, 30))).tobytes() for _ in range(20000)]
        ss = datagen.from_strings(strs + strs[:3000])
    h_chars, h_offs, h_lens = _host(ss)
    d_chars = torch.empty(h_chars.numel(), dtype=torch.uint8, device="cuda")
    d_offs = torch.empty(ss.n, dtype=torch.int64, device="cuda")
    d_lens = torch.empty(ss.n, dtype=torch.int32, device="cuda")
    h_perm = torch.full((ss.n,), -1, dtype=torch.int32).pin_memory()
    h_lcp = torch.full((ss.n,), -1, dtype=torch.int32).pin_memory()
    for _ in range(2):  # twice: the second call reuses the device buffers
        perm, lcp = m.sss_sort_host(h_chars, h_offs, h_lens, p, d_chars, d_offs, d_lens, h_out_perm=h_perm,
                                    h_out_lcp=h_lcp)
        m.context().sync()
        want = oracle.sort(ss)
        assert np.array_equal(m.u32(perm), want)
        assert np.array_equal(m.u32(lcp), oracle.lcp_array(ss, want))
        assert np.array_equal(h_perm.numpy().view(np.uint32), want)
        assert np.array_equal(h_lcp.numpy().view(np.uint32), m.u32(lcp))


def test_sort_host_equals_device_sort_full_size():
    """The 4,194,304 x 500 p = 16 workload: host-input path == device-input path."""
    import datagen.cuda as dgc
    import paper_2404_16517_gb300 as m
    chars, offs, lens = dgc.config2()
    perm, lcp, _, _ = m.sss_sort(chars, offs, lens, 16)
    h_chars = torch.empty(chars.numel(), dtype=torch.uint8).pin_memory()
    h_chars.copy_(chars)
    h_offs, h_lens = offs.cpu().pin_memory(), lens.cpu().pin_memory()
    d_chars, d_offs, d_lens = torch.empty_like(chars), torch.empty_like(offs), torch.empty_like(lens)
    perm2, lcp2 = m.sss_sort_host(h_chars, h_offs, h_lens, 16, d_chars, d_offs, d_lens)
    m.context().sync()
    assert torch.equal(perm, perm2) and torch.equal(lcp, lcp2)
