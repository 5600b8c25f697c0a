"""The device generator reproduces the numpy generator byte for byte (inputs of
the GPU benchmark and of the oracle baseline are the same strings)."""
import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_config1_identical():
    import datagen.cuda as dgc
    c, o, l = dgc.config1()
    ss = datagen.config1()
    assert np.array_equal(c.cpu().numpy(), ss.chars)
    assert np.array_equal(o.cpu().numpy().view(np.uint64), ss.offs)
    assert np.array_equal(l.cpu().numpy().view(np.uint32), ss.lens)


def test_config2_slices_identical():
    import datagen.cuda as dgc
    for first, count in ((0, 3000), (4194304 - 2000, 2000), (1234567, 777)):
        c, o, l = dgc.config2(4194304, first, count)
        ss = datagen.config2(4194304, first, count)
        assert np.array_equal(c.cpu().numpy(), ss.chars)
        assert np.array_equal(l.cpu().numpy().view(np.uint32), ss.lens)


def test_device_skew_set_identical():
    import datagen.cuda as dgc
    ss = datagen.skew_set(6, 5000)
    c, o, l = dgc.skew_set(6, 5000)
    assert np.array_equal(c.cpu().numpy()[:ss.N], ss.chars)
    assert np.array_equal(o.cpu().numpy().view(np.uint64), ss.offs)
    assert np.array_equal(l.cpu().numpy().view(np.uint32), ss.lens)
