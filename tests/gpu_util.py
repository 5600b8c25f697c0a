"""Helpers shared by the GPU parity tests (inputs from datagen, expected values
from the oracle, results through the C ABI via the Python binding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def have_gpu():
    return torch.cuda.is_available()


def dev(ss):
    import paper_2404_16517_gb300 as sss
    return sss.to_device(ss)


def u32(t):
    return t.cpu().numpy().view(np.uint32)
