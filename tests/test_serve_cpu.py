"""Server configuration checks on the host (no GPU needed)."""
import ctypes

import pytest


def test_default_config(saltlib):
    c = saltlib.serve_default_config()
    assert c.budget_bytes == 8 << 30 and c.streams == 2 and c.max_n == 1 << 24
    assert c.max_batch == 256 and c.tile_bytes == 65536


@pytest.mark.parametrize("field,value", [("budget_bytes", 1000), ("max_requests", 0), ("max_batch", 0),
                                         ("streams", 9), ("tile_bytes", 1000), ("unroll", 3), ("block", 96),
                                         ("max_n", 0)])
def test_invalid_config_rejected_before_cuda(saltlib, field, value):
    c = saltlib.serve_default_config()
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert saltlib.lib.salt_serve_start(ctypes.byref(h), ctypes.byref(c)) == saltlib.ERR_ARG


def test_start_without_gpu_fails_loudly(saltlib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c = saltlib.serve_default_config()
    h = ctypes.c_void_p()
    assert saltlib.lib.salt_serve_start(ctypes.byref(h), ctypes.byref(c)) == saltlib.ERR_CUDA
