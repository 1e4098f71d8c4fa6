"""salt_dot_noalloc: the dot product for callers that cannot let the library
allocate device memory -- runtimes that hand out all device memory from a
fixed reservation made up front, and loops that cannot take cudaMalloc's
implicit synchronisation.  Its scratch is a static device array, so n is
capped at 2^28.

The test calls the entry point through the C ABI twice in a row and checks
each result against the exactly rounded dot product (relative error of the
result within FP64 1e-13 / FP32 1e-6) and against salt_dot's result (within
twice that), so that an accumulator fault shared by both entry points would
still fail.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

from oracle import exact
from paper_1109_1264_gb300 import inputs
import tolerance

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = tolerance.TOL


def _call(salt, code, n, x, y, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return salt.lib.salt_dot_noalloc(code, n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_noalloc_dot_against_exact_and_salt_dot(saltlib, cuda_dev, dt):
    salt = saltlib
    code = salt.F32 if dt == np.float32 else salt.F64
    for n in (1, 7, 1000, 65536, 65537, (1 << 20) + 7, (1 << 24) + 3):
        x, y = inputs.uniform_vectors(40 + n % 97, n, 2, dt)
        tx, ty = torch.from_numpy(x).to(cuda_dev), torch.from_numpy(y).to(cuda_dev)
        ref = torch.zeros(1, dtype=torch.float64, device=cuda_dev)
        salt.salt_dot(tx, ty, ref)
        torch.cuda.synchronize()
        exact_value, scale = exact.exact_dot(x, y), exact.abs_dot(x, y)
        for call in range(2):  # two calls in a row share the static scratch
            out = torch.full((1,), float("nan"), dtype=torch.float64, device=cuda_dev)
            assert _call(salt, code, n, tx, ty, out) == salt.OK, salt.salt_last_error()
            torch.cuda.synchronize()
            got = out.item()
            tolerance.check(got, exact_value, scale, dt, ("against the exact dot", n, call))
            tolerance.check(got, ref.item(), scale, dt, ("against salt_dot", n, call), factor=2.0)


def test_noalloc_rejects_oversize_and_bad_args(saltlib, cuda_dev):
    salt = saltlib
    x = torch.zeros(16, dtype=torch.float32, device=cuda_dev)
    out = torch.zeros(1, dtype=torch.float64, device=cuda_dev)
    # n beyond the static scratch: rejected on the host, nothing launched
    assert _call(salt, salt.F32, (1 << 28) + 1, x, x, out) == salt.ERR_BUDGET
    assert "2^28" in salt.salt_last_error()
    assert _call(salt, 7, 16, x, x, out) == salt.ERR_DTYPE
    assert _call(salt, salt.F32, -1, x, x, out) == salt.ERR_ARG
    # n = 0 writes a zero result
    out.fill_(5.0)
    assert _call(salt, salt.F32, 0, x, x, out) == salt.OK
    torch.cuda.synchronize()
    assert out.item() == 0.0
