"""The run-time compiled kernels' sources compile (CPU; NVRTC needs no GPU).

The library hands NVRTC the device headers prog.cuh, common.cuh and fused.cuh
with no system headers; a type or function that only the offline build
provides fails there and sends every program without a compiled shape to the
interpreter.  This test compiles the same sources, with the library's
options, for the fused and the strided kernel in both dtypes."""
import ctypes
import ctypes.util
import os

import pytest

from paper_1109_1264_gb300 import build

CSRC = os.path.join(os.path.dirname(build.__file__), "csrc")


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so", ctypes.util.find_library("nvrtc")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("NVRTC is not available")


def _compile(lib, name_expr):
    heads = build.JIT_HEADERS
    srcs = [open(os.path.join(CSRC, h), "rb").read() for h in heads]
    prog = ctypes.c_void_p()
    arr = lambda xs: (ctypes.c_char_p * len(xs))(*xs)
    r = lib.nvrtcCreateProgram(ctypes.byref(prog), b'#include "fused.cuh"\n', b"salt_jit.cu", len(heads),
                               arr(srcs), arr([h.encode() for h in heads]))
    assert r == 0, f"nvrtcCreateProgram: {r}"
    assert lib.nvrtcAddNameExpression(prog, name_expr.encode()) == 0
    opts = [b"-arch=sm_103a", b"-std=c++17", b"--fmad=false"]
    r = lib.nvrtcCompileProgram(prog, len(opts), arr(opts))
    n = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(n.value)
    lib.nvrtcGetProgramLog(prog, log)
    lowered = ctypes.c_char_p()
    if r == 0:
        lib.nvrtcGetLoweredName(prog, name_expr.encode(), ctypes.byref(lowered))
    lib.nvrtcDestroyProgram(ctypes.byref(prog))
    assert r == 0, log.value.decode(errors="replace")[-3000:]
    assert lowered.value


# op * 16 + arg: e = alpha*a + beta*b - c o d (a scaled add), and a dot
E = "16,0,80,17,1,80,32,2,3,64,48,116"
DOT = "0,1,128"


@pytest.mark.parametrize("name_expr", [
    f"salt::fused_kernel<salt::Prog<{E}>,double,4,16>",
    f"salt::fused_kernel<salt::Prog<{E}>,float,4,16>",
    f"salt::fused_kernel<salt::Prog<{DOT}>,double,4,16,true>",
    f"salt::strided_kernel<salt::Prog<{E}>,double,4>",
])
def test_jit_sources_compile(name_expr):
    _compile(_nvrtc(), name_expr)
