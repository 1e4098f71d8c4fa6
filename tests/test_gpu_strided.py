"""Operands that are not 16-byte aligned or not contiguous (GPU): the
element-access kernels must give the oracle's bits, leave the elements
between strided positions untouched, and keep reductions within tolerance --
for compiled shapes, the interpreter and run-time compiled programs."""
import numpy as np
import pytest

import oracle
from paper_1109_1264_gb300 import inputs
import tolerance
from test_gpu_parity import PROGS, TOL, assert_bits_equal, check_reductions

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TDT = {np.float32: torch.float32, np.float64: torch.float64}
ODD = [("VEC", 0), ("NEG", 0), ("VEC", 1), ("MUL", 0), ("VEC", 2), ("ADD", 0), ("STORE", 1), ("VEC", 1),
       ("VEC", 0), ("DOT", 0)]  # not a compiled shape


def views(vecs, dt, layout, dev):
    """Device views of the host vectors: layout 'offset' puts each at a
    1- to 3-element (unaligned) offset, different per operand; 'same_offset'
    puts every operand at the same 1-element offset (for FP32 the vector
    kernels then start at the next 128-byte boundary and evaluate the head
    elements one by one); 'stride' at a stride of 2 or 3; returns (views,
    backing buffers, positions of the views in the buffers)."""
    out, bufs, pos = [], [], []
    for k, v in enumerate(vecs):
        n = len(v)
        if layout in ("offset", "same_offset"):
            off = 1 + k % 3 if layout == "offset" else 1
            buf = torch.full((n + 8,), 7.0, dtype=TDT[dt], device=dev)
            idx = np.arange(off, off + n)
            buf[off:off + n] = torch.from_numpy(v).to(dev)
            out.append(buf[off:off + n])
        else:
            st = 2 + k % 2
            buf = torch.full((n * st + 1,), 7.0, dtype=TDT[dt], device=dev)
            idx = np.arange(0, n * st, st)
            buf[0:n * st:st] = torch.from_numpy(v).to(dev)
            out.append(buf[0:n * st:st])
        bufs.append(buf)
        pos.append(idx)
    return out, bufs, pos


@pytest.mark.parametrize("layout", ["offset", "same_offset", "stride"])
@pytest.mark.parametrize("name", ["D", "E", "AXPBY", "CG", "DOT", "SUMSQ", "ODD", "ODD_JIT"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_unaligned_and_strided(saltlib, cuda_dev, layout, name, dt):
    s = saltlib
    if name.startswith("ODD"):
        prog, nv, ns = ODD, 3, 0
    else:
        prog, nv, ns = PROGS[name]
    prev = s.salt_jit_stats()["mode"]
    if name == "ODD_JIT":
        s.salt_set_jit(s.JIT_ON)
    elif name == "ODD":
        s.salt_set_jit(s.JIT_OFF)  # the interpreter's element mode
    try:
        for n in (1, 2, 3, 4, 5, 1000, 70001):
            vecs = inputs.uniform_vectors(50 + n, n, nv, dt)
            scalars = [1.5, -0.25][:ns]
            tv, bufs, pos = views(vecs, dt, layout, cuda_dev)
            if layout != "stride":
                assert any(t.data_ptr() % 16 for t in tv)
            elif n > 1:  # a one-element view is contiguous whatever its stride
                assert all(not t.is_contiguous() for t in tv)
            nred = sum(1 for o, _ in prog if o in ("DOT", "SUMSQ"))
            red = torch.full((max(nred, 1),), float("nan"), dtype=torch.float64, device=cuda_dev)
            s.salt_eval(prog, tv, scalars, red_out=red if nred else None)
            torch.cuda.synchronize()
            want = [v.copy() for v in vecs]
            oracle.eval_program(prog, want, scalars)
            for k, (buf, idx) in enumerate(zip(bufs, pos)):
                b = buf.cpu().numpy()
                assert_bits_equal(b[idx], want[k], f"{name} {layout} n={n} operand {k}")
                rest = np.delete(b, idx)
                assert np.all(rest == 7.0), f"{name} {layout}: elements outside the view were written"
            check_reductions(prog, vecs, scalars, red.cpu().numpy(), dt, f"{name} {layout}")
    finally:
        s.salt_set_jit(prev)


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_unaligned_dot_and_nrm2(saltlib, cuda_dev, dt):
    from oracle import exact
    s = saltlib
    for n in (3, 999, 123457):
        x, y = inputs.uniform_vectors(60, n, 2, dt)
        bx = torch.zeros(n + 1, dtype=TDT[dt], device=cuda_dev)
        by = torch.zeros(n + 3, dtype=TDT[dt], device=cuda_dev)
        bx[1:] = torch.from_numpy(x).to(cuda_dev)
        by[3:] = torch.from_numpy(y).to(cuda_dev)
        out = torch.zeros(2, dtype=torch.float64, device=cuda_dev)
        s.salt_dot(bx[1:], by[3:], out[0:1])
        s.salt_nrm2(bx[1:], out[1:2])
        d, nr = out.cpu().tolist()
        tolerance.check_dot(d, x, y, dt, ("unaligned dot", n))
        ref = exact.exact_nrm2(x)
        tolerance.check(nr, ref, ref, dt, ("unaligned nrm2", n))


@pytest.mark.parametrize("name", ["D", "E", "AXPBY", "CG", "DOT", "ODD", "ODD_JIT"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_negative_strides(saltlib, cuda_dev, name, dt):
    """BLAS incx < 0 through the C ABI: element i of operand k at
    vecs[k][i * strides[k]] with strides -1, -2, -3 mixed with positive
    ones; the oracle's bits at exactly those positions, nothing else
    written, reductions within tolerance."""
    import ctypes
    s = saltlib
    if name.startswith("ODD"):
        prog, nv, ns = ODD, 3, 0
    else:
        prog, nv, ns = PROGS[name]
    es = np.dtype(dt).itemsize
    code = s.F32 if dt == np.float32 else s.F64
    prev = s.salt_jit_stats()["mode"]
    if name == "ODD_JIT":
        s.salt_set_jit(s.JIT_ON)
    elif name == "ODD":
        s.salt_set_jit(s.JIT_OFF)  # the interpreter's element mode
    try:
        for n in (1, 5, 1000, 70001):
            vecs = inputs.uniform_vectors(90 + n, n, nv, dt)
            scalars = [1.5, -0.25][:ns]
            strides = [-(1 + k % 3) if k % 2 == 0 else 1 + k % 2 for k in range(nv)]
            bufs, pos, ptrs = [], [], []
            for v, st in zip(vecs, strides):
                m = abs(st)
                buf = torch.full((n * m + 1,), 7.0, dtype=TDT[dt], device=cuda_dev)
                first = (n - 1) * m if st < 0 else 0  # element 0's position in the buffer
                idx = first + np.arange(n, dtype=np.int64) * st
                assert idx.min() >= 0 and idx.max() < buf.numel()
                buf[torch.from_numpy(idx).to(cuda_dev)] = torch.from_numpy(v).to(cuda_dev)
                bufs.append(buf)
                pos.append(idx)
                ptrs.append(buf.data_ptr() + first * es)
            nred = sum(1 for o, _ in prog if o in ("DOT", "SUMSQ"))
            red = torch.full((max(nred, 1),), float("nan"), dtype=torch.float64, device=cuda_dev)
            arr, m_ = s.program(prog)
            cp = (ctypes.c_void_p * nv)(*ptrs)
            cs = (ctypes.c_int64 * nv)(*strides)
            sc = (ctypes.c_double * max(ns, 1))(*scalars)
            stream = torch.cuda.current_stream().cuda_stream
            st_ = s.lib.salt_eval_strided(arr, m_, code, n, cp, cs, nv, sc, ns,
                                          red.data_ptr() if nred else None, stream)
            assert st_ == s.OK, s.lib.salt_last_error()
            torch.cuda.synchronize()
            want = [v.copy() for v in vecs]
            oracle.eval_program(prog, want, scalars)
            for k, (buf, idx) in enumerate(zip(bufs, pos)):
                b = buf.cpu().numpy()
                assert_bits_equal(b[idx], want[k], f"{name} negative strides n={n} operand {k}")
                assert np.all(np.delete(b, idx) == 7.0), f"{name}: elements outside the strided positions written"
            check_reductions(prog, vecs, scalars, red.cpu().numpy()[:nred], dt, f"{name} negative strides")
    finally:
        s.salt_set_jit(prev)
