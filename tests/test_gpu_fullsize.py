"""Full-size parity (GPU): the BLAS-1 sweep's top size, n = 2^28 (+7 for the
elementwise ops, so the tail runs too), in the launch configuration the
benchmark times (autotuned first, as bench.py does).

Elementwise outputs are checked bit for bit on a sample of elements that the
oracle recomputes one by one from the counter-based inputs (its value at
index i depends on element i only).  Reductions use integer-valued data whose
sums are exact at this size, so the GPU result must equal the closed form."""
import math

import numpy as np
import pytest

import oracle
from paper_1109_1264_gb300 import inputs
from paper_1109_1264_gb300 import programs as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = (1 << 28) + 7
ALPHA, BETA = 1.5, -0.25


def gather_inputs(key, idx, dt):
    h = inputs.splitmix64(key, idx.astype(np.uint64))
    if dt == np.float64:
        return 2.0 * ((h >> np.uint64(11)).astype(np.float64) * 2.0 ** -53) - 1.0
    return (2.0 * ((h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24) - 1.0).astype(np.float32)


@pytest.mark.parametrize("sched", ["tuned", "staged"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_elementwise_full_size_sampled(saltlib, cuda_dev, dt, sched):
    """sched "tuned": the configuration the autotuner picks; "staged": the
    staged loop pinned (16 KiB stages for e, 8 KiB for axpby)."""
    s = saltlib
    tdt = torch.float32 if dt == np.float32 else torch.float64
    code = s.F32 if dt == np.float32 else s.F64
    keys = [101, 102, 103, 104, 105]
    a, b, c, d, y = (torch.empty(N, dtype=tdt, device=cuda_dev) for _ in range(5))
    out = torch.empty(N, dtype=tdt, device=cuda_dev)
    for t, k in zip((a, b, c, d, y), keys):
        s.salt_fill_uniform(t, key=k)
    s.salt_tune_clear()
    try:
        if sched == "tuned":
            s.salt_autotune(s.KERNEL_PROGRAM, P.PROG_E, [a, b, c, d, out], [ALPHA, BETA], reps=1)
            s.salt_autotune(s.KERNEL_PROGRAM, P.PROG_AXPBY, [a, y], [ALPHA, BETA], reps=1)
            # the autotuner ran axpby in place: start y afresh
            s.salt_fill_uniform(y, key=keys[4])
        else:
            s.salt_tune_set(P.PROG_E, code, N, 1, 16, 256, 0, 16384)
            s.salt_tune_set(P.PROG_AXPBY, code, N, 1, 16, 128, 0, 8192)
        s.salt_eval(P.PROG_E, [a, b, c, d, out], [ALPHA, BETA])
        s.salt_axpby(ALPHA, a, BETA, y)
        torch.cuda.synchronize()
    finally:
        s.salt_tune_clear()
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([np.arange(4096), np.arange(N - 4096, N), rng.integers(0, N, 200_000)]))
    assert idx.min() >= 0 and idx.max() < N
    ins = [gather_inputs(k, idx, dt) for k in keys]
    want_e = [ins[0].copy(), ins[1].copy(), ins[2].copy(), ins[3].copy(), np.zeros(len(idx), dt)]
    oracle.eval_program(oracle.PROG_E, want_e, [ALPHA, BETA])
    want_y = [ins[0].copy(), ins[4].copy()]
    oracle.eval_program(oracle.PROG_AXPBY, want_y, [ALPHA, BETA])
    tidx = torch.from_numpy(idx.astype(np.int64)).to(cuda_dev)
    got_e = out[tidx].cpu().numpy()
    got_y = y[tidx].cpu().numpy()
    iu = np.uint32 if dt == np.float32 else np.uint64
    assert np.array_equal(got_e.view(iu), want_e[4].view(iu))
    assert np.array_equal(got_y.view(iu), want_y[1].view(iu))


@pytest.mark.parametrize("sched", ["tuned", "staged"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_reductions_full_size_closed_form(saltlib, cuda_dev, dt, sched):
    """x_i = (i mod 1024) - 512, y_i = ((7 i) mod 512) - 256, n = 2^28: every
    product and partial sum is an integer below 2^53, so the compensated FP32
    and the FP64 paths must return the exact integer, and the norm the
    correctly rounded square root of the exact sum of squares.  sched
    "staged": the dot products on the staged loop (4 KiB stages)."""
    s = saltlib
    n = 1 << 28
    tdt = torch.float32 if dt == np.float32 else torch.float64
    code = s.F32 if dt == np.float32 else s.F64
    i = torch.arange(n, device=cuda_dev, dtype=torch.int64)
    x = ((i % 1024) - 512).to(tdt)
    yv = (((7 * i) % 512) - 256).to(tdt)
    del i
    outv = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
    s.salt_tune_clear()
    try:
        if sched == "tuned":
            s.salt_autotune(s.KERNEL_PROGRAM, P.PROG_DOT, [x, yv], red_out=outv[0:1], reps=1)
        else:
            s.salt_tune_set(P.PROG_DOT, code, n, 1, 16, 128, 0, 4096)
        s.salt_autotune(s.KERNEL_NRM2, None, [x], red_out=outv[1:2], reps=1)
        s.salt_dot(x, yv, outv[0:1])
        s.salt_nrm2(x, outv[1:2])
        s.salt_dot(x, x, outv[2:3])
        torch.cuda.synchronize()
    finally:
        s.salt_tune_clear()
    got_dot, got_nrm, got_sq = outv.cpu().tolist()
    # exact closed forms from one period (the data repeat every 1024 / 512 elements)
    j = np.arange(1024, dtype=np.int64)
    xs = j - 512
    per_x2 = int(np.sum(xs * xs))
    sumsq = per_x2 * (n // 1024)
    # dot: period lcm(1024, 512 * ...) -- compute on one period of 1024 of i, since 7 i mod 512 has period 512
    ys = ((7 * j) % 512) - 256
    dot = int(np.sum(xs * ys)) * (n // 1024)
    assert got_dot == dot, (got_dot, dot)
    assert got_sq == sumsq, (got_sq, sumsq)
    assert got_nrm == math.sqrt(sumsq), (got_nrm, math.sqrt(sumsq))


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_cg_passes_full_size_sampled(saltlib, cuda_dev, dt):
    """The two CG passes of salt_cg_diag at the bench's size (n = 2^28 + 5),
    on the compiled device-scalar kernels, with device scalars uploaded from
    the host: sampled elements of p, q, x and r bit-identical to the oracle
    recomputing them from the counter-based inputs."""
    from oracle_pins import CG_PQ, CG_XR_RHO
    s = saltlib
    n = (1 << 28) + 5
    tdt = torch.float32 if dt == np.float32 else torch.float64
    keys = {"d": 121, "p": 122, "x": 123, "r": 124}
    t = {k: torch.empty(n, dtype=tdt, device=cuda_dev) for k in ("d", "p", "q", "x", "r")}
    for k, key in keys.items():
        s.salt_fill_uniform(t[k], key=key)
    t["q"].zero_()
    ds = torch.tensor([0.75, 1.0 / 3.0, 2.5], dtype=torch.float64, device=cuda_dev)
    red = torch.zeros(2, dtype=torch.float64, device=cuda_dev)
    vecs = [t["d"], t["p"], t["q"], t["x"], t["r"], t["r"]]  # slot 5 (b) is not used by these passes
    s.salt_eval(CG_PQ, vecs, red_out=red[0:1], dscalars=[ds[0:1], ds[1:2]])
    s.salt_eval(CG_XR_RHO, vecs, red_out=red[1:2], dscalars=[ds[0:1], ds[2:3]])
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    idx = np.unique(np.concatenate([np.arange(4096), np.arange(n - 4096, n), rng.integers(0, n, 200_000)]))
    assert idx.min() >= 0 and idx.max() < n
    ins = {k: gather_inputs(key, idx, dt) for k, key in keys.items()}
    m = len(idx)
    want = [ins["d"], ins["p"].copy(), np.zeros(m, dt), ins["x"].copy(), ins["r"].copy(), np.zeros(m, dt)]
    oracle.eval_program(CG_PQ, want, dscalars=[0.75, 1.0 / 3.0])
    oracle.eval_program(CG_XR_RHO, want, dscalars=[0.75, 2.5])
    tidx = torch.from_numpy(idx.astype(np.int64)).to(cuda_dev)
    iu = np.uint32 if dt == np.float32 else np.uint64
    for name, slot in (("p", 1), ("q", 2), ("x", 3), ("r", 4)):
        got = t[name][tidx].cpu().numpy()
        assert np.array_equal(got.view(iu), want[slot].view(iu)), name


BIG = (1 << 31) + 13  # more elements than a 32-bit index can address


@pytest.mark.parametrize("sched", ["default", "staged"])
def test_elementwise_beyond_2e31_elements_sampled(saltlib, cuda_dev, sched):
    """axpby and e over n = 2^31 + 13 FP32 elements (every index computation
    must be 64-bit): sampled elements, including both sides of 2^31 and the
    tail, bit-identical to the oracle on the counter-based inputs.  sched
    "staged": both on the staged loop (16 KiB stages)."""
    s = saltlib
    keys = [131, 132, 133, 134, 135]
    a, b, c, d, y, out = (torch.empty(BIG, dtype=torch.float32, device=cuda_dev) for _ in range(6))
    for t, k in zip((a, b, c, d, y), keys):
        s.salt_fill_uniform(t, key=k)
    try:
        if sched == "staged":
            s.salt_tune_set(P.PROG_E, s.F32, BIG, 1, 16, 256, 0, 16384)
            s.salt_tune_set(P.PROG_AXPBY, s.F32, BIG, 1, 16, 128, 0, 16384)
        s.salt_axpby(ALPHA, a, BETA, y)
        s.salt_eval(P.PROG_E, [a, b, c, d, out], [ALPHA, BETA])
        torch.cuda.synchronize()
    finally:
        s.salt_tune_clear()
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([np.arange(4096), np.arange((1 << 31) - 4096, BIG),
                                    rng.integers(0, BIG, 100_000)]))
    assert idx.min() >= 0 and idx.max() < BIG  # checked on the host before any device gather
    ins = [gather_inputs(k, idx, np.float32) for k in keys]
    want_y = [ins[0].copy(), ins[4].copy()]
    oracle.eval_program(oracle.PROG_AXPBY, want_y, [ALPHA, BETA])
    want_e = [ins[0].copy(), ins[1].copy(), ins[2].copy(), ins[3].copy(), np.zeros(len(idx), np.float32)]
    oracle.eval_program(oracle.PROG_E, want_e, [ALPHA, BETA])
    tidx = torch.from_numpy(idx.astype(np.int64)).to(cuda_dev)
    assert np.array_equal(y[tidx].cpu().numpy().view(np.uint32), want_y[1].view(np.uint32))
    assert np.array_equal(out[tidx].cpu().numpy().view(np.uint32), want_e[4].view(np.uint32))


@pytest.mark.parametrize("sched", ["default", "staged"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_reductions_beyond_2e31_elements(saltlib, cuda_dev, dt, sched):
    """dot and nrm2 over n = 2^31 + 13 integer-valued elements: the FP64 path
    returns the exact integer (every partial sum is below 2^53), the
    compensated FP32 path is within 1e-6 of it.  sched "staged": the dot
    products on the staged loop (8 KiB stages)."""
    s = saltlib
    tdt = torch.float32 if dt == np.float32 else torch.float64
    code = s.F32 if dt == np.float32 else s.F64
    i = torch.arange(BIG, device=cuda_dev, dtype=torch.int64)
    x = ((i % 1024) - 512).to(tdt)
    yv = (((7 * i) % 512) - 256).to(tdt)
    del i
    torch.cuda.empty_cache()
    outv = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
    try:
        if sched == "staged":
            s.salt_tune_set(P.PROG_DOT, code, BIG, 1, 16, 128, 0, 8192)
        s.salt_dot(x, yv, outv[0:1])
        s.salt_nrm2(x, outv[1:2])
        s.salt_dot(x, x, outv[2:3])
        torch.cuda.synchronize()
    finally:
        s.salt_tune_clear()
    got_dot, got_nrm, got_sq = outv.cpu().tolist()
    j = np.arange(BIG % 1024, dtype=np.int64)  # the partial period at the end
    full = BIG // 1024
    xs_all = np.arange(1024, dtype=np.int64) - 512
    ys_all = ((7 * np.arange(1024, dtype=np.int64)) % 512) - 256
    sumsq = int(np.sum(xs_all * xs_all)) * full + int(np.sum((j - 512) ** 2))
    dot = int(np.sum(xs_all * ys_all)) * full + int(np.sum((j - 512) * (((7 * j) % 512) - 256)))
    absdot = int(np.sum(np.abs(xs_all * ys_all))) * full + int(np.sum(np.abs((j - 512) * (((7 * j) % 512) - 256))))
    if dt == np.float64:
        assert got_dot == dot and got_sq == sumsq, (got_dot, dot, got_sq, sumsq)
        assert got_nrm == math.sqrt(sumsq)
    else:
        assert abs(got_dot - dot) <= 1e-6 * absdot, (got_dot, dot)
        assert abs(got_sq - sumsq) <= 1e-6 * sumsq and abs(got_nrm - math.sqrt(sumsq)) <= 1e-6 * math.sqrt(sumsq)


def host_dot_reference(kx: int, ky: int, n: int, dt, same_sign: bool, piece: int = 1 << 22):
    """Exact sum x_i y_i and sum |x_i y_i| of the counter-based vectors keyed
    kx, ky (absolute values when same_sign), generated on the host piece by
    piece on a thread pool and summed in exact integer arithmetic."""
    import concurrent.futures as cf
    import os
    from oracle import exact
    fb = 52 if dt == np.float64 else 23

    def one(lo):
        m = min(piece, n - lo)
        x = inputs.hash_uniform(kx, m, dt, offset=lo)
        y = inputs.hash_uniform(ky, m, dt, offset=lo)
        if same_sign:
            x, y = np.abs(x), np.abs(y)
        f = exact.FixedPointDot(fb, fb)
        f.add(x, y)
        return f

    with cf.ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        parts = list(ex.map(one, range(0, n, piece)))
    f = exact.FixedPointDot.combine(parts)
    return f.value(), f.abs_value()


@pytest.mark.parametrize("data", ["random_sign", "same_sign"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_dot_full_size_relative_error(saltlib, cuda_dev, dt, data):
    """dot at the bench's size n = 2^28 on the counter-based uniform[-1, 1)
    data (random sign), and on its absolute values (one sign: the relative
    error of the result and the error relative to sum|x_i y_i| coincide),
    in the autotuned configuration and on the staged loop: the relative
    error of the result against the exact value is within 1e-13 (FP64) /
    1e-6 (compensated FP32) -- the tolerance stated on the value itself."""
    import tolerance
    s = saltlib
    n = 1 << 28
    tdt = torch.float32 if dt == np.float32 else torch.float64
    code = s.F32 if dt == np.float32 else s.F64
    kx, ky = 141, 142
    x, y = torch.empty(n, dtype=tdt, device=cuda_dev), torch.empty(n, dtype=tdt, device=cuda_dev)
    s.salt_fill_uniform(x, key=kx)
    s.salt_fill_uniform(y, key=ky)
    if data == "same_sign":
        x.abs_()
        y.abs_()
    out = torch.zeros(2, dtype=torch.float64, device=cuda_dev)
    s.salt_tune_clear()
    try:
        s.salt_autotune(s.KERNEL_PROGRAM, P.PROG_DOT, [x, y], red_out=out[0:1], reps=1)
        s.salt_dot(x, y, out[0:1])
        s.salt_tune_set(P.PROG_DOT, code, n, 1, 16, 128, 0, 16384)
        s.salt_dot(x, y, out[1:2])
        torch.cuda.synchronize()
    finally:
        s.salt_tune_clear()
    del x, y
    ref, scale = host_dot_reference(kx, ky, n, dt, data == "same_sign")
    for got, sched in zip(out.cpu().tolist(), ("tuned", "staged")):
        e = tolerance.check(got, ref, scale, dt, (data, sched))
        # judged on the relative error of the result, not on sum|x_i y_i|
        assert e["cond"] <= tolerance.COND_LITERAL, e
        if data == "same_sign":
            assert e["rel_value"] == e["rel_scale"]
        print(f"dot {dt.__name__} n=2^28 {data} {sched}: rel_value {e['rel_value']:.3e} "
              f"rel_scale {e['rel_scale']:.3e} cond {e['cond']:.3e}")
