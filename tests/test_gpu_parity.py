"""Parity of the CUDA path with the oracle (GPU).

Elementwise results must be bit-identical to the oracle's node-by-node
evaluation; reductions must be within the stated tolerance of the exactly
rounded reference: FP64 1e-13, FP32 (compensated) 1e-6, as the relative
error of the result (tests/tolerance.py: relative to the condition scale
sum|x_i y_i| only for ill-conditioned sums)."""
import math
import random

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1109_1264_gb300 import inputs
import oracle_pins
import tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = tolerance.TOL
TORCH_DT = {np.float64: torch.float64, np.float32: torch.float32}

PROGS = {
    "D": (oracle.PROG_D, 4, 0),
    "AXPBY": (oracle.PROG_AXPBY, 2, 2),
    "AXPBYZ": ([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("SCAL", 1), ("VEC", 1), ("SMUL", 0), ("ADD", 0),
                ("STORE", 2)], 3, 2),
    "AXPY": ([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("ADD", 0), ("STORE", 1)], 2, 1),
    "E": (oracle.PROG_E, 5, 2),
    "SCAL": ([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 0)], 1, 1),
    "SCALE": (oracle.PROG_SCALE, 2, 1),
    "COPY": ([("VEC", 0), ("STORE", 1)], 2, 0),
    "CG": (oracle.PROG_CG, 3, 2),
    "DOT": (oracle.PROG_DOT, 2, 0),
    "SUMSQ": ([("VEC", 0), ("SUMSQ", 0)], 1, 0),
}

SIZES = [0, 1, 2, 3, 7, 8, 63, 64, 65, 1000, 2047, 2048, 2049, 4096 + 7, 65536 + 13, (1 << 20) + 7, 3 * (1 << 20) + 5]


def assert_bits_equal(got: np.ndarray, want: np.ndarray, what=""):
    assert got.shape == want.shape, what
    iu = np.uint32 if got.dtype == np.float32 else np.uint64
    same = got.view(iu) == want.view(iu)
    both_nan = np.isnan(got) & np.isnan(want)
    bad = ~(same | both_nan)
    if bad.any():
        i = int(np.argmax(bad))
        raise AssertionError(f"{what}: {int(bad.sum())} elements differ, first at {i}: got {got[i]!r} want {want[i]!r}")


def run_gpu(salt, prog, vecs_np, scalars, dt, n=None):
    dev = torch.device("cuda:0")
    tv = [torch.from_numpy(v.copy()).to(dev) for v in vecs_np]
    nred = sum(1 for o, _ in prog if o in ("DOT", "SUMSQ"))
    red = torch.full((max(nred, 1),), float("nan"), dtype=torch.float64, device=dev)
    salt.salt_eval(prog, tv, scalars, red_out=red if nred else None, n=n)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in tv], red.cpu().numpy()[:nred]


def run_oracle(prog, vecs_np, scalars):
    vs = [v.copy() for v in vecs_np]
    red = oracle.eval_program(prog, vs, scalars)
    return vs, red


@pytest.fixture(scope="module")
def salt(saltlib, cuda_dev):
    return saltlib


def make_inputs(name, n, dt, seed):
    prog, nv, ns = PROGS[name]
    vecs = inputs.uniform_vectors(seed, n, nv, dt)
    scalars = [1.5, -0.25][:ns]
    return prog, vecs, scalars


@pytest.mark.parametrize("name", list(PROGS))
@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
def test_named_programs_bit_exact(salt, name, dt):
    for i, n in enumerate(SIZES):
        prog, vecs, scalars = make_inputs(name, n, dt, seed=100 + i)
        got, red = run_gpu(salt, prog, vecs, scalars, dt)
        want, red_o = run_oracle(prog, vecs, scalars)
        for k, (g, w) in enumerate(zip(got, want)):
            assert_bits_equal(g, w, f"{name} n={n} operand {k}")
        check_reductions(prog, vecs, scalars, red, dt, f"{name} n={n}")


def reduction_operands(prog, vecs_np, scalars, dscalars=()):
    """The operand vectors of every DOT / SUMSQ of ``prog``, materialised by
    the oracle: each reduction is rewritten into STOREs to fresh operands
    (same stack effect), so the oracle's node-by-node evaluation produces
    exactly the values the reduction consumes."""
    nv = len(vecs_np)
    rewritten, pairs, extra = [], [], 0
    for op, arg in prog:
        if op == "DOT":
            rewritten += [("STORE", nv + extra + 1), ("STORE", nv + extra)]
            pairs.append((nv + extra, nv + extra + 1))
            extra += 2
        elif op == "SUMSQ":
            rewritten += [("STORE", nv + extra)]
            pairs.append((nv + extra, nv + extra))
            extra += 1
        else:
            rewritten.append((op, arg))
    vs = [v.copy() for v in vecs_np] + [np.zeros_like(vecs_np[0]) for _ in range(extra)]
    oracle.eval_program(rewritten, vs, scalars, dscalars=dscalars)
    return [(vs[a], vs[b]) for a, b in pairs]


def check_reductions(prog, vecs_np, scalars, red, dt, what="", dscalars=()):
    out = []
    for k, (a, b) in enumerate(reduction_operands(prog, vecs_np, scalars, dscalars)):
        out.append(tolerance.check_dot(red[k], a, b, dt, (what, k)))
        if a.size == 0:
            assert red[k] == 0.0
    return out


CONFIGS = [(u, vb, blk, bps) for u in (1, 2, 4) for vb in (16, 32) for blk, bps in ((64, 4), (128, 3), (256, 8), (256, 1))]


@pytest.mark.parametrize("name", ["D", "E", "CG", "DOT", "AXPBY"])
@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
def test_every_launch_configuration(salt, name, dt):
    """Every instantiated unroll depth / vector width and several block and
    grid shapes give the same bits (reductions: within tolerance)."""
    n = (1 << 18) + 77
    prog, vecs, scalars = make_inputs(name, n, dt, seed=7)
    want, _ = run_oracle(prog, vecs, scalars)
    code = salt.F32 if dt == np.float32 else salt.F64
    try:
        for cfg in CONFIGS:
            salt.salt_tune_set(prog, code, n, *cfg)
            got, red = run_gpu(salt, prog, vecs, scalars, dt)
            for k, (g, w) in enumerate(zip(got, want)):
                assert_bits_equal(g, w, f"{name} cfg={cfg} operand {k}")
            check_reductions(prog, vecs, scalars, red, dt, f"{name} cfg={cfg}")
    finally:
        salt.salt_tune_clear()


@pytest.fixture
def interpreter(salt):
    """Run-time compilation off: programs without a compiled instantiation
    run on the interpreter kernel."""
    prev = salt.salt_jit_stats()["mode"]
    salt.salt_set_jit(salt.JIT_OFF)
    yield salt
    salt.salt_set_jit(prev)


def test_interpreter_random_programs(salt, interpreter):
    """Programs without a compiled instantiation run on the interpreter and
    must match the oracle bit for bit (reductions within tolerance)."""
    rng = random.Random(11)
    nrng = np.random.default_rng(11)
    ran_interp = 0
    for t in range(80):
        dt = np.float64 if t % 2 == 0 else np.float32
        nvecs = rng.randint(1, 6)
        nscal = rng.randint(0, 3)
        while True:  # programs within the ABI limits (32 nodes, 4 reductions)
            prog = oracle_pins.random_program(rng, nvecs, nscal)
            if len(prog) <= salt.MAX_PROG and sum(o in ("DOT", "SUMSQ") for o, _ in prog) <= salt.MAX_REDS:
                break
        nred, compiled = salt.salt_check_program(prog, nvecs, nscal)
        ran_interp += not compiled
        n = rng.choice([1, 5, 17, 255, 256, 1023, 4099, 70001, 300007])
        vecs = [nrng.uniform(-1, 1, n).astype(dt) for _ in range(nvecs)]
        scalars = list(nrng.uniform(-2, 2, nscal))
        got, red = run_gpu(salt, prog, vecs, scalars, dt)
        want, red_o = run_oracle(prog, vecs, scalars)
        for k, (g, w) in enumerate(zip(got, want)):
            assert_bits_equal(g, w, f"prog {prog} n={n} operand {k}")
        check_reductions(prog, vecs, scalars, red, dt, f"prog {prog} n={n}")
    assert ran_interp > 50


def test_interpreter_reductions_exact_reference(salt, interpreter):
    """Interpreter-only programs with reductions, judged against the exact
    reference of their operands."""
    progs = [
        # dot of (x - y) with (x + y), a non-canonical shape
        ([("VEC", 0), ("VEC", 1), ("SUB", 0), ("VEC", 0), ("VEC", 1), ("ADD", 0), ("DOT", 0)], 2, 0,
         lambda x, y: (x - y, x + y)),
        ([("VEC", 1), ("NEG", 0), ("SUMSQ", 0)], 2, 0, lambda x, y: (-y, -y)),
    ]
    for prog, nv, ns, ops in progs:
        for dt in (np.float64, np.float32):
            for n in (1, 1000, 100003, (1 << 20) + 3):
                x, y = inputs.uniform_vectors(3, n, 2, dt)
                _, red = run_gpu(salt, prog, [x, y], [], dt)
                a, b = ops(x, y)
                a = a.astype(dt)
                b = b.astype(dt)
                tolerance.check_dot(red[0], a, b, dt, (prog, dt, n))


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
def test_dot_nrm2_tolerance(salt, dt):
    dev = torch.device("cuda:0")
    for n in (1, 3, 1000, 65536 + 3, (1 << 20) + 7, 1 << 23):
        x, y = inputs.uniform_vectors(21, n, 2, dt)
        tx, ty = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
        out = torch.zeros(3, dtype=torch.float64, device=dev)
        salt.salt_dot(tx, ty, out[0:1])
        salt.salt_nrm2(tx, out[1:2])
        salt.salt_dot(tx, tx, out[2:3])
        d, nr, dd = out.cpu().tolist()
        e = tolerance.check_dot(d, x, y, dt, ("dot", n))
        assert e["cond"] <= tolerance.COND_LITERAL  # judged relative to its value
        nref = exact.exact_nrm2(x)
        tolerance.check(nr, nref, nref, dt, ("nrm2", n))
        sref = exact.exact_sumsq(x)
        tolerance.check(dd, sref, sref, dt, ("sumsq", n))


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
def test_reduction_closed_forms_exact(salt, dt):
    """Integer data: every partial sum is exact, so the GPU result must equal
    the closed form n(n-1)/2, and the norm the correctly rounded
    sqrt((n-1)n(2n-1)/6)."""
    dev = torch.device("cuda:0")
    for n in (1, 2, 7, 1000, 65537, 1 << 17):
        x = torch.arange(n, dtype=TORCH_DT[dt], device=dev)
        one = torch.ones(n, dtype=TORCH_DT[dt], device=dev)
        out = torch.zeros(2, dtype=torch.float64, device=dev)
        salt.salt_dot(x, one, out[0:1])
        salt.salt_nrm2(x, out[1:2])
        d, nr = out.cpu().tolist()
        assert d == n * (n - 1) // 2, (n, d)
        assert nr == math.sqrt((n - 1) * n * (2 * n - 1) // 6), (n, nr)


def test_nrm2_no_overflow_underflow(salt):
    dev = torch.device("cuda:0")
    cases = [(np.float64, c) for c in (2.0 ** 600, 2.0 ** -600, 2.0 ** 1000, 2.0 ** -1000, 3.0)] + \
            [(np.float32, c) for c in (2.0 ** 100, 2.0 ** -100, 2.0 ** 120, 2.0 ** -140, 3.0)]
    for dt, c in cases:
        for k in (0, 1, 5, 9):
            x = torch.full((4 ** k,), c, dtype=TORCH_DT[dt], device=dev)
            out = torch.zeros(1, dtype=torch.float64, device=dev)
            salt.salt_nrm2(x, out)
            got = out.item()
            assert abs(got - c * 2 ** k) <= 4e-16 * c * 2 ** k, (dt, c, k, got)
    # mixed ranges in one vector
    for dt in (np.float64, np.float32):
        rng = np.random.default_rng(4)
        big, small = (2.0 ** 500, 2.0 ** -530) if dt == np.float64 else (2.0 ** 70, 2.0 ** -80)
        x = rng.uniform(-1, 1, 100003)
        x[::7] *= big
        x[3::11] *= small
        x = x.astype(dt)
        out = torch.zeros(1, dtype=torch.float64, device=dev)
        salt.salt_nrm2(torch.from_numpy(x).to(dev), out)
        ref = exact.exact_nrm2(x)
        assert abs(out.item() - ref) <= TOL[dt] * ref
        y = rng.uniform(-1, 1, 1003) * small
        y = y.astype(dt)
        salt.salt_nrm2(torch.from_numpy(y).to(dev), out)
        ref = exact.exact_nrm2(y)
        assert abs(out.item() - ref) <= TOL[dt] * ref, (dt, out.item(), ref)
    # special values
    for dt in (np.float64, np.float32):
        for v, check in ((np.inf, math.isinf), (np.nan, math.isnan)):
            x = np.ones(1000, dtype=dt)
            x[500] = v
            out = torch.zeros(1, dtype=torch.float64, device=dev)
            salt.salt_nrm2(torch.from_numpy(x).to(dev), out)
            assert check(out.item())
        salt.salt_nrm2(torch.zeros(77, dtype=TORCH_DT[dt], device=dev), out)
        assert out.item() == 0.0


def test_special_values_bit_exact(salt):
    for dt in (np.float64, np.float32):
        tiny = np.finfo(dt).smallest_subnormal
        base = np.array([np.nan, np.inf, -np.inf, 0.0, -0.0, 1.0, tiny, -tiny, np.finfo(dt).max, 3.0], dtype=dt)
        a = np.tile(base, 100)
        b = np.roll(a, 3)
        c = np.roll(a, 7)
        d = np.roll(a, 1)
        for name in ("D", "E", "AXPBY", "CG"):
            prog, nv, ns = PROGS[name]
            vecs = [a, b, c, d, np.zeros_like(a)][:nv]
            scalars = [1.5, -0.25][:ns]
            got, _ = run_gpu(salt, prog, vecs, scalars, dt)
            want, _ = run_oracle(prog, vecs, scalars)
            for k, (g, w) in enumerate(zip(got, want)):
                assert_bits_equal(g, w, f"{name} specials operand {k}")
        # -0 results and subnormal outputs of the interpreter as well
        prog = [("VEC", 0), ("NEG", 0), ("VEC", 1), ("MUL", 0), ("STORE", 2)]
        got, _ = run_gpu(salt, prog, [a, b, np.zeros_like(a)], [], dt)
        want, _ = run_oracle(prog, [a, b, np.zeros_like(a)], [])
        assert_bits_equal(got[2], want[2], "interpreter specials")


def test_config1_full(salt):
    """d = a + (b - c), FP64, n = 2^20, a, b, c uniform[-1, 1] from seed 0."""
    n = 1 << 20
    a, b, c = inputs.uniform_vectors(0, n, 3, np.float64)
    d = np.zeros(n)
    got, _ = run_gpu(salt, oracle.PROG_D, [a, b, c, d], [], np.float64)
    want, _ = run_oracle(oracle.PROG_D, [a, b, c, d], [])
    assert_bits_equal(got[3], want[3], "config 1")


def test_fill_matches_counter_generator(salt):
    dev = torch.device("cuda:0")
    for dt in (np.float64, np.float32):
        n = (1 << 20) + 3
        x = torch.empty(n, dtype=TORCH_DT[dt], device=dev)
        salt.salt_fill_uniform(x, key=0xDEADBEEF, offset=12345)
        want = inputs.hash_uniform(0xDEADBEEF, n, dt, offset=12345)
        assert_bits_equal(x.cpu().numpy(), want, "fill")


def test_edge_cases(salt):
    dev = torch.device("cuda:0")
    # in-place axpby with x and y the same tensor: y = alpha*y + beta*y
    for dt in (np.float64, np.float32):
        y = inputs.uniform_vectors(5, 10007, 1, dt)[0]
        ty = torch.from_numpy(y.copy()).to(dev)
        salt.salt_axpby(1.5, ty, -0.25, ty)
        want = y.copy()
        oracle.eval_program([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("SCAL", 1), ("VEC", 0), ("SMUL", 0),
                             ("ADD", 0), ("STORE", 0)], [want], [1.5, -0.25])
        assert_bits_equal(ty.cpu().numpy(), want, "in-place axpby")
    # operands 16-byte but not 32-byte aligned: the 32-byte kernels are skipped
    for dt in (np.float64, np.float32):
        el = 16 // np.dtype(dt).itemsize
        n = 50001
        prog, vecs, scalars = make_inputs("E", n, dt, 9)
        code = salt.F32 if dt == np.float32 else salt.F64
        salt.salt_tune_set(prog, code, n, 2, 32, 256, 4)
        try:
            big = [torch.from_numpy(np.concatenate([np.zeros(el, dt), v])).to(dev) for v in vecs]
            views = [t[el:] for t in big]
            assert all(v.data_ptr() % 32 == 16 for v in views)
            salt.salt_eval(prog, views, scalars)
            want, _ = run_oracle(prog, vecs, scalars)
            assert_bits_equal(views[4].cpu().numpy(), want[4], "16-byte aligned views")
        finally:
            salt.salt_tune_clear()
    # misaligned operand, overlap, dtype mismatch: rejected before launch
    x = torch.zeros(1000, dtype=torch.float32, device=dev)
    with pytest.raises(salt.SaltError) as ei:
        salt.salt_eval(oracle.PROG_SCALE, [x[1:], x[:-1]], [2.0])
    assert ei.value.status in (salt.ERR_ALIGN, salt.ERR_ALIAS)
    with pytest.raises(salt.SaltError) as ei:
        salt.salt_eval(oracle.PROG_SCALE, [x[4:], x[:-4]], [2.0])
    assert ei.value.status == salt.ERR_ALIAS
    with pytest.raises(salt.SaltError) as ei:
        salt.salt_eval(oracle.PROG_SCALE, [x, torch.zeros(1000, dtype=torch.float64, device=dev)], [2.0])
    assert ei.value.status == salt.ERR_DTYPE
    # n = 0 leaves outputs alone and returns zero reductions
    out = torch.full((1,), 7.0, dtype=torch.float64, device=dev)
    e = torch.empty(0, dtype=torch.float32, device=dev)
    salt.salt_dot(e, e, out)
    assert out.item() == 0.0


def test_reductions_reproducible_and_stream_ordered(salt):
    dev = torch.device("cuda:0")
    x, y = inputs.uniform_vectors(8, (1 << 22) + 5, 2, np.float32)
    tx, ty = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    outs = torch.zeros(8, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for i in range(4):
            salt.salt_dot(tx, ty, outs[i:i + 1])
    for i in range(4, 8):
        salt.salt_dot(tx, ty, outs[i:i + 1])
    torch.cuda.synchronize()
    v = outs.cpu().numpy()
    assert np.all(v.view(np.uint64) == v.view(np.uint64)[0])


def test_precision_form_config3(salt):
    """n = 2^26, FP32 values sign-random with magnitudes log-uniform in
    [1e-3, 1e3]: compensated FP32 dot / nrm2 within 1e-6 of the exact value;
    the plain FP32 run is less accurate; the FP64 run on widened data within
    1e-13."""
    dev = torch.device("cuda:0")
    n = 1 << 26
    x, y = inputs.logmag_vectors(0, n, 2, np.float32)
    ref = exact.exact_dot(x, y)
    scale = exact.abs_dot(x, y)
    nref = exact.exact_nrm2(x)
    tx, ty = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    out = torch.zeros(6, dtype=torch.float64, device=dev)
    salt.salt_dot(tx, ty, out[0:1])
    salt.salt_dot(tx, ty, out[1:2], plain=True)
    salt.salt_dot(tx.double(), ty.double(), out[2:3])
    salt.salt_nrm2(tx, out[3:4])
    salt.salt_nrm2(tx, out[4:5], plain=True)
    salt.salt_nrm2(tx.double(), out[5:6])
    comp, plain, wide, nc, npl, nw = out.cpu().tolist()
    # Plain FP32 summation depth: at most ceil(n / (152 * 64)) terms per thread
    # (>= 152 blocks of >= 64 threads at this size) plus < 100 tree levels.
    plain_gamma = exact.gamma(-(-n // (152 * 64)) + 100, 2.0 ** -24)
    ec = tolerance.check(comp, ref, scale, np.float32, "compensated FP32 dot")
    ew = tolerance.check(wide, ref, scale, np.float64, "FP64 dot of the widened data")
    # this data's cond is about 1e3, so both are judged relative to the value
    assert ec["cond"] <= tolerance.COND_LITERAL and ew["rel_value"] <= 1e-13
    assert abs(plain - ref) <= plain_gamma * scale
    assert abs(comp - ref) <= abs(plain - ref)
    assert abs(nc - nref) <= 1e-6 * nref
    assert abs(nw - nref) <= 1e-13 * nref
    assert abs(npl - nref) <= plain_gamma * nref


def test_concurrent_host_threads_on_separate_streams(salt):
    """Four host threads, each on its own stream, run reductions and fused
    expressions at the same time: every result equals the single-threaded
    one (per-stream workspaces, thread-safe tables, thread-local errors)."""
    import threading
    dev = torch.device("cuda:0")
    n = (1 << 20) + 3
    x, y = (torch.from_numpy(v).to(dev) for v in inputs.uniform_vectors(77, n, 2, np.float64))
    ref = torch.zeros(2, dtype=torch.float64, device=dev)
    salt.salt_dot(x, y, ref[0:1])
    salt.salt_nrm2(x, ref[1:2])
    torch.cuda.synchronize()
    want = ref.cpu().numpy()
    outs, errors = {}, []

    def work(t):
        try:
            s = torch.cuda.Stream()
            red = torch.zeros(2 * 50, dtype=torch.float64, device=dev)
            z = torch.empty(n, dtype=torch.float64, device=dev)
            with torch.cuda.stream(s):
                for i in range(50):
                    salt.salt_dot(x, y, red[2 * i:2 * i + 1], stream=s)
                    salt.salt_nrm2(x, red[2 * i + 1:2 * i + 2], stream=s)
                    salt.salt_eval(oracle.PROG_SCALE, [x, z], [0.5 + t], stream=s)
                    try:  # an error on one thread stays on that thread
                        salt.salt_eval([("ADD", 0)], [x])
                    except salt.SaltError as e:
                        assert "needs two operands" in e.message
            s.synchronize()
            outs[t] = (red.cpu().numpy(), z.cpu().numpy())
        except Exception as e:  # noqa: BLE001
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    xh = x.cpu().numpy()
    for t, (red, z) in outs.items():
        assert np.array_equal(red.reshape(-1, 2), np.tile(want, (50, 1))), t
        want_z = [xh.copy(), np.zeros(n)]
        oracle.eval_program(oracle.PROG_SCALE, want_z, [0.5 + t])
        assert_bits_equal(z, want_z[1], f"thread {t}")


POW2_PROGS = {
    "E": (oracle.PROG_E, 5, 2),
    "AXPBY": (oracle.PROG_AXPBY, 2, 2),
    "AXPY": ([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("ADD", 0), ("STORE", 1)], 2, 1),
    "CG": (oracle.PROG_CG, 3, 2),
    "X_MINUS_SV": ([("VEC", 0), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("SUB", 0), ("STORE", 2)], 3, 1),
    "SV_MINUS_W": ([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("SUB", 0), ("STORE", 2)], 3, 1),
    # no compiled shape: the run-time compiled kernel
    "JIT": ([("VEC", 0), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("VEC", 2), ("MUL", 0),
             ("SCAL", 1), ("VEC", 2), ("SMUL", 0), ("VEC", 0), ("SUB", 0), ("ADD", 0), ("STORE", 3)], 4, 2),
}


def edge_values(rng, n, runs=False):
    """FP64 values spread over the whole exponent range: ordinary values,
    normals near the bottom and the top of the range, subnormals, signed
    zeros, infinities and NaN -- each element's class drawn on its own, or
    (runs) one class for runs of 1 to 64 elements, so that whole chunks of
    a thread hold one class."""
    kind = rng.integers(0, 8, n)
    if runs:
        kind = np.repeat(kind, rng.integers(1, 65, n))[:n]
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    v = rng.uniform(-1, 1, n)
    frac = 1.0 + rng.random(n)
    lo = np.ldexp(frac, rng.integers(-1022, -1000, n))
    hi = np.ldexp(frac * 0.99, rng.integers(1000, 1023, n))
    sub = np.ldexp(rng.random(n), -1022)
    v = np.where(kind == 1, sign * lo, v)
    v = np.where(kind == 2, sign * hi, v)
    v = np.where(kind == 3, sign * sub, v)
    v = np.where(kind == 4, sign * 0.0, v)
    v = np.where(kind == 5, sign * np.inf, v)
    v = np.where(kind == 6, np.nan, v)
    return v


@pytest.mark.parametrize("name", list(POW2_PROGS))
def test_power_of_two_scalars_bit_exact(salt, name):
    """FP64 programs whose by-value scalars are powers of two run X +- s*v as
    one FMA on chunks where s*v is exact, and as the two rounded nodes
    elsewhere: the results must be the oracle's bits for every scalar
    exponent (both ends of the range, both signs, mixed with scalars that
    are not powers of two) and every operand class (ordinary, tiny and huge
    normals, subnormals, zeros, infinities, NaN), on the register-tiled
    loop and the run-time compiled kernel; the strided and staged loops and
    the batch kernel, which take every node as its own operation, must give
    the same bits."""
    prog, nv, ns = POW2_PROGS[name]
    import zlib
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    n = 4096 * 3 + 37
    scalar_sets = [[2.0 ** e, -(2.0 ** f)] for e, f in ((-2, 3), (0, -1), (-1022, 1023), (1000, -1000), (5, 0))]
    scalar_sets += [[1.5, -0.25], [-0.25, 1.5], [3.0, 0.1]]
    _, compiled = salt.salt_check_program(prog, nv, ns)
    # the staged loop and the batch kernel take compiled shapes only
    scheds = ("register", "strided", "staged", "batch") if compiled else ("register", "strided")
    try:
        for sched in scheds:
            if sched == "staged":
                salt.salt_tune_set(prog, salt.F64, n, 1, 16, 128, 0, 4096)
            for sc, runs in ((sc, runs) for sc in scalar_sets for runs in (False, True)):
                scalars = sc[:ns]
                vecs = [edge_values(rng, n, runs) for _ in range(nv)]
                want, _ = run_oracle(prog, vecs, scalars)
                if sched == "batch":
                    tv = [torch.from_numpy(v.copy()).cuda() for v in vecs]
                    b = salt.Batch(1)
                    b.add(prog, tv, scalars)
                    red = torch.zeros(4, dtype=torch.float64, device="cuda")
                    b.launch(red)
                    torch.cuda.synchronize()
                    got = [t.cpu().numpy() for t in tv]
                    b.close()
                elif sched == "strided":  # every other element of a buffer twice as long
                    bufs = [torch.zeros(2 * n, dtype=torch.float64, device="cuda") for _ in vecs]
                    for bb, v in zip(bufs, vecs):
                        bb[::2] = torch.from_numpy(v)
                    red = torch.zeros(4, dtype=torch.float64, device="cuda")
                    salt.salt_eval(prog, [bb[::2] for bb in bufs], scalars, red_out=red)
                    torch.cuda.synchronize()
                    got = [bb[::2].cpu().numpy() for bb in bufs]
                else:
                    got, _ = run_gpu(salt, prog, vecs, scalars, np.float64)
                for k, (g, w) in enumerate(zip(got, want)):
                    assert_bits_equal(g, w, f"{name} {sched} scalars {scalars} runs {runs} operand {k}")
    finally:
        salt.salt_tune_clear()


def test_fp64_rate_probe(salt, cuda_dev):
    """The register-only FP64 issue rates are positive and within the peak
    derived from unit counts (2 per clock per SM at the maximum SM clock),
    and DFMA issues about as fast as DADD and DMUL or faster (the reason
    every FP64 node issues as an FMA)."""
    props = torch.cuda.get_device_properties(cuda_dev)
    derived = 2 * props.multi_processor_count * 2.2  # G instr/s, a clock above any GB300's
    fma, add, mul = (salt.salt_fp64_rate(op) for op in (salt.FP64_FMA, salt.FP64_ADD, salt.FP64_MUL))
    for name, r in (("fma", fma), ("add", add), ("mul", mul)):
        assert 0.2 * derived < r < derived, (name, r)
    # the loops run one after another: allow for the clock moving between them
    assert fma >= 0.9 * max(add, mul), (fma, add, mul)
