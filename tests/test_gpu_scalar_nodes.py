"""Scalar subexpressions, elementwise DIV and device-resident scalars on the
GPU, against the oracle: elementwise results bit-identical (scalar nodes are
one operation each in the program's dtype, computed once per launch),
reductions within tolerance, and conjugate gradients driven entirely by
device scalars (alpha = rho / (p.q), beta = rho' / rho) with no host read
between its steps."""
import math
import random

import numpy as np
import pytest

import oracle
from oracle_pins import (CG_P, CG_P0, CG_PQ, CG_Q_PQ, CG_R0, CG_XR_RHO, cg_diagonal, cg_diagonal_two_pass,
                         random_program)
from oracle import exact
import tolerance
from test_gpu_parity import TOL, assert_bits_equal, check_reductions

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TDT = {np.float32: torch.float32, np.float64: torch.float64}
AXPY_DS = [("DSCAL", 0), ("DSCAL", 1), ("DIV", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("ADD", 0),
           ("STORE", 1)]


def _signed(rng, n, dt):
    """Magnitudes in [0.5, 2) with random signs: quotients stay in range."""
    return (rng.uniform(0.5, 2.0, n) * rng.choice([-1.0, 1.0], n)).astype(dt)


def _run(s, prog, vecs, scalars, dscalars, dev, views=None):
    tv = [torch.from_numpy(v.copy()).to(dev) for v in vecs] if views is None else views
    nred = sum(1 for o, _ in prog if o in ("DOT", "SUMSQ"))
    red = torch.full((max(nred, 1),), float("nan"), dtype=torch.float64, device=dev)
    ds = torch.tensor(list(dscalars) or [0.0], dtype=torch.float64, device=dev)
    s.salt_eval(prog, tv, scalars, red_out=red if nred else None,
                dscalars=[ds[k:k + 1] for k in range(len(dscalars))] if dscalars else None)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in tv], red.cpu().numpy()[:nred]


def _check(prog, vecs, scalars, dscalars, got, red, dt, what):
    want = [v.copy() for v in vecs]
    oracle.eval_program(prog, want, scalars, dscalars=dscalars)
    for k, (g, w) in enumerate(zip(got, want)):
        assert_bits_equal(g, w, f"{what} operand {k}")
    if red.size and all(np.all(np.isfinite(w)) for w in want):
        check_reductions(prog, vecs, scalars, red, dt, what, dscalars=dscalars)


@pytest.mark.parametrize("jit", [False, True], ids=["interp", "jit"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_random_extended_programs(saltlib, cuda_dev, dt, jit):
    """Random programs with DIV, scalar-typed nodes and device scalars."""
    s = saltlib
    rng = random.Random(31 + jit)
    nrng = np.random.default_rng(31)
    prev = s.salt_jit_stats()["mode"]
    s.salt_set_jit(s.JIT_ON if jit else s.JIT_OFF)
    try:
        done = 0
        while done < 24:
            nv, ns, nd = rng.randint(1, 5), rng.randint(0, 2), rng.randint(1, 3)
            prog = random_program(rng, nv, ns, max_len=12, ndscal=nd, ext=True)
            try:
                s.salt_check_program(prog, nv, ns)
            except s.SaltError:
                continue  # beyond the library's size limits
            for n in (1, 7, 1000, 70001):
                vecs = [_signed(nrng, n, dt) for _ in range(nv)]
                scalars = list(nrng.uniform(0.5, 2.0, ns))
                dscalars = list(nrng.uniform(-2.0, 2.0, nd))
                got, red = _run(s, prog, vecs, scalars, dscalars, cuda_dev)
                _check(prog, vecs, scalars, dscalars, got, red, dt, f"{prog} n={n}")
            done += 1
    finally:
        s.salt_set_jit(prev)


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_hoisted_subexpressions_on_compiled_shapes(saltlib, cuda_dev, dt):
    """Programs whose scalar subtrees hoist to a slot run on the compiled
    kernels: the slot computed at kernel start (device scalars) or on the
    host (by-value scalars) gives the oracle's bits, including the FP32
    rounding of each scalar node."""
    s = saltlib
    nrng = np.random.default_rng(32)
    folded = [("SCAL", 0), ("SCAL", 1), ("MUL", 0), ("NEG", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1),
              ("ADD", 0), ("STORE", 1)]
    e_ds = [("DSCAL", 0), ("VEC", 0), ("SMUL", 0), ("DSCAL", 1), ("DSCAL", 2), ("SUB", 0), ("VEC", 1),
            ("SMUL", 0), ("ADD", 0), ("VEC", 2), ("VEC", 3), ("MUL", 0), ("SUB", 0), ("STORE", 4)]
    cases = [(AXPY_DS, 2, (), (3.0, 7.0)),
             (AXPY_DS, 2, (), (1.0 + 2.0 ** -24 + 2.0 ** -40, 1.0 + 2.0 ** -23)),
             (folded, 2, (1.0 / 3.0, -2.5), ()),
             (folded, 2, (1.0, 1.0 + 2.0 ** -24), ()),
             (e_ds, 5, (), (1.5, 0.75, 1.0))]
    for prog, nv, scalars, dscalars in cases:
        assert s.salt_check_program(prog, nv, len(scalars))[1], prog
        for n in (1, 5, 4096 + 7, (1 << 20) + 3):
            vecs = [nrng.uniform(-1, 1, n).astype(dt) for _ in range(nv)]
            got, red = _run(s, prog, vecs, scalars, dscalars, cuda_dev)
            _check(prog, vecs, scalars, dscalars, got, red, dt, f"{prog} n={n}")


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_device_scalars_with_strided_operands(saltlib, cuda_dev, dt):
    s = saltlib
    nrng = np.random.default_rng(33)
    for n in (3, 999, 65537):
        vecs = [nrng.uniform(-1, 1, n).astype(dt) for _ in range(2)]
        bufs = [torch.full((2 * n + 1,), 7.0, dtype=TDT[dt], device=cuda_dev) for _ in range(2)]
        for b, v in zip(bufs, vecs):
            b[0:2 * n:2] = torch.from_numpy(v).to(cuda_dev)
        views = [b[0:2 * n:2] for b in bufs]
        got, _ = _run(s, AXPY_DS, vecs, (), (2.0, -3.0), cuda_dev, views=views)
        _check(AXPY_DS, vecs, (), (2.0, -3.0), got, np.zeros(0), dt, f"strided n={n}")
        assert torch.all(bufs[1][1::2] == 7.0)


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_device_scalar_follows_stream_order(saltlib, cuda_dev, dt):
    """A DOT result written by one call steers the next call on the same
    stream with no synchronisation between them.  The dot is of integer-
    valued vectors, so its value is the exact integer (checked), which the
    oracle then takes as the device scalar."""
    s = saltlib
    nrng = np.random.default_rng(34)
    n = (1 << 22) + 5
    xi = nrng.integers(-8, 8, n)
    yi = nrng.integers(-8, 8, n)
    x, y = xi.astype(dt), yi.astype(dt)
    dot = int(np.dot(xi, yi))
    scale = 2.0 ** -20  # keeps y + dot * 2^-20 * x inexact in FP32 and FP64
    tx, ty = (torch.from_numpy(v.copy()).to(cuda_dev) for v in (x, y))
    red = torch.zeros(2, dtype=torch.float64, device=cuda_dev)
    s.salt_eval([("VEC", 0), ("VEC", 1), ("DOT", 0)], [tx, ty], red_out=red[0:1])
    prog = [("DSCAL", 0), ("SCAL", 0), ("MUL", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("ADD", 0),
            ("STORE", 1)]
    s.salt_eval(prog, [tx, ty], [scale], dscalars=[red[0:1]])
    torch.cuda.synchronize()
    assert float(red[0].cpu()) == float(dot)
    want = [x.copy(), y.copy()]
    oracle.eval_program(prog, want, [scale], dscalars=[float(dot)])
    assert_bits_equal(ty.cpu().numpy(), want[1], "y")


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_cg_diagonal_device_scalars(saltlib, cuda_dev, dt):
    """CG for diag(d) x = b with every scalar on the device: three calls per
    iteration, reduction results feeding DSCAL nodes, one synchronisation at
    the end.  Four distinct eigenvalues: converged after four iterations,
    and close to the oracle's CG iterate (the two differ only through the
    rounding of their reductions)."""
    s = saltlib
    rng = np.random.default_rng(35)
    for n in (1001, (1 << 20) + 3):
        d = rng.choice([1.0, 2.0, 5.0, 8.0], n).astype(dt)
        b = rng.uniform(-1, 1, n).astype(dt)
        iters = 4
        tv = [torch.from_numpy(v.copy()).to(cuda_dev) for v in (d, b, np.zeros(n, dt), np.zeros(n, dt), b)]
        red = torch.zeros(1 + 2 * iters, dtype=torch.float64, device=cuda_dev)
        s.salt_eval([("VEC", 4), ("SUMSQ", 0)], tv, red_out=red[0:1])
        rho = 0
        for i in range(iters):
            pq, rho_new = 1 + 2 * i, 2 + 2 * i
            s.salt_eval(CG_Q_PQ, tv, red_out=red[pq:pq + 1])
            s.salt_eval(CG_XR_RHO, tv, red_out=red[rho_new:rho_new + 1],
                        dscalars=[red[rho:rho + 1], red[pq:pq + 1]])
            s.salt_eval(CG_P, tv, dscalars=[red[rho_new:rho_new + 1], red[rho:rho + 1]])
            rho = rho_new
        torch.cuda.synchronize()
        x = tv[3].cpu().numpy().astype(np.float64)
        xs = b.astype(np.float64) / d.astype(np.float64)
        err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
        assert err < (1e-13 if dt == np.float64 else 2e-6), (n, err)
        res = red.cpu().numpy()
        assert math.sqrt(res[2 * iters]) < (1e-13 if dt == np.float64 else 2e-6) * math.sqrt(res[0])

        def evalp(prog, vecs, ds):
            return oracle.eval_program(prog, vecs, dscalars=ds)

        xo, _ = cg_diagonal(evalp, d, b, iters)
        rel = np.linalg.norm(x - xo) / np.linalg.norm(xo)
        assert rel < (1e-12 if dt == np.float64 else 1e-5), (n, rel)


def test_batch_folds_by_value_scalar_subexpressions(saltlib, cuda_dev):
    """A batch item whose scalars are a subexpression of by-value scalars runs
    on the batch kernel with the folded value: the same bits as salt_eval."""
    s = saltlib
    nrng = np.random.default_rng(36)
    folded = [("SCAL", 0), ("SCAL", 1), ("DIV", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("ADD", 0),
              ("STORE", 1)]
    n = 10007
    for dt in (np.float32, np.float64):
        x, y = (nrng.uniform(-1, 1, n).astype(dt) for _ in range(2))
        tx, ty = (torch.from_numpy(v).to(cuda_dev) for v in (x, y))
        b = s.Batch(capacity=4)
        try:
            b.add(folded, [tx, ty], [1.0, 3.0])
            b.launch(torch.zeros(1, dtype=torch.float64, device=cuda_dev))
            torch.cuda.synchronize()
        finally:
            b.close()
        want = [x.copy(), y.copy()]
        oracle.eval_program(folded, want, [1.0, 3.0])
        assert_bits_equal(ty.cpu().numpy(), want[1], f"batch {dt.__name__}")


CG_SLOTS = ("d", "p", "q", "x", "r", "b")


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_cg_passes_bit_exact(saltlib, cuda_dev, dt):
    """The four programs of salt_cg_diag on the compiled device-scalar
    kernels, with device scalars uploaded from the host: vectors bit-identical
    to the oracle's, reductions within tolerance of the exact value."""
    s = saltlib
    rng = np.random.default_rng(38)
    for n in (1, 999, (1 << 20) + 5):
        vals = {"d": rng.uniform(1, 8, n), "p": rng.uniform(-1, 1, n), "q": np.zeros(n),
                "x": rng.uniform(-3, 3, n), "r": rng.uniform(-1, 1, n), "b": rng.uniform(-1, 1, n)}
        vecs = [vals[k].astype(dt) for k in CG_SLOTS]
        dscal = [0.75, 1.0 / 3.0]
        for prog in (CG_R0, CG_P0, CG_PQ, CG_XR_RHO):
            assert s.salt_check_program(prog, 6, 0)[1], prog
            ds = dscal if any(o == "DSCAL" for o, _ in prog) else ()
            got, red = _run(s, prog, vecs, (), ds, cuda_dev)
            _check(prog, vecs, (), ds, got, red, dt, f"{prog[:3]} n={n}")


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_cg_diag_entry_point(saltlib, cuda_dev, dt):
    """salt_cg_diag from x0 != 0: converged to b / d in four iterations (four
    distinct eigenvalues), its residual history consistent with x, and close
    to the oracle's own two-pass CG (the two differ only through the rounding
    of their reductions)."""
    s = saltlib
    rng = np.random.default_rng(37)
    for n in (999, (1 << 20) + 5):
        d = rng.choice([1.0, 2.0, 5.0, 8.0], n).astype(dt)
        b = rng.uniform(-1, 1, n).astype(dt)
        x0 = rng.uniform(-3, 3, n).astype(dt)
        iters = 4
        td, tb, tx = (torch.from_numpy(v.copy()).to(cuda_dev) for v in (d, b, x0))
        tr, tp, tq = (torch.zeros(n, dtype=TDT[dt], device=cuda_dev) for _ in range(3))
        rho = torch.full((2 * iters + 1,), float("nan"), dtype=torch.float64, device=cuda_dev)
        s.salt_cg_diag(td, tb, tx, tr, tp, tq, iters, rho)
        torch.cuda.synchronize()
        g = rho.cpu().numpy()
        xg = tx.cpu().numpy().astype(np.float64)
        rg = tr.cpu().numpy()
        xs = b.astype(np.float64) / d.astype(np.float64)
        tol = 1e-12 if dt == np.float64 else 2e-5
        assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) < tol
        # rho_0 = |b - d x0|^2 of the host data, rho_4 = |r|^2 of the returned r
        # r_0 = b - d x0 elementwise in the vectors' dtype (one rounding per
        # node, as the kernels do), so rho_0 has an exact reference
        r0 = b - d * x0
        sq0 = exact.exact_sumsq(r0)
        tolerance.check(g[0], sq0, sq0, dt, "rho_0")
        sq = exact.exact_sumsq(rg)
        tolerance.check(g[-1], sq, sq, dt, "rho of the returned r")
        # The oracle's own iterate differs through its reductions only: a
        # sequential FP64 sum is off by up to gamma_n relative (about 1e-10
        # at n = 2^20; a few 1e-13 typically), which perturbs alpha and beta.
        xo, ho = cg_diagonal_two_pass(lambda pr, vs, ds: oracle.eval_program(pr, vs, dscalars=ds), d, b, x0, iters)
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < (1e-10 if dt == np.float64 else 1e-5)
        assert abs(g[2] - ho[2]) <= (1e-9 if dt == np.float64 else 1e-5) * ho[2]


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_cg_persistent(saltlib, cuda_dev, dt):
    """salt_cg_diag_persistent (one cooperative launch, grid barriers): the
    same convergence, residual history and agreement with the oracle's CG as
    the launch-per-pass form, and agreement with that form to the reductions'
    tolerance."""
    s = saltlib
    rng = np.random.default_rng(39)
    for n, iters in ((0, 3), (1, 1), (999, 4), (4096, 0), ((1 << 20) + 5, 4)):
        d = rng.choice([1.0, 2.0, 5.0, 8.0], n).astype(dt)
        b = rng.uniform(-1, 1, n).astype(dt)
        x0 = rng.uniform(-3, 3, n).astype(dt)
        runs = {}
        for persistent in (False, True):
            td, tb, tx = (torch.from_numpy(v.copy()).to(cuda_dev) for v in (d, b, x0))
            tr, tp, tq = (torch.zeros(n, dtype=TDT[dt], device=cuda_dev) for _ in range(3))
            rho = torch.full((2 * iters + 1,), float("nan"), dtype=torch.float64, device=cuda_dev)
            s.salt_cg_diag(td, tb, tx, tr, tp, tq, iters, rho, persistent=persistent)
            torch.cuda.synchronize()
            runs[persistent] = (tx.cpu().numpy().astype(np.float64), tr.cpu().numpy(), rho.cpu().numpy())
        xg, rg, g = runs[True]
        xl, _, gl = runs[False]
        assert not np.any(np.isnan(g)) or n == 0, g
        if n == 0:
            assert np.all(xg.shape == (0,)) and g[0] == 0.0
            continue
        r0 = b - d * x0  # in the vectors' dtype, as the kernels compute it
        sq0 = exact.exact_sumsq(r0)
        tolerance.check(g[0], sq0, sq0, dt, ("rho_0", n))
        sq = exact.exact_sumsq(rg)
        tolerance.check(g[-1], sq, sq, dt, ("rho of the returned r", n))
        if iters == 4 and n > 1:
            xs = b.astype(np.float64) / d.astype(np.float64)
            tol = 1e-12 if dt == np.float64 else 2e-5
            assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) < tol
            xo, _ = cg_diagonal_two_pass(lambda pr, vs, ds: oracle.eval_program(pr, vs, dscalars=ds), d, b, x0,
                                         iters)
            assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < (1e-10 if dt == np.float64 else 1e-5)
        # against the launch-per-pass form: the start residual agrees to the
        # reduction tolerance, the iterates to the propagated rounding
        tolerance.check(g[0], gl[0], gl[0], dt, ("rho_0 of the two forms", n), factor=2.0)
        if iters:
            assert np.linalg.norm(xg - xl) <= (1e-10 if dt == np.float64 else 1e-4) * max(np.linalg.norm(xl), 1.0)


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_cg_one_reduction(saltlib, cuda_dev, dt):
    """salt_cg_diag_one_reduction (one pass and one grid barrier per
    iteration): its start gamma_0 and last gamma equal r.r of the start and
    returned residuals within the reduction tolerance; after 4 iterations on
    4 distinct eigenvalues it reaches the solution; its iterates agree with
    the oracle's one-reduction CG (same recurrence; the scalars differ only
    through the reductions' rounding) and with the two-pass Hestenes-Stiefel
    form on the GPU to the propagated rounding."""
    from oracle_pins import cg_diagonal_one_reduction
    s = saltlib
    rng = np.random.default_rng(41)
    for n, iters in ((0, 3), (1, 1), (999, 4), (4096, 0), ((1 << 20) + 5, 4), (70001, 9)):
        if iters == 9:
            d = rng.uniform(1.0, 4.0, n).astype(dt)
        else:
            d = rng.choice([1.0, 2.0, 5.0, 8.0], n).astype(dt)
        b = rng.uniform(-1, 1, n).astype(dt)
        x0 = rng.uniform(-3, 3, n).astype(dt)
        td, tb, tx = (torch.from_numpy(v.copy()).to(cuda_dev) for v in (d, b, x0))
        tr, tp, ts = (torch.zeros(n, dtype=TDT[dt], device=cuda_dev) for _ in range(3))
        rho = torch.full((2 * iters + 2,), float("nan"), dtype=torch.float64, device=cuda_dev)
        s.salt_cg_diag(td, tb, tx, tr, tp, ts, iters, rho, one_reduction=True)
        td2, tb2, tx2 = (torch.from_numpy(v.copy()).to(cuda_dev) for v in (d, b, x0))
        tr2, tp2, tq2 = (torch.zeros(n, dtype=TDT[dt], device=cuda_dev) for _ in range(3))
        rho2 = torch.full((2 * iters + 1,), float("nan"), dtype=torch.float64, device=cuda_dev)
        s.salt_cg_diag(td2, tb2, tx2, tr2, tp2, tq2, iters, rho2)
        torch.cuda.synchronize()
        xg, rg, g = tx.cpu().numpy().astype(np.float64), tr.cpu().numpy(), rho.cpu().numpy()
        xl = tx2.cpu().numpy().astype(np.float64)
        if n == 0:
            assert xg.shape == (0,) and g[0] == 0.0
            continue
        assert not np.any(np.isnan(g)), g
        # gamma_0 = r0.r0 and delta_0 = (d o r0).r0 with r0 = b - d x0, and the
        # last gamma, delta of the returned residual, each product d o r
        # rounded in the vectors' dtype as the kernel forms it
        r0 = b - d * x0
        sq0 = exact.exact_sumsq(r0)
        tolerance.check(g[0], sq0, sq0, dt, ("gamma_0", n))
        tolerance.check_dot(g[1], d * r0, r0, dt, ("delta_0", n))
        sq = exact.exact_sumsq(rg)
        tolerance.check(g[-2], sq, sq, dt, ("last gamma", n, iters))
        tolerance.check_dot(g[-1], d * rg, rg, dt, ("last delta", n, iters))
        if iters == 4 and n > 1:
            xs = b.astype(np.float64) / d.astype(np.float64)
            tol = 1e-11 if dt == np.float64 else 1e-4
            assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) < tol
        if iters:
            xo, ho = cg_diagonal_one_reduction(lambda pr, vs, ds: oracle.eval_program(pr, vs, dscalars=ds), d, b,
                                               x0, iters)
            scale = max(np.linalg.norm(xo.astype(np.float64)), 1.0)
            tx_ = 1e-10 if dt == np.float64 else 1e-4
            assert np.linalg.norm(xg - xo) <= tx_ * scale, (n, iters)
            assert np.linalg.norm(xg - xl) <= tx_ * max(np.linalg.norm(xl), 1.0), (n, iters)
            for j in range(iters + 1):
                assert abs(g[2 * j] - ho[2 * j]) <= tx_ * ho[0] + 1e-300, (n, iters, j)


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_cg_auto_and_autotune(saltlib, cuda_dev, dt):
    """salt_cg_diag_auto runs the form its table names, bit for bit the same
    as calling that form directly; salt_cg_autotune times the three forms,
    gives x back as passed, and pins the winner for the size's bucket."""
    s = saltlib
    rng = np.random.default_rng(43)
    code = s.F32 if dt == np.float32 else s.F64
    iters = 4
    try:
        for n in (999, 70001, (1 << 20) + 5):
            d = rng.choice([1.0, 2.0, 5.0, 8.0], n).astype(dt)
            b = rng.uniform(-1, 1, n).astype(dt)
            x0 = rng.uniform(-3, 3, n).astype(dt)

            def fresh():
                td, tb, tx = (torch.from_numpy(v.copy()).to(cuda_dev) for v in (d, b, x0))
                return [td, tb, tx] + [torch.zeros(n, dtype=TDT[dt], device=cuda_dev) for _ in range(3)]

            for form in (s.CG_TWO_PASS, s.CG_PERSISTENT, s.CG_ONE_REDUCTION):
                s.salt_cg_form_set(code, n, form)
                va = fresh()
                rho_a = torch.zeros(2 * iters + 2, dtype=torch.float64, device=cuda_dev)
                assert s.salt_cg_diag_auto(*va, iters, rho_a) == form
                vd = fresh()
                rho_d = torch.zeros(2 * iters + 2, dtype=torch.float64, device=cuda_dev)
                s.salt_cg_diag(*vd, iters, rho_d, persistent=form == s.CG_PERSISTENT,
                               one_reduction=form == s.CG_ONE_REDUCTION)
                torch.cuda.synchronize()
                assert torch.equal(va[2], vd[2]) and torch.equal(rho_a, rho_d), (n, form)
                xs = b.astype(np.float64) / d.astype(np.float64)
                xg = va[2].cpu().numpy().astype(np.float64)
                assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) < (1e-11 if dt == np.float64 else 1e-4)
            s.salt_cg_form_set(code, n, -1)
            v = fresh()
            rho = torch.zeros(2 * iters + 2, dtype=torch.float64, device=cuda_dev)
            form, ms = s.salt_cg_autotune(*v, iters, rho, reps=2)
            assert form in (s.CG_TWO_PASS, s.CG_PERSISTENT, s.CG_ONE_REDUCTION) and ms > 0
            assert s.salt_cg_form_get(code, n) == form
            assert np.array_equal(v[2].cpu().numpy(), x0)  # x given back as passed
    finally:
        for n in (999, 70001, (1 << 20) + 5):
            s.salt_cg_form_set(code, n, -1)
