"""The library's two bounded device waits, made to run out on purpose (GPU).

Nothing here faults or hangs: a wait whose poll limit is 0 gives up at once,
with every copy and every memory access still valid.

* Staged loop: thread 0 of a block stops waiting for a tile's bulk copies,
  counts a timeout, and the block computes that tile and every later one
  from direct loads; before it exits it still waits, with the full bound,
  for the copies it issued.  Results must not change.
* Cooperative CG: a grid barrier that runs out records a timeout in the
  stream's status word; every block returns at its next barrier, rho[0]
  becomes NaN, and salt_cg_status reports SALT_ERR_TIMEOUT.
"""
import math

import numpy as np
import pytest

import oracle
import tolerance
from paper_1109_1264_gb300 import inputs
from paper_1109_1264_gb300 import programs as P
from test_gpu_parity import assert_bits_equal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TDT = {np.float32: torch.float32, np.float64: torch.float64}


@pytest.fixture
def salt(saltlib, cuda_dev):
    s = saltlib
    yield s
    s.salt_set_wait_limit(s.WAIT_STAGED, s.WAIT_DEFAULT_POLLS)
    s.salt_set_wait_limit(s.WAIT_CG_BARRIER, s.WAIT_DEFAULT_POLLS)
    s.salt_tune_clear()


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_staged_wait_runs_out(salt, cuda_dev, dt):
    """With the staged loop's tile wait limited to 0 polls, every block gives
    up staging at its first tile (timeouts counted) and finishes from direct
    loads: e and axpby bit-identical to the oracle, dot within tolerance; with
    the default limit restored, no wait runs out."""
    s = salt
    code = s.F32 if dt == np.float32 else s.F64
    n = (1 << 20) + 7
    a, b, c, d, y = inputs.uniform_vectors(90, n, 5, dt)
    for prog in (P.PROG_E, P.PROG_AXPBY, P.PROG_DOT):
        s.salt_tune_set(prog, code, n, 1, 16, 128, 0, 4096)  # staged loop, many tiles per block

    def run():
        ta, tb, tc, td, ty = (torch.from_numpy(v.copy()).to(cuda_dev) for v in (a, b, c, d, y))
        out = torch.zeros(n, dtype=TDT[dt], device=cuda_dev)
        red = torch.full((1,), float("nan"), dtype=torch.float64, device=cuda_dev)
        s.salt_eval(P.PROG_E, [ta, tb, tc, td, out], [1.5, -0.25])
        s.salt_axpby(1.5, ta, -0.25, ty)
        s.salt_dot(ta, tb, red)
        torch.cuda.synchronize()
        return out.cpu().numpy(), ty.cpu().numpy(), red.item()

    want_e = [a.copy(), b.copy(), c.copy(), d.copy(), np.zeros(n, dt)]
    oracle.eval_program(oracle.PROG_E, want_e, [1.5, -0.25])
    want_y = [a.copy(), y.copy()]
    oracle.eval_program(oracle.PROG_AXPBY, want_y, [1.5, -0.25])

    before = s.salt_staged_timeouts()
    s.salt_set_wait_limit(s.WAIT_STAGED, 0)
    assert s.salt_get_wait_limit(s.WAIT_STAGED) == 0
    e, yy, dot = run()
    after = s.salt_staged_timeouts()
    assert after > before, (before, after)  # the waits ran out ...
    assert_bits_equal(e, want_e[4], "e after timed-out stage waits")  # ... and nothing changed
    assert_bits_equal(yy, want_y[1], "axpby after timed-out stage waits")
    tolerance.check_dot(dot, a, b, dt, "dot after timed-out stage waits")

    s.salt_set_wait_limit(s.WAIT_STAGED, s.WAIT_DEFAULT_POLLS)
    e, yy, dot = run()
    assert s.salt_staged_timeouts() == after
    assert_bits_equal(e, want_e[4], "e")
    assert_bits_equal(yy, want_y[1], "axpby")
    tolerance.check_dot(dot, a, b, dt, "dot")


@pytest.mark.parametrize("one_reduction", [False, True], ids=["two_barriers", "one_reduction"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_cg_barrier_runs_out(salt, cuda_dev, dt, one_reduction):
    """With the grid barrier limited to 0 polls, a launch of several blocks
    ends early: salt_cg_status reports SALT_ERR_TIMEOUT and rho[0] is NaN.
    A one-block launch never waits (its barriers are passed on arrival) and
    completes normally.  With the default limit restored the same call
    converges and the status is SALT_OK."""
    s = salt
    rng = np.random.default_rng(47)
    iters = 4
    for n, blocks in (((1 << 20) + 5, "several"), (999, "one")):
        d = rng.choice([1.0, 2.0, 5.0, 8.0], n).astype(dt)
        b = rng.uniform(-1, 1, n).astype(dt)
        x0 = rng.uniform(-3, 3, n).astype(dt)

        def run():
            td, tb, tx = (torch.from_numpy(v.copy()).to(cuda_dev) for v in (d, b, x0))
            tr, tp, tq = (torch.zeros(n, dtype=TDT[dt], device=cuda_dev) for _ in range(3))
            rho = torch.zeros(2 * iters + 2, dtype=torch.float64, device=cuda_dev)
            s.salt_cg_diag(td, tb, tx, tr, tp, tq, iters, rho, persistent=not one_reduction,
                           one_reduction=one_reduction)
            return tx, rho

        s.salt_set_wait_limit(s.WAIT_CG_BARRIER, 0)
        tx, rho = run()
        if blocks == "several":
            with pytest.raises(s.SaltError) as ei:
                s.salt_cg_status()
            assert ei.value.status == s.ERR_TIMEOUT
            assert math.isnan(rho[0].item())
        else:
            s.salt_cg_status()
            assert not np.any(np.isnan(rho.cpu().numpy()))
        s.salt_set_wait_limit(s.WAIT_CG_BARRIER, s.WAIT_DEFAULT_POLLS)
        tx, rho = run()
        s.salt_cg_status()  # SALT_OK
        g = rho.cpu().numpy()
        assert not np.any(np.isnan(g))
        xs = b.astype(np.float64) / d.astype(np.float64)
        xg = tx.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) < (1e-11 if dt == np.float64 else 1e-4)


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_trace_timeline(salt, cuda_dev, dt):
    """salt_trace_set: a traced launch writes one record per block -- start
    <= whole tiles done <= before the combine <= end, an SM id below the
    SM count, exactly one block marked as the final combine -- and the
    traced call's results equal the untraced call's."""
    s = salt
    n = (1 << 22) + 5
    x, y = (torch.from_numpy(v).to(cuda_dev) for v in inputs.uniform_vectors(93, n, 2, dt))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cap = sms * 32
    trace = torch.zeros(cap * s.TRACE_WORDS, dtype=torch.int64, device=cuda_dev)
    out = torch.zeros(4, dtype=torch.float64, device=cuda_dev)
    s.salt_dot(x, y, out[0:1])
    s.salt_nrm2(x, out[1:2])
    for k, fn in ((2, lambda r: s.salt_dot(x, y, r)), (3, lambda r: s.salt_nrm2(x, r))):
        trace.zero_()
        s.salt_trace_set(trace, cap)
        try:
            fn(out[k:k + 1])
            torch.cuda.synchronize()
        finally:
            s.salt_trace_set(None)
        w = trace.view(-1, s.TRACE_WORDS).cpu().numpy()
        w = w[w[:, 0] != 0]
        assert w.shape[0] >= 2
        assert np.all(w[:, 0] <= w[:, 1]) and np.all(w[:, 1] <= w[:, 2]) and np.all(w[:, 2] <= w[:, 3])
        assert np.all(w[:, 4] < sms) and int(w[:, 5].sum()) == 1
        # the final combine ends last
        assert w[w[:, 5] == 1, 3][0] == w[:, 3].max()
    got = out.cpu().numpy()
    assert got[2] == got[0] and got[3] == got[1]
    # tracing off: nothing is written
    trace.zero_()
    s.salt_dot(x, y, out[0:1])
    torch.cuda.synchronize()
    assert int(trace.abs().sum().item()) == 0
