"""Guard-band canaries around every contiguous output (GPU).

compute-sanitizer is not available on this machine, so out-of-bounds writes are
caught the plain way: each operand a kernel may store to, and each reduction
output, sits in the middle of a larger allocation whose guard bands before
and after it hold a signalling-NaN bit pattern that no arithmetic produces.
After the call the guards are compared bit for bit.  The paths covered are
those that write near the ends of a vector: the vector and scalar remainder
loops after the last whole tile (every unroll depth, vector width and block
shape the autotuner can pick), the staged loop's per-element tail (every
stage size), the head elements of FP32 operands that share a misalignment
(written at negative offsets from the vector body), the batch kernel's tiles
at item ends, and caller-owned outputs of the server."""
import numpy as np
import pytest

import oracle
from paper_1109_1264_gb300 import inputs
from paper_1109_1264_gb300 import programs as P
from test_gpu_parity import CONFIGS, PROGS, assert_bits_equal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

G = 1024  # guard elements on each side (a multiple of 8: views stay 32-byte aligned)
POISON = {np.float32: np.uint32(0x7FA5A5A5), np.float64: np.uint64(0x7FF4A5A5A5A5A5A5)}
IU = {np.float32: np.uint32, np.float64: np.uint64}
TDT = {np.float32: torch.float32, np.float64: torch.float64}
SIZES = [1, 2, 3, 7, 8, 63, 65, 1000, 2049, 4103, 65549, (1 << 20) + 7]


class Guarded:
    """A device copy of `host` inside a poisoned allocation: `view` starts
    `G + shift` elements into it."""

    def __init__(self, host: np.ndarray, dev, shift: int = 0):
        dt = host.dtype.type
        self.n, self.lo, self.dt = host.size, G + shift, dt
        buf = np.empty(host.size + 2 * G + shift, dt)
        buf.view(IU[dt])[:] = POISON[dt]
        buf[self.lo:self.lo + self.n] = host
        self.buf = torch.from_numpy(buf).to(dev)
        self.view = self.buf[self.lo:self.lo + self.n]

    def check(self, what):
        h = self.buf.cpu().numpy().view(IU[self.dt])
        before, after = h[:self.lo], h[self.lo + self.n:]
        bad_b = np.nonzero(before != POISON[self.dt])[0]
        bad_a = np.nonzero(after != POISON[self.dt])[0]
        assert bad_b.size == 0, f"{what}: {bad_b.size} guard elements before the view written, last at " \
                                f"{int(bad_b[-1]) - self.lo}"
        assert bad_a.size == 0, f"{what}: {bad_a.size} guard elements after the view written, first at " \
                                f"n + {int(bad_a[0])}"


def run_guarded(salt, prog, vecs, scalars, dev, shift=0, what=""):
    """Runs prog with every operand and the reduction output guarded; checks
    the guards and returns the outputs."""
    g = [Guarded(v, dev, shift) for v in vecs]
    nred = sum(1 for o, _ in prog if o in ("DOT", "SUMSQ"))
    red = Guarded(np.full(max(nred, 1), np.nan), dev) if nred else None
    salt.salt_eval(prog, [x.view for x in g], scalars, red_out=red.view if red else None)
    torch.cuda.synchronize()
    for k, x in enumerate(g):
        x.check(f"{what} operand {k}")
    if red:
        red.check(f"{what} red_out")
    return [x.view.cpu().numpy() for x in g]


@pytest.fixture(scope="module")
def salt(saltlib, cuda_dev):
    yield saltlib
    saltlib.salt_tune_clear()


@pytest.mark.parametrize("name", ["E", "AXPBY", "CG", "DOT", "SCALE"])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_canaries_register_tiled(salt, cuda_dev, name, dt):
    """Every launch configuration of the register-tiled loop, at sizes whose
    remainders exercise the guarded vector pass and the scalar pass."""
    prog, nv, ns = PROGS[name]
    code = salt.F32 if dt == np.float32 else salt.F64
    try:
        for i, n in enumerate(SIZES):
            vecs = inputs.uniform_vectors(500 + i, n, nv, dt)
            want = [v.copy() for v in vecs]
            oracle.eval_program(prog, want, [1.5, -0.25][:ns])
            cfgs = CONFIGS if n < (1 << 20) else CONFIGS[::5]
            for cfg in cfgs:
                salt.salt_tune_set(prog, code, n, *cfg)
                got = run_guarded(salt, prog, vecs, [1.5, -0.25][:ns], cuda_dev, what=f"{name} n={n} cfg={cfg}")
                for k in range(nv):
                    assert_bits_equal(got[k], want[k], f"{name} n={n} cfg={cfg} operand {k}")
    finally:
        salt.salt_tune_clear()


@pytest.mark.parametrize("stage", [4096, 8192, 16384])
@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_canaries_staged(salt, cuda_dev, stage, dt):
    """The staged loop at every stage size: whole tiles through shared memory,
    the per-element tail after the last tile."""
    code = salt.F32 if dt == np.float32 else salt.F64
    try:
        for name in ("E", "AXPBY", "CG", "DOT"):
            prog, nv, ns = PROGS[name]
            for i, n in enumerate([1, 7, 1000, 4103, 65549, (1 << 20) + 7]):
                salt.salt_tune_set(prog, code, n, 1, 16, 128, 0, stage)
                vecs = inputs.uniform_vectors(600 + i, n, nv, dt)
                want = [v.copy() for v in vecs]
                oracle.eval_program(prog, want, [1.5, -0.25][:ns])
                got = run_guarded(salt, prog, vecs, [1.5, -0.25][:ns], cuda_dev, what=f"staged {stage} {name} n={n}")
                for k in range(nv):
                    assert_bits_equal(got[k], want[k], f"staged {name} n={n} operand {k}")
    finally:
        salt.salt_tune_clear()


@pytest.mark.parametrize("shift", [1, 2, 3, 5, 7, 31])
def test_canaries_head_peeled(salt, cuda_dev, shift):
    """FP32 operands that share a misalignment of `shift` elements: the head
    elements before the next 128- (or 32-) byte boundary are written one by
    one at negative offsets from the vector body; the guard before the view
    must stay intact."""
    try:
        for name in ("E", "AXPBY", "CG", "DOT"):
            prog, nv, ns = PROGS[name]
            for i, n in enumerate([1, 2, 3, 7, 31, 33, 1000, 65549]):
                for sched in ("register", "staged"):
                    if sched == "staged":
                        salt.salt_tune_set(prog, salt.F32, n, 1, 16, 128, 0, 4096)
                    vecs = inputs.uniform_vectors(700 + i, n, nv, np.float32)
                    want = [v.copy() for v in vecs]
                    oracle.eval_program(prog, want, [1.5, -0.25][:ns])
                    got = run_guarded(salt, prog, vecs, [1.5, -0.25][:ns], cuda_dev, shift=shift,
                                      what=f"head {shift} {sched} {name} n={n}")
                    for k in range(nv):
                        assert_bits_equal(got[k], want[k], f"head {shift} {name} n={n} operand {k}")
                    salt.salt_tune_clear()
    finally:
        salt.salt_tune_clear()


@pytest.mark.parametrize("dt", [np.float32, np.float64], ids=["f32", "f64"])
def test_canaries_batch(salt, cuda_dev, dt):
    """Batch items of lengths 0..2^20 + 7, each operand in its own guarded
    allocation, for every tile size the autotuner may pick."""
    shapes = [(P.PROG_E, 5, 2), (P.PROG_AXPBY, 2, 2), (P.PROG_CG, 3, 2), (P.PROG_D, 4, 0)]
    lengths = [0, 1, 7, 100, 1000] + [(1 << k) + 7 for k in range(6, 21, 2)]
    for tile_bytes in (16384, 32768, 131072):
        b = salt.Batch(len(shapes) * len(lengths))
        items = []
        for si, (prog, nv, ns) in enumerate(shapes):
            for li, n in enumerate(lengths):
                vecs = inputs.uniform_vectors(800 + 31 * si + li, n, nv, dt)
                g = [Guarded(v, cuda_dev) for v in vecs]
                b.add(prog, [x.view for x in g], [1.5, -0.25][:ns])
                items.append((prog, ns, vecs, g))
        b.set_config(4, 128, 0, tile_bytes)
        red = Guarded(np.full(len(items), np.nan), cuda_dev)
        b.launch(red.view)
        torch.cuda.synchronize()
        red.check(f"batch red_out tile {tile_bytes}")
        for prog, ns, vecs, g in items:
            want = [v.copy() for v in vecs]
            oracle.eval_program(prog, want, [1.5, -0.25][:ns])
            for k, x in enumerate(g):
                x.check(f"batch tile {tile_bytes} n={len(vecs[0])} operand {k}")
                assert_bits_equal(x.view.cpu().numpy(), want[k], f"batch n={len(vecs[0])} operand {k}")
        b.close()


def test_canaries_served_caller_owned(salt, cuda_dev):
    """Served requests whose outputs are caller-owned device vectors (e's
    result; axpby's y, read and written) inside guarded allocations."""
    srv = salt.Server(budget_bytes=1 << 28, max_n=1 << 20)
    try:
        for dt, code in ((np.float32, salt.F32), (np.float64, salt.F64)):
            for n in (1, 7, 1000, 65549, (1 << 20) - 3):
                keys = [inputs.vector_key(41, n, k) for k in range(5)]
                host = [inputs.hash_uniform(k, n, dt) for k in keys]
                g = [Guarded(h, cuda_dev) for h in host]
                out = Guarded(np.zeros(n, dt), cuda_dev)
                a = srv.submit(P.PROG_E, code, n, keys, [1.5, -0.25], ptrs=[x.view for x in g[:4]] + [out.view])
                yb = srv.submit(P.PROG_AXPBY, code, n, keys[:2], [1.5, -0.25], ptrs=[g[0].view, g[4].view])
                for rid in (a, yb):
                    srv.wait(rid, 20_000_000)
                for x in g + [out]:
                    x.check(f"served n={n}")
                want = [h.copy() for h in host[:4]] + [np.zeros(n, dt)]
                oracle.eval_program(P.PROG_E, want, [1.5, -0.25])
                assert_bits_equal(out.view.cpu().numpy(), want[4], f"served e n={n}")
                want_y = [host[0].copy(), host[4].copy()]
                oracle.eval_program(P.PROG_AXPBY, want_y, [1.5, -0.25])
                assert_bits_equal(g[4].view.cpu().numpy(), want_y[1], f"served axpby n={n}")
                for rid in (a, yb):
                    srv.release(rid)
    finally:
        srv.stop()
