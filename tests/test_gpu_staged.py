"""The staged loop (stage_bytes != 0: operand tiles copied into shared memory
by bulk asynchronous copies, two stages deep) against the oracle (GPU).

Element results must be bit-identical to the oracle's node-by-node
evaluation, reductions within the tolerance of the exactly rounded
reference, for every compiled shape, both dtypes and every stage size, at
lengths with no whole tile (tail only), exactly one tile, several tiles with
a ragged tail, and many tiles per block (the two stages each reused many
times, so both mbarrier phase parities recur)."""
import numpy as np
import pytest

import oracle
from oracle_pins import CG_PQ, CG_R0, CG_XR_RHO
from paper_1109_1264_gb300 import inputs
from test_gpu_parity import PROGS, assert_bits_equal, check_reductions, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (stage_bytes, block, blocks_per_sm)
STAGED = [(4096, 128, 0), (8192, 256, 1), (16384, 256, 0), (16384, 64, 2)]


def tile_elems(sb, dt):
    return sb // np.dtype(dt).itemsize


def sizes_for(sb, dt):
    te = tile_elems(sb, dt)
    return [1, te - 1, te, 5 * te + 3, (3 << 20) + 5]


@pytest.fixture(scope="module")
def salt(saltlib, cuda_dev):
    return saltlib


@pytest.mark.parametrize("name", list(PROGS))
@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
def test_staged_every_shape_bit_exact(salt, name, dt):
    prog, nv, ns = PROGS[name]
    code = salt.F32 if dt == np.float32 else salt.F64
    scalars = [1.5, -0.25][:ns]
    try:
        for sb, blk, bps in STAGED:
            for i, n in enumerate(sizes_for(sb, dt)):
                vecs = inputs.uniform_vectors(300 + i, n, nv, dt)
                salt.salt_tune_set(prog, code, n, 1, 16, blk, bps, sb)
                assert salt.salt_tune_get(prog, code, n)["stage_bytes"] == sb
                got, red = run_gpu(salt, prog, vecs, scalars, dt)
                want, _ = run_oracle(prog, vecs, scalars)
                what = f"{name} stage={sb} block={blk} bps={bps} n={n}"
                for k, (g, w) in enumerate(zip(got, want)):
                    assert_bits_equal(g, w, f"{what} operand {k}")
                check_reductions(prog, vecs, scalars, red, dt, what)
    finally:
        salt.salt_tune_clear()
    assert salt.salt_staged_timeouts() == 0


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
def test_staged_device_scalar_passes(salt, cuda_dev, dt):
    """The conjugate-gradient passes with device-scalar quotients (scalar
    code run by thread 0 of every block) on the staged loop."""
    code = salt.F32 if dt == np.float32 else salt.F64
    tdt = torch.float32 if dt == np.float32 else torch.float64
    n = (1 << 20) + 37
    d, p, q, x, r, b = inputs.uniform_vectors(41, n, 6, dt)
    d = np.abs(d) + dt(1.0)
    vecs = [d, p, np.zeros(n, dt), x, r, b]
    dsv = [0.75, 1.0 / 3.0, 2.5]
    try:
        for sb, blk, bps in STAGED:
            for prog in (CG_R0, CG_PQ, CG_XR_RHO):
                salt.salt_tune_set(prog, code, n, 1, 16, blk, bps, sb)
            tv = [torch.from_numpy(v.copy()).to(cuda_dev) for v in vecs]
            ds = torch.tensor(dsv, dtype=torch.float64, device=cuda_dev)
            red = torch.zeros(3, dtype=torch.float64, device=cuda_dev)
            salt.salt_eval(CG_R0, tv, red_out=red[0:1])
            salt.salt_eval(CG_PQ, tv, red_out=red[1:2], dscalars=[ds[0:1], ds[1:2]])
            salt.salt_eval(CG_XR_RHO, tv, red_out=red[2:3], dscalars=[ds[0:1], ds[2:3]])
            torch.cuda.synchronize()
            want = [v.copy() for v in vecs]
            wr0 = oracle.eval_program(CG_R0, want)
            vs_pq = [v.copy() for v in want]
            wpq = oracle.eval_program(CG_PQ, want, dscalars=dsv[0:2])
            vs_xr = [v.copy() for v in want]
            wxr = oracle.eval_program(CG_XR_RHO, want, dscalars=[dsv[0], dsv[2]])
            for k in range(6):
                assert_bits_equal(tv[k].cpu().numpy(), want[k], f"stage={sb} operand {k}")
            got = red.cpu().numpy()
            check_reductions(CG_PQ, vs_pq, [], got[1:2], dt, f"stage={sb} p.q", dscalars=dsv[0:2])
            check_reductions(CG_XR_RHO, vs_xr, [], got[2:3], dt, f"stage={sb} rho", dscalars=[dsv[0], dsv[2]])
            assert np.isfinite(wr0).all() and np.isfinite(wpq).all() and np.isfinite(wxr).all()
    finally:
        salt.salt_tune_clear()
    assert salt.salt_staged_timeouts() == 0


@pytest.mark.parametrize("layout", ["same_offset", "mixed_offsets"])
def test_staged_unaligned_operands(salt, cuda_dev, layout):
    """A staged configuration with FP32 operands that are not 16-byte
    aligned: all at the same offset, the staged loop runs from the next
    128-byte boundary and the head elements are evaluated one by one; at
    different offsets the element-access kernel runs.  Both match the
    oracle, and the elements around the views stay untouched."""
    prog, nv, ns = PROGS["D"]
    try:
        for n in (3, 4 * 1024 + 1, 3 * 4096 + 11, (1 << 20) + 3):
            vecs = inputs.uniform_vectors(55 + n, n, nv, np.float32)
            salt.salt_tune_set(prog, salt.F32, n, 1, 16, 128, 0, 4096)
            offs = [1, 1, 1, 1] if layout == "same_offset" else [1, 2, 3, 1]
            bufs = [torch.full((n + 8,), 7.0, dtype=torch.float32, device=cuda_dev) for _ in range(nv)]
            tv = []
            for b, v, o in zip(bufs, vecs, offs):
                b[o:o + n] = torch.from_numpy(v).to(cuda_dev)
                tv.append(b[o:o + n])
            salt.salt_eval(prog, tv)
            torch.cuda.synchronize()
            want, _ = run_oracle(prog, vecs, [])
            for k, (b, o) in enumerate(zip(bufs, offs)):
                h = b.cpu().numpy()
                assert_bits_equal(h[o:o + n], want[k], f"{layout} n={n} operand {k}")
                assert np.all(np.delete(h, np.arange(o, o + n)) == 7.0)
    finally:
        salt.salt_tune_clear()


def test_autotune_includes_staged_loop(salt, cuda_dev):
    """The autotuner's pick (register-tiled or staged) is stored, reported
    and bit-exact; a staged pick names a valid stage size."""
    prog, nv, ns = PROGS["E"]
    n = (1 << 22) + 9
    vecs = inputs.uniform_vectors(77, n, nv, np.float32)
    tv = [torch.from_numpy(v.copy()).to(cuda_dev) for v in vecs]
    try:
        cfg, ms = salt.salt_autotune(salt.KERNEL_PROGRAM, prog, tv, [1.5, -0.25], reps=2)
        assert ms > 0 and cfg["stage_bytes"] in (0, 4096, 8192, 16384)
        assert salt.salt_tune_get(prog, salt.F32, n) == cfg
        tv[4].zero_()
        salt.salt_eval(prog, tv, [1.5, -0.25])
        want, _ = run_oracle(prog, vecs, [1.5, -0.25])
        assert_bits_equal(tv[4].cpu().numpy(), want[4], f"E under {cfg}")
    finally:
        salt.salt_tune_clear()
