"""Batched persistent launch (GPU): every item against the oracle, the batch
against the plain per-call path, and an item alone against the same item in
a mix (bit-identical reductions by construction)."""
import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1109_1264_gb300 import inputs
from paper_1109_1264_gb300 import programs as P
import tolerance

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = tolerance.TOL
TDT = {np.float64: torch.float64, np.float32: torch.float32}
SHAPES = [  # (program, vectors, scalars)
    (P.PROG_D, 4, 0), (P.PROG_AXPBY, 2, 2), (P.PROG_E, 5, 2), (P.PROG_CG, 3, 2), (P.PROG_DOT, 2, 0),
    (P.PROG_SUMSQ, 1, 0), (P.PROG_SCALE, 2, 1), (None, 1, 0),  # None: nrm2
]
LENGTHS = [0, 1, 7, 100, 4096 + 5, 70001, (1 << 20) + 3]


def assert_bits_equal(got, want, what=""):
    iu = np.uint32 if got.dtype == np.float32 else np.uint64
    bad = ~((got.view(iu) == want.view(iu)) | (np.isnan(got) & np.isnan(want)))
    assert not bad.any(), f"{what}: {int(bad.sum())} elements differ"


def make_items(seed, dtypes=(np.float64, np.float32), lengths=LENGTHS):
    rng = np.random.default_rng(seed)
    items = []
    k = 0
    for dt in dtypes:
        for prog, nv, ns in SHAPES:
            for n in lengths:
                vecs = [rng.uniform(-1, 1, n).astype(dt) for _ in range(nv)]
                scal = list(rng.uniform(-2, 2, ns))
                items.append((prog, dt, vecs, scal))
                k += 1
    return items


def build(salt, items, dev, spare=0):
    b = salt.Batch(len(items) + spare)
    tensors, slots = [], []
    for prog, dt, vecs, scal in items:
        tv = [torch.from_numpy(v.copy()).to(dev) for v in vecs]
        slots.append(b.add_nrm2(tv[0]) if prog is None else b.add(prog, tv, scal))
        tensors.append(tv)
    return b, tensors, slots


def reference(item):
    """Oracle outputs and exact reductions of one item."""
    prog, dt, vecs, scal = item
    if prog is None:
        return vecs, [exact.exact_nrm2(vecs[0])], [exact.exact_nrm2(vecs[0])]
    outs = [v.copy() for v in vecs]
    oracle.eval_program(prog, outs, scal)
    refs, scales = [], []
    if any(o in ("DOT", "SUMSQ") for o, _ in prog):
        if prog == P.PROG_CG:
            a, c = outs[0], outs[0]
        elif prog == P.PROG_DOT:
            a, c = vecs[0], vecs[1]
        else:
            a, c = vecs[0], vecs[0]
        refs.append(exact.exact_dot(a, c))
        scales.append(exact.abs_dot(a, c))
    return outs, refs, scales


def check(items, tensors, slots, red):
    for item, tv, slot in zip(items, tensors, slots):
        prog, dt, vecs, scal = item
        outs, refs, scales = reference(item)
        for k, (t, w) in enumerate(zip(tv, outs)):
            assert_bits_equal(t.cpu().numpy(), w, f"{prog} n={len(vecs[0])} operand {k}")
        for r, (ref, sc) in enumerate(zip(refs, scales)):
            got = red[slot + r]
            tolerance.check(got, ref, sc, dt, (prog, dt, len(vecs[0])))
            if len(vecs[0]) == 0:
                assert got == 0.0


@pytest.fixture(scope="module")
def salt(saltlib, cuda_dev):
    return saltlib


def test_mixed_batch_matches_oracle(salt, cuda_dev):
    items = make_items(1)
    b, tensors, slots = build(salt, items, cuda_dev)
    nres = b.info()["results"]
    red = torch.full((nres,), float("nan"), dtype=torch.float64, device=cuda_dev)
    b.launch(red)
    torch.cuda.synchronize()
    check(items, tensors, slots, red.cpu().numpy())
    b.close()


@pytest.mark.parametrize("cfg", [(1, 128, 0, 1024), (2, 256, 0, 65536), (4, 256, 2, 16384), (2, 64, 1, 4096),
                                 (4, 128, 0, 1 << 20)])
def test_every_launch_shape(salt, cuda_dev, cfg):
    items = make_items(2, lengths=[0, 5, 999, 33333, (1 << 18) + 9])
    b, tensors, slots = build(salt, items, cuda_dev)
    b.set_config(*cfg)
    red = torch.full((b.info()["results"],), float("nan"), dtype=torch.float64, device=cuda_dev)
    b.launch(red)
    torch.cuda.synchronize()
    check(items, tensors, slots, red.cpu().numpy())
    b.close()


def test_batch_equals_plain_and_alone(salt, cuda_dev):
    """Elementwise outputs of the batch and of the plain per-call path are
    bit-identical; each reduction equals, bit for bit, the same item run
    alone in its own batch (the partition depends only on n and the tile)."""
    items = make_items(3, lengths=[17, 5000, 123457])
    b, tensors, slots = build(salt, items, cuda_dev)
    red = torch.zeros(b.info()["results"], dtype=torch.float64, device=cuda_dev)
    b.launch(red)
    bp, tensors_p, slots_p = build(salt, items, cuda_dev)
    red_p = torch.zeros(bp.info()["results"], dtype=torch.float64, device=cuda_dev)
    bp.launch_plain(red_p)
    torch.cuda.synchronize()
    for tv, tp in zip(tensors, tensors_p):
        for t, u in zip(tv, tp):
            assert_bits_equal(t.cpu().numpy(), u.cpu().numpy(), "batch vs plain")
    check(items, tensors_p, slots_p, red_p.cpu().numpy())
    mix = red.cpu().numpy()
    for i, item in enumerate(items):
        if slots[i] < 0:
            continue
        b1, t1, s1 = build(salt, [item], cuda_dev)
        r1 = torch.zeros(b1.info()["results"], dtype=torch.float64, device=cuda_dev)
        b1.launch(r1)
        torch.cuda.synchronize()
        alone = r1.cpu().numpy()
        nres = len(reference(item)[1])
        assert np.array_equal(alone[s1[0]:s1[0] + nres].view(np.uint64), mix[slots[i]:slots[i] + nres].view(np.uint64))
        b1.close()
    b.close()
    bp.close()


def test_graph_replay_and_rebuild(salt, cuda_dev):
    """Replays of an unchanged batch give identical results; adding items
    rebuilds the table."""
    items = make_items(4, dtypes=(np.float32,), lengths=[3000, 77777])
    items = [it for it in items if it[0] in (P.PROG_DOT, P.PROG_SUMSQ, None, P.PROG_D)]
    b, tensors, slots = build(salt, items, cuda_dev, spare=1)
    red = torch.zeros((2, b.info()["results"]), dtype=torch.float64, device=cuda_dev)
    b.launch(red[0])
    b.launch(red[1])
    r = red.cpu().numpy()
    assert np.array_equal(r[0].view(np.uint64), r[1].view(np.uint64))
    x = torch.ones(1000, dtype=torch.float32, device=cuda_dev)
    s = b.add_nrm2(x)
    red2 = torch.zeros(b.info()["results"], dtype=torch.float64, device=cuda_dev)
    b.launch(red2)
    torch.cuda.synchronize()
    assert red2[s].item() == pytest.approx(1000 ** 0.5, rel=1e-15)
    assert np.array_equal(red2.cpu().numpy()[:len(r[0])].view(np.uint64), r[0].view(np.uint64))
    b.close()


def test_cg_batch_sample_config4(salt, cuda_dev):
    """4096 CG-style updates, lengths log-uniform in [64, 2^20], operands from
    the counter-based generator in three pooled buffers; a sample of items is
    checked against the oracle."""
    nitems = 4096
    lens = inputs.loguniform_lengths(0, nitems, 64, 1 << 20)
    ab = inputs.cg_scalars(0, nitems)
    for dt in (np.float32, np.float64):
        align = 16 // np.dtype(dt).itemsize
        offs = np.zeros(nitems, dtype=np.int64)
        o = 0
        for i, n in enumerate(lens):
            offs[i] = o
            o += -(-int(n) // align) * align
        bufs = [torch.empty(o, dtype=TDT[dt], device=cuda_dev) for _ in range(3)]
        keys = [inputs.vector_key(0, 0, k) for k in range(3)]
        for buf, key in zip(bufs, keys):
            salt.salt_fill_uniform(buf, key)
        b = salt.Batch(nitems)
        slots = []
        for i in range(nitems):
            n = int(lens[i])
            vs = [buf[offs[i]:offs[i] + n] for buf in bufs]
            slots.append(b.add(P.PROG_CG, vs, list(ab[i])))
        red = torch.full((nitems,), float("nan"), dtype=torch.float64, device=cuda_dev)
        b.launch(red)
        torch.cuda.synchronize()
        redh = red.cpu().numpy()
        rng = np.random.default_rng(9)
        for i in sorted(set(rng.integers(0, nitems, 40).tolist()) | {0, nitems - 1}):
            n = int(lens[i])
            r, q, p = (inputs.hash_uniform(key, n, dt, offset=int(offs[i])) for key in keys)
            want = [r.copy(), q.copy(), p.copy()]
            oracle.eval_program(P.PROG_CG, want, list(ab[i]))
            got_r = bufs[0][offs[i]:offs[i] + n].cpu().numpy()
            got_p = bufs[2][offs[i]:offs[i] + n].cpu().numpy()
            assert_bits_equal(got_r, want[0], f"item {i} r")
            assert_bits_equal(got_p, want[2], f"item {i} p")
            ref = exact.exact_sumsq(want[0])
            tolerance.check(redh[slots[i]], ref, ref, dt, ("item", i))
        b.close()
        del bufs
        torch.cuda.empty_cache()


def test_fp32_items_both_access_widths(salt, cuda_dev):
    """FP32 items whose operands are all 32-byte aligned take 32-byte
    accesses, the others 16-byte accesses: in one batch, both give the
    oracle's bits, and their reductions are within tolerance."""
    rng = np.random.default_rng(17)
    items, tensors, slots = [], [], []
    for n in (5, 1000, 4096 + 3, 70001, 300007):
        for off in (0, 4):  # elements: 0 -> 32-byte aligned views, 4 -> 16-byte aligned only
            for prog, nv, ns in ((P.PROG_E, 5, 2), (P.PROG_CG, 3, 2), (P.PROG_DOT, 2, 0)):
                vecs = [rng.uniform(-1, 1, n).astype(np.float32) for _ in range(nv)]
                tv = []
                for v in vecs:
                    buf = torch.zeros(n + 8, dtype=torch.float32, device=cuda_dev)
                    view = buf[off:off + n]
                    view.copy_(torch.from_numpy(v))
                    tv.append(view)
                assert all((t.data_ptr() % 32 == 0) == (off == 0) for t in tv)
                items.append((prog, np.float32, vecs, list(rng.uniform(-2, 2, ns))))
                tensors.append(tv)
    b = salt.Batch(len(items))
    for (prog, dt, vecs, scal), tv in zip(items, tensors):
        slots.append(b.add(prog, tv, scal))
    red = torch.full((max(b.info()["results"], 1),), float("nan"), dtype=torch.float64, device=cuda_dev)
    b.launch(red)
    torch.cuda.synchronize()
    check(items, tensors, slots, red.cpu().numpy())
    b.close()


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
def test_reductions_after_divergent_tails(salt, cuda_dev, dt):
    """Lengths whose last elements are taken by lane 0 alone (a scalar tail
    after the vector loop) or by a partial warp: n in 1..13, 64, 65, 100, 101,
    513, 1025, 4097, for DOT, SUMSQ and the CG update, at every unroll depth,
    in the batch kernel and in the single-expression kernel.  The block sums
    that follow the divergent tails use full-warp shuffles; every reduction
    must be within tolerance of its exact value."""
    import tolerance
    code = salt.F32 if dt == np.float32 else salt.F64
    lengths = list(range(1, 14)) + [64, 65, 100, 101, 513, 1025, 4097]
    progs = [(P.PROG_DOT, 2, 0), (P.PROG_SUMSQ, 1, 0), (P.PROG_CG, 3, 2)]
    rng = np.random.default_rng(61)
    items = []
    for prog, nv, ns in progs:
        for n in lengths:
            items.append((prog, dt, [rng.uniform(-1, 1, n).astype(dt) for _ in range(nv)],
                          list(rng.uniform(-2, 2, ns))))
    for unroll in (1, 2, 4):
        b, tensors, slots = build(salt, items, cuda_dev)
        b.set_config(unroll, 128, 0, 16 * 128 * unroll * 4)
        red = torch.full((len(items),), float("nan"), dtype=torch.float64, device=cuda_dev)
        b.launch(red)
        torch.cuda.synchronize()
        check(items, tensors, slots, red.cpu().numpy())
        b.close()
        for prog, _, vecs, scal in items:
            n = len(vecs[0])
            salt.salt_tune_set(prog, code, n, unroll, 16, 128, 0)
            tv = [torch.from_numpy(v.copy()).to(cuda_dev) for v in vecs]
            r = torch.full((1,), float("nan"), dtype=torch.float64, device=cuda_dev)
            salt.salt_eval(prog, tv, scal, red_out=r)
            torch.cuda.synchronize()
            _, refs, scales = reference((prog, dt, vecs, scal))
            tolerance.check(r.item(), refs[0], scales[0], dt, (prog, n, unroll))
        salt.salt_tune_clear()


def test_batch_vector_width(salt, cuda_dev):
    """The batch's vector width: 32-byte accesses for 32-byte aligned FP32
    items, or 16-byte accesses throughout -- the same bits for every
    elementwise result, both within tolerance of the exact reductions; the
    autotuner reports the width it keeps."""
    items = make_items(71, dtypes=(np.float32,), lengths=[8, 1000, 4096 + 8, 70000, (1 << 20) + 8])
    outs = {}
    for vb in (32, 16):
        b, tensors, slots = build(salt, items, cuda_dev)
        b.set_vec_bytes(vb)
        assert b.get_config()["vec_bytes"] == vb
        red = torch.full((len(items),), float("nan"), dtype=torch.float64, device=cuda_dev)
        b.launch(red)
        torch.cuda.synchronize()
        check(items, tensors, slots, red.cpu().numpy())
        outs[vb] = [[t.cpu().numpy() for t in tv] for tv in tensors]
        if vb == 16:
            b.autotune(red, reps=1)
            assert b.get_config()["vec_bytes"] in (16, 32)
        b.close()
    for a, c in zip(outs[32], outs[16]):
        for x, y in zip(a, c):
            assert_bits_equal(x, y, "vector widths 32 and 16")
    with pytest.raises(salt.SaltError):
        bb = salt.Batch(1)
        try:
            bb.set_vec_bytes(8)
        finally:
            bb.close()
