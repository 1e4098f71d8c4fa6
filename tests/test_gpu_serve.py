"""Serving loop (GPU): served results against the oracle, each result the same
alone and in a mix, admission by the device-memory budget, bounded waits,
cancellation, and the trace replayer."""
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
SHAPES = [(P.PROG_D, 4, 3), (P.PROG_AXPBY, 2, 1), (P.PROG_E, 5, 4), (P.PROG_DOT, 2, None), (None, 1, None)]
SC = [1.5, -0.25]


def assert_bits_equal(got, want, what=""):
    iu = np.uint32 if got.dtype == np.float32 else np.uint64
    bad = ~((got.view(iu) == want.view(iu)) | (np.isnan(got) & np.isnan(want)))
    assert not bad.any(), f"{what}: {int(bad.sum())} elements differ"


@pytest.fixture(scope="module")
def salt(saltlib, cuda_dev):
    return saltlib


def host_inputs(keys, nv, n, dt):
    return [inputs.hash_uniform(k, n, dt) for k in keys[:nv]]


def expected(shape_i, keys, n, dt):
    prog, nv, out = SHAPES[shape_i]
    vecs = host_inputs(keys, nv, n, dt)
    if prog is None:
        return vecs, None, exact.exact_nrm2(vecs[0]), exact.exact_nrm2(vecs[0])
    if prog == P.PROG_D:
        vecs[3] = np.zeros(n, dt)
    if prog == P.PROG_E:
        vecs[4] = np.zeros(n, dt)
    want = [v.copy() for v in vecs]
    oracle.eval_program(prog, want, SC[:2])
    if prog == P.PROG_DOT:
        return want, None, exact.exact_dot(vecs[0], vecs[1]), exact.abs_dot(vecs[0], vecs[1])
    return want, out, None, None


@pytest.mark.parametrize("persistent", [0, 1])
def test_served_results_match_oracle(salt, persistent):
    srv = salt.Server(budget_bytes=1 << 28, max_n=1 << 20, persistent=persistent)
    try:
        reqs = []
        for dt, code in ((np.float64, salt.F64), (np.float32, salt.F32)):
            for si, (prog, nv, _) in enumerate(SHAPES):
                for n in (0, 1, 7, 300, 65536 + 3, (1 << 20)):
                    keys = [inputs.vector_key(77, len(reqs), k) for k in range(nv)]
                    rid = srv.submit(prog, code, n, keys, SC if prog is not None else ())
                    reqs.append((rid, si, dt, n, keys))
        for rid, si, dt, n, keys in reqs:
            srv.wait(rid, 20_000_000)
            state, lat, red = srv.poll(rid)
            assert state == 2 and lat > 0
            want, out, ref, scale = expected(si, keys, n, dt)
            if out is not None:
                got = srv.read(rid, out, np.empty(n, dt))
                assert_bits_equal(got, want[out], f"shape {si} n={n}")
            if ref is not None:
                tolerance.check(red[0], ref, scale, dt, (si, dt, n))
            srv.release(rid)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["resident_bytes"] == 0 and st["waiting"] == 0
    finally:
        srv.stop()


@pytest.mark.parametrize("persistent", [0, 1])
def test_alone_vs_mix_bit_identical(salt, persistent):
    """>= 200 requests, each run alone (one request per step) and then all
    submitted at once (steps of many requests on two streams)."""
    srv = salt.Server(budget_bytes=1 << 30, max_n=1 << 16, persistent=persistent)
    try:
        shapes, is64, lens = inputs.request_mix(5, 240, lo=2 ** 8, hi=2 ** 16)
        def submit_all():
            ids = []
            for i in range(len(lens)):
                prog, nv, _ = SHAPES[int(shapes[i])]
                keys = [inputs.vector_key(5, i, k) for k in range(nv)]
                ids.append(srv.submit(prog, salt.F64 if is64[i] else salt.F32, int(lens[i]), keys,
                                      SC if prog is not None else ()))
            return ids

        def collect(ids):
            res = []
            for i, rid in enumerate(ids):
                srv.wait(rid, 20_000_000)
                _, _, red = srv.poll(rid)
                prog, nv, out = SHAPES[int(shapes[i])]
                dt = np.float64 if is64[i] else np.float32
                vec = srv.read(rid, out, np.empty(int(lens[i]), dt)) if out is not None else None
                res.append((red[0], vec))
                srv.release(rid)
            return res

        alone = []
        for i in range(len(lens)):  # one at a time: each request is alone in its step
            prog, nv, _ = SHAPES[int(shapes[i])]
            keys = [inputs.vector_key(5, i, k) for k in range(nv)]
            rid = srv.submit(prog, salt.F64 if is64[i] else salt.F32, int(lens[i]), keys,
                             SC if prog is not None else ())
            alone += collect_one(srv, rid, shapes[i], is64[i], lens[i])
        before = srv.stats()["steps"]
        mix = collect(submit_all())
        steps = srv.stats()["steps"] - before
        # Python submits one request every few tens of microseconds while
        # small steps finish quickly, so steps carry a few requests each (a
        # persistent step can end before the next submission: no bound there;
        # the replay tests load it enough to batch).
        if not persistent:
            assert steps < 0.6 * len(lens), f"the mix ran in {steps} steps: requests were not batched"
        for i, ((ra, va), (rm, vm)) in enumerate(zip(alone, mix)):
            if SHAPES[int(shapes[i])][0] in (P.PROG_DOT, None):
                assert np.float64(ra).view(np.uint64) == np.float64(rm).view(np.uint64), i
            if va is not None:
                assert_bits_equal(vm, va, f"request {i}")
    finally:
        srv.stop()


def collect_one(srv, rid, shape, is64, n):
    srv.wait(rid, 20_000_000)
    _, _, red = srv.poll(rid)
    prog, nv, out = SHAPES[int(shape)]
    dt = np.float64 if is64 else np.float32
    vec = srv.read(rid, out, np.empty(int(n), dt)) if out is not None else None
    srv.release(rid)
    return [(red[0], vec)]


@pytest.mark.parametrize("persistent", [0, 1])
def test_budget_admission_timeout_and_cancel(salt, persistent):
    srv = salt.Server(budget_bytes=4 << 20, max_n=1 << 20, persistent=persistent)
    try:
        n = 300_000  # 2 FP32 operands = 2.4 MB: two such requests do not fit in 4 MiB
        keys = [1, 2]
        a = srv.submit(P.PROG_DOT, salt.F32, n, keys)
        srv.wait(a, 20_000_000)
        b = srv.submit(P.PROG_DOT, salt.F32, n, keys)
        c = srv.submit(P.PROG_DOT, salt.F32, 10, keys)  # small, but queued behind b (arrival order)
        with pytest.raises(salt.SaltError) as ei:
            srv.wait(b, 50_000)
        assert ei.value.status == salt.ERR_TIMEOUT
        assert srv.poll(b)[0] == 0 and srv.poll(c)[0] == 0
        srv.release(c)  # cancel a waiting request
        with pytest.raises(salt.SaltError) as ei:
            srv.poll(c)
        assert ei.value.status == salt.ERR_NOTFOUND
        srv.release(a)  # frees the budget: b is admitted and runs
        srv.wait(b, 20_000_000)
        assert srv.poll(b)[2][0] == srv.poll(b)[2][0]
        srv.release(b)
        with pytest.raises(salt.SaltError) as ei:
            srv.submit(P.PROG_DOT, salt.F64, 1 << 20, keys)  # 16 MiB > whole budget
        assert ei.value.status == salt.ERR_BUDGET
    finally:
        srv.stop()


@pytest.mark.parametrize("persistent", [0, 1])
def test_replay_poisson_trace(salt, persistent):
    srv = salt.Server(budget_bytes=1 << 30, max_n=1 << 18, persistent=persistent)
    try:
        count = 400
        shapes, is64, lens = inputs.request_mix(9, count, lo=2 ** 8, hi=2 ** 18)
        arr = inputs.poisson_arrivals(9, count, 20_000.0) * 1e6  # 20k requests/s, in µs
        lat, red, wall = srv.replay(arr, shapes, is64.astype(np.int32), lens, seed=9)
        assert np.all(lat > 0) and wall > 0
        for i in list(range(0, count, 37)):
            si = int(shapes[i])
            if SHAPES[si][0] in (P.PROG_DOT, None):
                dt = np.float64 if is64[i] else np.float32
                keys = [inputs.vector_key(9, i, k) for k in range(SHAPES[si][1])]
                _, _, ref, scale = expected(si, keys, int(lens[i]), dt)
                tolerance.check(red[i], ref, scale, dt, ("request", i))
        assert srv.stats()["resident_bytes"] == 0
    finally:
        srv.stop()


M64 = (1 << 64) - 1


def store_place(seed, i, k, n, length, count, itemsize):
    """Store vector and offset of input operand k of replayed request i
    (the formula salt_serve_replay_store documents)."""
    key = (seed * 0x100000001B3 + i * 16 + k + 1) & M64
    h = ((key * 0x9E3779B97F4A7C15) & M64) >> 11
    o = h % (length - n + 1)
    return (i * 5 + k) % count, o - o % (32 // itemsize)


@pytest.mark.parametrize("persistent", [0, 1])
def test_caller_owned_operands(salt, cuda_dev, persistent):
    """Inputs in caller-owned device memory (no fill), the output server-owned
    or caller-owned: the same bits as the oracle."""
    srv = salt.Server(budget_bytes=1 << 28, max_n=1 << 20, persistent=persistent)
    try:
        for dt, code, tdt in ((np.float32, salt.F32, torch.float32), (np.float64, salt.F64, torch.float64)):
            for n in (1, 1000, (1 << 20) - 3):
                keys = [inputs.vector_key(31, n, k) for k in range(5)]
                host = [inputs.hash_uniform(k, n, dt) for k in keys]
                dev = [torch.from_numpy(h).to(cuda_dev) for h in host]
                out_dev = torch.zeros(n, dtype=tdt, device=cuda_dev)
                want = [h.copy() for h in host[:4]] + [np.zeros(n, dt)]
                oracle.eval_program(P.PROG_E, want, SC)
                # caller-owned operands are ready when submitted: the server does
                # not order its work after the caller's streams
                torch.cuda.current_stream().synchronize()
                # inputs caller-owned, output server-owned
                a = srv.submit(P.PROG_E, code, n, keys, SC, ptrs=dev[:4] + [None])
                # everything caller-owned (keys unused)
                b = srv.submit(P.PROG_E, code, n, keys, SC, ptrs=dev[:4] + [out_dev])
                # dot with caller-owned inputs
                c = srv.submit(P.PROG_DOT, code, n, keys[:2], ptrs=dev[:2])
                for rid in (a, b, c):
                    srv.wait(rid, 20_000_000)
                assert_bits_equal(srv.read(a, 4, np.empty(n, dt)), want[4], f"server-owned out n={n}")
                assert_bits_equal(out_dev.cpu().numpy(), want[4], f"caller-owned out n={n}")
                assert_bits_equal(srv.read(b, 0, np.empty(n, dt)), host[0], "read of a caller-owned operand")
                red = srv.poll(c)[2][0]
                tolerance.check_dot(red, host[0], host[1], dt, ("caller-owned dot", n))
                for rid in (a, b, c):
                    srv.release(rid)
        assert srv.stats()["resident_bytes"] == 0
        with pytest.raises(salt.SaltError) as ei:
            x = torch.zeros(64, dtype=torch.float32, device=cuda_dev)
            srv.submit(P.PROG_DOT, salt.F32, 10, [1, 2], ptrs=[x[1:], x])  # 4-byte offset
        assert ei.value.status == salt.ERR_ALIGN
    finally:
        srv.stop()


@pytest.mark.parametrize("persistent", [0, 1])
def test_replay_resident_store(salt, cuda_dev, persistent):
    """The load generator reading inputs from a resident store: dot and norm
    results against the exact values of the store slices they read."""
    srv = salt.Server(budget_bytes=1 << 30, max_n=1 << 18, persistent=persistent)
    try:
        length = (1 << 20) + 8
        skeys = {np.float32: [901, 902, 903], np.float64: [911, 912]}
        store = {dt: [torch.empty(length, dtype=torch.float32 if dt == np.float32 else torch.float64,
                                  device=cuda_dev) for _ in skeys[dt]] for dt in skeys}
        for dt in skeys:
            for t, k in zip(store[dt], skeys[dt]):
                salt.salt_fill_uniform(t, k)
        torch.cuda.current_stream().synchronize()  # the server does not order its work after other streams
        count = 400
        shapes, is64, lens = inputs.request_mix(13, count, lo=2 ** 8, hi=2 ** 18)
        arr = inputs.poisson_arrivals(13, count, 20_000.0) * 1e6
        lat, red, wall = srv.replay(arr, shapes, is64.astype(np.int32), lens, seed=13,
                                    store=(store[np.float32], store[np.float64]))
        assert np.all(lat > 0) and wall > 0
        checked = 0
        for i in range(count):
            si = int(shapes[i])
            if SHAPES[si][0] not in (P.PROG_DOT, None):
                continue
            dt = np.float64 if is64[i] else np.float32
            n = int(lens[i])
            vecs = []
            for k in range(SHAPES[si][1]):
                j, o = store_place(13, i, k, n, length, len(skeys[dt]), np.dtype(dt).itemsize)
                vecs.append(inputs.hash_uniform(skeys[dt][j], n, dt, offset=o))
            if si == 4:
                ref, scale = exact.exact_nrm2(vecs[0]), exact.exact_nrm2(vecs[0])
            else:
                ref, scale = exact.exact_dot(vecs[0], vecs[1]), exact.abs_dot(vecs[0], vecs[1])
            tolerance.check(red[i], ref, scale, dt, ("request", i))
            checked += 1
        assert checked > 100
        assert srv.stats()["resident_bytes"] == 0
    finally:
        srv.stop()


def test_server_rejects_programs_outside_the_batch_kernel(salt):
    """The server runs the batch kernel's compiled shapes only: elementwise
    DIV, device scalars and the CG pass shapes are refused at submission."""
    srv = salt.Server(budget_bytes=1 << 24, max_n=1 << 16)
    try:
        div = [("VEC", 0), ("VEC", 1), ("DIV", 0), ("STORE", 2)]
        ds = [("DSCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)]
        cgxr = [("VEC", 3), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 3),
                ("VEC", 4), ("SCAL", 0), ("VEC", 2), ("SMUL", 0), ("SUB", 0), ("STORE", 4),
                ("VEC", 4), ("SUMSQ", 0)]
        for prog, nk, sc in ((div, 3, ()), (ds, 2, ()), (cgxr, 5, (0.5,))):
            with pytest.raises(salt.SaltError) as ei:
                srv.submit(prog, salt.F32, 100, list(range(1, nk + 1)), sc)
            assert ei.value.status == salt.ERR_PROGRAM, prog
        assert srv.stats()["waiting"] == 0
    finally:
        srv.stop()


def test_server_folds_by_value_scalar_subexpressions(salt):
    """A request whose scalars form a subexpression of by-value scalars runs
    on the compiled shape with the folded value: the oracle's bits."""
    srv = salt.Server(budget_bytes=1 << 26, max_n=1 << 16)
    try:
        prog = [("SCAL", 0), ("SCAL", 1), ("DIV", 0), ("VEC", 0), ("SMUL", 0), ("SCAL", 2), ("VEC", 1),
                ("SMUL", 0), ("ADD", 0), ("STORE", 1)]
        for dt, code in ((np.float32, salt.F32), (np.float64, salt.F64)):
            n = 4099
            keys = [inputs.vector_key(41, code, k) for k in range(2)]
            rid = srv.submit(prog, code, n, keys, [1.0, 3.0, -0.5])
            srv.wait(rid, 20_000_000)
            got = srv.read(rid, 1, np.empty(n, dt))
            want = host_inputs(keys, 2, n, dt)
            oracle.eval_program(prog, want, [1.0, 3.0, -0.5])
            assert_bits_equal(got, want[1], f"folded {dt}")
            srv.release(rid)
    finally:
        srv.stop()


def test_persistent_same_bits_as_default(salt):
    """The same requests (every served shape, both dtypes, empty, tiny and
    multi-tile lengths), all submitted at once, through the default mode and
    through persistent mode with 2 and 4 ring entries: the same bits."""
    reqs = [(si, dt, n) for si in range(len(SHAPES)) for dt in (np.float32, np.float64)
            for n in (0, 1, 7, 4099, (1 << 18) + 5)]
    results = []
    for persistent, streams in ((0, 2), (1, 2), (1, 4)):
        srv = salt.Server(budget_bytes=1 << 28, max_n=1 << 20, persistent=persistent, streams=streams)
        try:
            ids = []
            for i, (si, dt, n) in enumerate(reqs):
                prog, nv, _ = SHAPES[si]
                keys = [inputs.vector_key(61, i, k) for k in range(nv)]
                ids.append(srv.submit(prog, salt.F32 if dt == np.float32 else salt.F64, n, keys,
                                      SC if prog is not None else ()))
            res = []
            for (si, dt, n), rid in zip(reqs, ids):
                srv.wait(rid, 20_000_000)
                red = np.array(srv.poll(rid)[2][:1])
                out = SHAPES[si][2]
                res.append((red, srv.read(rid, out, np.empty(n, dt)) if out is not None else None))
                srv.release(rid)
            results.append(res)
        finally:
            srv.stop()
    for other in results[1:]:
        for req, (ra, va), (rb, vb) in zip(reqs, results[0], other):
            assert ra.view(np.uint64)[0] == rb.view(np.uint64)[0], req
            if va is not None:
                assert_bits_equal(vb, va, str(req))


def test_persistent_idle_end_and_relaunch(salt):
    """Persistent mode: the resident launch ends after idle_us with nothing
    posted, and the next request launches it again (from the first step not
    complete); results stay within tolerance of the exact value."""
    import time
    srv = salt.Server(budget_bytes=1 << 26, max_n=1 << 16, persistent=1, idle_us=2000)
    try:
        for rnd in range(3):
            n = 1000 + rnd
            keys = [inputs.vector_key(41, rnd, k) for k in range(2)]
            rid = srv.submit(P.PROG_DOT, salt.F64, n, keys)
            srv.wait(rid, 10_000_000)
            x, y = host_inputs(keys, 2, n, np.float64)
            tolerance.check_dot(srv.poll(rid)[2][0], x, y, np.float64, ("persistent dot", rnd))
            srv.release(rid)
            time.sleep(0.05)  # 50 ms, far beyond the 2 ms idle time: the launch has ended
            launches, live = srv.launches()
            assert launches == rnd + 1 and not live, (rnd, launches, live)
        assert srv.stats()["steps"] == 3
    finally:
        srv.stop()


def test_persistent_wait_runs_out(salt, cuda_dev):
    """A wait of the persistent kernel that runs out (poll limit 0: the other
    blocks stop waiting for block 0's release of the step at once) ends the
    launch and fails the server with an error; no fault, and the device keeps
    working."""
    prev = salt.salt_get_wait_limit(salt.WAIT_SERVE)
    salt.salt_set_wait_limit(salt.WAIT_SERVE, 0)
    try:
        srv = salt.Server(budget_bytes=1 << 26, max_n=1 << 20, persistent=1)
        try:
            rid = srv.submit(P.PROG_DOT, salt.F32, 1 << 20, [1, 2])
            with pytest.raises(salt.SaltError) as ei:
                srv.wait(rid, 10_000_000)
            assert ei.value.status == salt.ERR_CUDA and "bounded wait ran out" in ei.value.message
        finally:
            srv.stop()
    finally:
        salt.salt_set_wait_limit(salt.WAIT_SERVE, prev)
    x = torch.arange(1000, dtype=torch.float64, device=cuda_dev)
    out = torch.zeros(1, dtype=torch.float64, device=cuda_dev)
    salt.salt_dot(x, x, out)
    assert out.item() == 999 * 1000 * 1999 // 6
