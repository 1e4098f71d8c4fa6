"""Run-time compiled fused kernels (GPU): programs without a compile-time
instantiation, compiled by NVRTC, must match the oracle bit for bit, be
cached, and beat the interpreter."""
import random

import numpy as np
import pytest

import oracle
from oracle import exact
import oracle_pins
from paper_1109_1264_gb300 import inputs
from test_gpu_parity import assert_bits_equal, check_reductions, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture
def jit(saltlib, cuda_dev):
    prev = saltlib.salt_jit_stats()["mode"]
    saltlib.salt_set_jit(saltlib.JIT_ON)
    yield saltlib
    saltlib.salt_set_jit(prev)


def test_jit_random_programs_match_oracle(jit):
    s = jit
    rng = random.Random(23)
    nrng = np.random.default_rng(23)
    st0 = s.salt_jit_stats()
    before = st0["kernels"] + st0["disk_hits"]  # compiled here, or loaded from the on-disk cache
    ran = 0
    for t in range(24):
        dt = np.float64 if t % 2 == 0 else np.float32
        nvecs, nscal = rng.randint(1, 6), rng.randint(0, 3)
        while True:
            prog = oracle_pins.random_program(rng, nvecs, nscal)
            if len(prog) <= s.MAX_PROG and sum(o in ("DOT", "SUMSQ") for o, _ in prog) <= s.MAX_REDS:
                break
        _, compiled = s.salt_check_program(prog, nvecs, nscal)
        ran += not compiled
        n = rng.choice([1, 17, 1023, 70001, 300007])
        vecs = [nrng.uniform(-1, 1, n).astype(dt) for _ in range(nvecs)]
        scalars = list(nrng.uniform(-2, 2, nscal))
        got, red = run_gpu(s, prog, vecs, scalars, dt)
        want, _ = run_oracle(prog, vecs, scalars)
        for k, (g, w) in enumerate(zip(got, want)):
            assert_bits_equal(g, w, f"jit prog {prog} n={n} operand {k}")
        check_reductions(prog, vecs, scalars, red, dt, f"jit prog {prog}")
    st1 = s.salt_jit_stats()
    assert ran > 10 and st1["kernels"] + st1["disk_hits"] > before


def test_jit_cache_and_speed_over_interpreter(jit, cuda_dev):
    """A 6-operand expression that no compiled shape covers:
    f = (a - b) o (c + d) - 2.5 e, plus sum f^2."""
    s = jit
    prog = [("VEC", 0), ("VEC", 1), ("SUB", 0), ("VEC", 2), ("VEC", 3), ("ADD", 0), ("MUL", 0),
            ("SCAL", 0), ("VEC", 4), ("SMUL", 0), ("SUB", 0), ("STORE", 5), ("VEC", 5), ("SUMSQ", 0)]
    assert s.salt_check_program(prog, 6, 1) == (1, False)
    n = 1 << 25
    x = [torch.empty(n, dtype=torch.float32, device=cuda_dev) for _ in range(6)]
    for k, t in enumerate(x):
        s.salt_fill_uniform(t, 500 + k)
    red = torch.zeros(1, dtype=torch.float64, device=cuda_dev)
    stream = torch.cuda.current_stream()

    def timed():
        s.salt_eval(prog, x, [2.5], red_out=red)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            s.salt_eval(prog, x, [2.5], red_out=red)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 5

    k0 = s.salt_jit_stats()["kernels"]
    t_jit = timed()
    k1 = s.salt_jit_stats()["kernels"]
    assert k1 - k0 <= 1  # compiled at most once, then cached
    out_jit = x[5].clone()
    r_jit = red.item()
    s.salt_set_jit(s.JIT_OFF)
    t_int = timed()
    assert s.salt_jit_stats()["kernels"] == k1
    assert_bits_equal(x[5].cpu().numpy(), out_jit.cpu().numpy(), "jit vs interpreter")
    # the oracle from the host's copy of the counter-based inputs
    want = [inputs.hash_uniform(500 + k, n, np.float32) for k in range(6)]
    oracle.eval_program(prog, want, [2.5])
    assert_bits_equal(out_jit.cpu().numpy(), want[5], "jit vs oracle")
    ref = exact.exact_sumsq(want[5])
    assert abs(r_jit - ref) <= 1e-6 * ref and abs(red.item() - ref) <= 1e-6 * ref
    gbs = lambda ms: 6 * 4 * n / (ms * 1e-3) / 1e9  # algorithmic: 5 reads + 1 write of 4 B
    print(f"jit {t_jit:.3f} ms ({gbs(t_jit):.0f} GB/s), interpreter {t_int:.3f} ms ({gbs(t_int):.0f} GB/s)")
    assert t_jit < t_int


_CHILD = r"""
import hashlib, json, sys
import torch
from paper_1109_1264_gb300 import salt
prog = [("VEC", 0), ("VEC", 1), ("ADD", 0), ("VEC", 1), ("MUL", 0), ("NEG", 0), ("VEC", 0), ("SUB", 0),
        ("STORE", 2)]
x, y, z = (torch.empty(100003, dtype=torch.float64, device="cuda") for _ in range(3))
salt.salt_fill_uniform(x, 1)
salt.salt_fill_uniform(y, 2)
salt.salt_eval(prog, [x, y, z])
torch.cuda.synchronize()
st = salt.salt_jit_stats()
print(json.dumps({"kernels": st["kernels"], "hits": st["disk_hits"], "writes": st["disk_writes"],
                  "dir": st["cache_dir"], "digest": hashlib.sha256(z.cpu().numpy().tobytes()).hexdigest()}))
"""


def test_jit_disk_cache_across_processes(saltlib, cuda_dev, tmp_path):
    """A program compiled in one process is loaded from the on-disk cache by
    the next (no compile) with the same results; a cache file whose payload
    was altered fails its check and is recompiled, never loaded."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SALT_JIT_CACHE=str(tmp_path / "jit"), PYTHONPATH=root)

    def child():
        r = subprocess.run([sys.executable, "-c", _CHILD], env=env, cwd=root, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        return json.loads(r.stdout.strip().splitlines()[-1])

    first = child()
    assert first["dir"] == str(tmp_path / "jit")
    assert (first["kernels"], first["hits"], first["writes"]) == (1, 0, 1)
    files = list((tmp_path / "jit").glob("*.cubin"))
    assert len(files) == 1
    second = child()
    assert (second["kernels"], second["hits"], second["writes"]) == (0, 1, 0)
    assert second["digest"] == first["digest"]
    data = bytearray(files[0].read_bytes())
    data[-100] ^= 0x5A  # inside the cubin payload: the stored hash no longer matches
    files[0].write_bytes(bytes(data))
    third = child()
    assert (third["kernels"], third["hits"], third["writes"]) == (1, 0, 1)
    assert third["digest"] == first["digest"]


def test_debug_mode_checks_each_call(saltlib, cuda_dev):
    """SALT_DEBUG=1 (a child process): calls synchronise and still return
    the same results."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = (
        "import torch\n"
        "from paper_1109_1264_gb300 import salt\n"
        "x = torch.arange(1000, dtype=torch.float64, device='cuda')\n"
        "out = torch.zeros(2, dtype=torch.float64, device='cuda')\n"
        "salt.salt_dot(x, x, out[0:1]); salt.salt_nrm2(x, out[1:2])\n"
        "print(out[0].item(), out[1].item())\n")
    r = subprocess.run([sys.executable, "-c", child], env=dict(os.environ, SALT_DEBUG="1", PYTHONPATH=root),
                       cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    d, nr = (float(v) for v in r.stdout.split())
    import math
    assert d == 999 * 1000 * 1999 // 6 and nr == math.sqrt(d)
