"""The C ABI without a GPU: exported symbols, program validation, argument
errors (all detected on the host before any launch), tuning table, and a
loud failure instead of any CPU fallback when no device exists."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "salt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(salt_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(saltlib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(saltlib.lib, name), name
    assert sorted(saltlib.EXPORTS) == names


def test_version_and_status_strings(saltlib):
    assert saltlib.salt_version() >= 10000
    assert saltlib.salt_status_str(saltlib.ERR_ALIAS) == "SALT_ERR_ALIAS"
    assert saltlib.salt_status_str(99) == "unknown status"


D = [("VEC", 0), ("VEC", 1), ("VEC", 2), ("SUB", 0), ("ADD", 0), ("STORE", 3)]
CG = [("VEC", 0), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("SUB", 0), ("STORE", 0), ("VEC", 0), ("SUMSQ", 0),
      ("VEC", 0), ("SCAL", 1), ("VEC", 2), ("SMUL", 0), ("ADD", 0), ("STORE", 2)]


def test_check_program_valid(saltlib):
    assert saltlib.salt_check_program(D, 4, 0) == (0, True)
    # same tree with operands renumbered is still the compiled shape
    D2 = [("VEC", 3), ("VEC", 0), ("VEC", 1), ("SUB", 0), ("ADD", 0), ("STORE", 2)]
    assert saltlib.salt_check_program(D2, 4, 0) == (0, True)
    assert saltlib.salt_check_program(CG, 3, 2) == (1, True)
    assert saltlib.salt_check_program([("VEC", 0), ("VEC", 1), ("DOT", 0)], 2, 0) == (1, True)
    # not instantiated: runs on the interpreter
    odd = [("VEC", 0), ("NEG", 0), ("VEC", 1), ("MUL", 0), ("STORE", 1), ("VEC", 1), ("VEC", 0), ("DOT", 0)]
    assert saltlib.salt_check_program(odd, 2, 0) == (1, False)


@pytest.mark.parametrize("prog,nv,ns,status", [
    ([], 1, 0, 1),
    ([("VEC", 0)] * 33, 1, 0, 1),
    ([("ADD", 0)], 1, 0, 2),
    ([("VEC", 0), ("SCAL", 0), ("SMUL", 0), ("STORE", 0)], 1, 1, 2),
    ([("VEC", 0), ("VEC", 0)], 1, 0, 2),
    ([("VEC", 1), ("STORE", 0)], 1, 0, 2),
    ([("SCAL", 0), ("STORE", 0)], 1, 1, 2),
    ([("VEC", 0), ("STORE", 0), ("VEC", 0), ("NEG", 0)], 1, 0, 2),
    ([("VEC", 0)] * 9 + [("ADD", 0)] * 8 + [("STORE", 0)], 1, 0, 2),
    ([("VEC", 0), ("SUMSQ", 0)] * 5, 1, 0, 2),
    ([(12, 0)], 1, 0, 2),
    ([("VEC", 0), ("NEG", 0)], 1, 0, 2),
    ([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 0)], 9, 0, 1),
])
def test_check_program_rejects(saltlib, prog, nv, ns, status):
    with pytest.raises(saltlib.SaltError) as ei:
        saltlib.salt_check_program(prog, nv, ns)
    assert ei.value.status == status, ei.value


def _raw_eval(saltlib, prog, dtype, n, ptrs, scalars=(), red=None):
    arr, m = saltlib.program(prog)
    p = (ctypes.c_void_p * max(len(ptrs), 1))(*ptrs)
    sc = (ctypes.c_double * max(len(scalars), 1))(*scalars)
    return saltlib.lib.salt_eval(arr, m, dtype, n, p, len(ptrs), sc, len(scalars), red, None)


BASE = 0x7F0000000000  # fake device addresses: never dereferenced, the host rejects first


def test_eval_argument_errors(saltlib):
    ok = [BASE, BASE + 2 ** 20, BASE + 2 ** 21, BASE + 2 ** 22]
    assert _raw_eval(saltlib, D, 2, 10, ok) == saltlib.ERR_DTYPE
    assert _raw_eval(saltlib, D, 0, -1, ok) == saltlib.ERR_ARG
    assert _raw_eval(saltlib, D, 0, 10, [ok[0], ok[1] + 2, ok[2], ok[3]]) == saltlib.ERR_ALIGN
    assert _raw_eval(saltlib, D, 1, 10, [ok[0], ok[1] + 4, ok[2], ok[3]]) == saltlib.ERR_ALIGN
    assert _raw_eval(saltlib, D, 0, 10, [ok[0], None, ok[2], ok[3]]) == saltlib.ERR_ARG
    # output overlapping an input through a different operand index
    assert _raw_eval(saltlib, D, 1, 100, [ok[0], ok[1], ok[2], ok[0] + 16]) == saltlib.ERR_ALIAS
    assert "overlap" in saltlib.salt_last_error()
    # identical pointers for two read-only operands are fine (fails later, on the missing GPU)
    assert _raw_eval(saltlib, D, 1, 100, [ok[0], ok[0], ok[0], ok[3]]) == saltlib.ERR_CUDA
    # reduction without a result buffer
    assert _raw_eval(saltlib, [("VEC", 0), ("SUMSQ", 0)], 0, 10, ok[:1], red=None) == saltlib.ERR_ARG
    assert _raw_eval(saltlib, [("VEC", 0), ("SUMSQ", 0)], 0, 10, ok[:1], red=BASE + 4) == saltlib.ERR_ALIGN
    # scalars referenced but not given
    arr, m = saltlib.program([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 0)])
    p = (ctypes.c_void_p * 1)(BASE)
    assert saltlib.lib.salt_eval(arr, m, 0, 10, p, 1, None, 1, None, None) == saltlib.ERR_ARG


def test_no_cpu_fallback_without_gpu(saltlib):
    """A valid call on a machine without a GPU fails loudly (SALT_ERR_CUDA);
    nothing is computed on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ok = [BASE, BASE + 2 ** 20, BASE + 2 ** 21, BASE + 2 ** 22]
    assert _raw_eval(saltlib, D, 1, 10, ok) == saltlib.ERR_CUDA
    assert saltlib.lib.salt_dot(0, 10, BASE, BASE, BASE, 0, None) == saltlib.ERR_CUDA
    assert saltlib.lib.salt_nrm2(1, 10, BASE, BASE, 0, None) == saltlib.ERR_CUDA


def test_dot_nrm2_argument_errors(saltlib):
    L = saltlib.lib
    assert L.salt_dot(0, 10, BASE, BASE, BASE, 7, None) == saltlib.ERR_ARG
    assert L.salt_dot(3, 10, BASE, BASE, BASE, 0, None) == saltlib.ERR_DTYPE
    assert L.salt_dot(0, 10, BASE + 2, BASE, BASE, 0, None) == saltlib.ERR_ALIGN
    assert L.salt_dot(0, 10, BASE + 4, BASE, BASE, 1, None) == saltlib.ERR_ALIGN  # plain mode needs 16 B
    assert L.salt_dot(0, 10, BASE, BASE, None, 0, None) == saltlib.ERR_ARG
    assert L.salt_nrm2(1, -3, BASE, BASE, 0, None) == saltlib.ERR_ARG
    assert L.salt_nrm2(1, 10, BASE + 4, BASE, 0, None) == saltlib.ERR_ALIGN
    assert L.salt_axpby(0, 10, 1.0, BASE, 1.0, BASE + 16, None) == saltlib.ERR_ALIAS
    assert L.salt_fill_uniform(0, -1, 1, 0, BASE, None) == saltlib.ERR_ARG


def test_tune_table(saltlib):
    saltlib.salt_tune_clear()
    default = saltlib.salt_tune_get(D, saltlib.F32, 1 << 20)
    assert default["block"] == 256
    saltlib.salt_tune_set(D, saltlib.F32, 1 << 20, 4, 32, 128, 8)
    assert saltlib.salt_tune_get(D, saltlib.F32, (1 << 21) - 1) == {"unroll": 4, "vec_bytes": 32, "block": 128,
                                                                    "blocks_per_sm": 8, "stage_bytes": 0}
    assert saltlib.salt_tune_get(D, saltlib.F32, 1 << 21) == default  # other bucket
    assert saltlib.salt_tune_get(D, saltlib.F64, 1 << 20) == default  # other dtype
    saltlib.salt_tune_set(D, saltlib.F32, 1 << 22, 2, 32, 256, 0)  # 0: as many blocks as fit
    assert saltlib.salt_tune_get(D, saltlib.F32, 1 << 22)["blocks_per_sm"] == 0
    for bad in ((3, 16, 128, 4), (2, 8, 128, 4), (2, 16, 100, 4), (2, 16, 512, 4), (2, 16, 256, 9),
                (2, 16, 256, -1), (1, 16, 128, 0, 2048), (1, 16, 128, 0, 6000), (1, 16, 128, 0, 32768),
                (1, 16, 128, 0, -4096)):
        with pytest.raises(saltlib.SaltError):
            saltlib.salt_tune_set(D, saltlib.F32, 1 << 20, *bad)
    saltlib.salt_tune_clear()
    assert saltlib.salt_tune_get(D, saltlib.F32, 1 << 20) == default


def test_tune_table_staged_loop(saltlib):
    """The staged loop (stage_bytes 4096 / 8192 / 16384) is pinned like any
    configuration, for compiled shapes only."""
    s = saltlib
    s.salt_tune_clear()
    try:
        for sb in (4096, 8192, 16384):
            s.salt_tune_set(D, s.F64, 1 << 26, 1, 16, 128, 0, sb)
            assert s.salt_tune_get(D, s.F64, 1 << 26) == {"unroll": 1, "vec_bytes": 16, "block": 128,
                                                          "blocks_per_sm": 0, "stage_bytes": sb}
        # a program that runs on the interpreter has no staged form
        interp = [("VEC", 0), ("VEC", 1), ("MUL", 0), ("VEC", 2), ("MUL", 0), ("VEC", 0), ("ADD", 0),
                  ("STORE", 3)]
        with pytest.raises(s.SaltError) as ei:
            s.salt_tune_set(interp, s.F32, 1 << 20, 1, 16, 128, 0, 4096)
        assert ei.value.status == s.ERR_ARG
        s.salt_tune_set(interp, s.F32, 1 << 20, 1, 16, 128, 0, 0)
    finally:
        s.salt_tune_clear()


def test_tune_save_load_roundtrip(saltlib, tmp_path):
    s = saltlib
    s.salt_tune_clear()
    s.salt_tune_set(D, s.F64, 1 << 24, 4, 32, 128, 2)
    s.salt_tune_set(CG, s.F32, 1000, 1, 16, 64, 8)
    s.salt_tune_set(D, s.F32, 1 << 26, 1, 16, 256, 0, 16384)
    path = str(tmp_path / "tune.txt")
    s.salt_tune_save(path)
    s.salt_tune_clear()
    assert s.salt_tune_get(D, s.F64, 1 << 24)["block"] == 256
    s.salt_tune_load(path)
    assert s.salt_tune_get(D, s.F64, 1 << 24) == {"unroll": 4, "vec_bytes": 32, "block": 128, "blocks_per_sm": 2,
                                                  "stage_bytes": 0}
    assert s.salt_tune_get(CG, s.F32, 1000) == {"unroll": 1, "vec_bytes": 16, "block": 64, "blocks_per_sm": 8,
                                                "stage_bytes": 0}
    assert s.salt_tune_get(D, s.F32, 1 << 26)["stage_bytes"] == 16384
    # a table written without the stage_bytes column still loads (register-tiled loop)
    s.salt_tune_clear()
    old = tmp_path / "old.txt"
    old.write_text("# family dtype bucket unroll vec_bytes block blocks_per_sm\n0 1 24 4 32 128 2\n")
    s.salt_tune_load(str(old))
    assert s.salt_tune_get(D, s.F64, 1 << 24) == {"unroll": 4, "vec_bytes": 32, "block": 128, "blocks_per_sm": 2,
                                                  "stage_bytes": 0}
    for text in ("0 0 20 3 16 128 2\n", "0 0 20 1 16 128 0 1000\n", "200 0 20 1 16 128 0 4096\n",
                 "101 1 20 1 16 128 0 8192\n"):
        bad = tmp_path / "bad.txt"
        bad.write_text(text)
        with pytest.raises(s.SaltError):
            s.salt_tune_load(str(bad))
    with pytest.raises(s.SaltError):
        s.salt_tune_load(str(tmp_path / "missing.txt"))
    s.salt_tune_clear()


def test_autotune_argument_errors(saltlib):
    import ctypes
    s = saltlib
    p = (ctypes.c_void_p * 1)(BASE)
    assert s.lib.salt_autotune(9, None, 0, 0, 100, p, 1, None, 0, BASE, 3, None, None, None) == s.ERR_ARG
    assert s.lib.salt_autotune(s.KERNEL_NRM2_PLAIN, None, 0, 1, 100, p, 1, None, 0, BASE, 3, None, None,
                               None) == s.ERR_DTYPE
    assert s.lib.salt_autotune(s.KERNEL_NRM2, None, 0, 0, 100, p, 1, None, 0, BASE, 0, None, None, None) == s.ERR_ARG


def test_jit_mode_switch(saltlib):
    s = saltlib
    assert s.salt_jit_stats()["mode"] == s.JIT_AUTO  # the default
    with pytest.raises(s.SaltError):
        s.salt_set_jit(5)
    for m in (s.JIT_ON, s.JIT_OFF, s.JIT_AUTO):
        s.salt_set_jit(m)
        assert s.salt_jit_stats()["mode"] == m


def test_jit_cache_dir_setting(saltlib, tmp_path):
    s = saltlib
    before = s.salt_jit_stats()["cache_dir"]
    try:
        s.salt_jit_cache_dir(tmp_path / "k")
        assert s.salt_jit_stats()["cache_dir"] == str(tmp_path / "k")
        s.salt_jit_cache_dir(None)
        assert s.salt_jit_stats()["cache_dir"] == ""
    finally:
        s.salt_jit_cache_dir(before or None)


def test_strided_argument_errors(saltlib):
    s = saltlib
    arr, m = s.program(D)
    p = (ctypes.c_void_p * 4)(BASE, BASE + 2 ** 20, BASE + 2 ** 21, BASE + 2 ** 22)
    sc = (ctypes.c_double * 1)(0.0)
    bad = (ctypes.c_int64 * 4)(1, 0, 1, 1)
    assert s.lib.salt_eval_strided(arr, m, 0, 10, p, bad, 4, sc, 0, None, None) == s.ERR_ARG
    assert s.lib.salt_eval_strided(arr, m, 0, 10, p, None, 4, sc, 0, None, None) == s.ERR_ARG
    # a strided output spanning another operand's memory
    st = (ctypes.c_int64 * 4)(1, 1, 1, 100000)
    q = (ctypes.c_void_p * 4)(BASE, BASE + 2 ** 20, BASE + 2 ** 21, BASE + 2 ** 20 - 4096)
    assert s.lib.salt_eval_strided(arr, m, 0, 10, q, st, 4, sc, 0, None, None) == s.ERR_ALIAS
    # a negative stride spans downwards from the pointer (element n-1 lowest):
    # output d walks back from 4 KiB above b's start over b's memory
    neg = (ctypes.c_int64 * 4)(1, 1, 1, -2)
    r = (ctypes.c_void_p * 4)(BASE, BASE + 2 ** 20, BASE + 2 ** 21, BASE + 2 ** 20 + 40)
    assert s.lib.salt_eval_strided(arr, m, 0, 10, r, neg, 4, sc, 0, None, None) == s.ERR_ALIAS
    # the same walk starting below b overlaps nothing: validation passes (then,
    # with no GPU, the call fails at the device)
    r2 = (ctypes.c_void_p * 4)(BASE, BASE + 2 ** 20, BASE + 2 ** 21, BASE + 2 ** 20 - 4)
    assert s.lib.salt_eval_strided(arr, m, 0, 10, r2, neg, 4, sc, 0, None, None) not in (s.ERR_ALIAS, s.ERR_ARG)


def test_program_marshalling_cache_sees_edits(saltlib):
    """A program list passed again reuses its marshalled form; a list edited
    in place is marshalled afresh (the cache compares it with its copy)."""
    s = saltlib
    prog = [("VEC", 0), ("VEC", 1), ("ADD", 0), ("STORE", 2)]
    a1, m1 = s.program(prog)
    a2, m2 = s.program(prog)
    assert a1 is a2 and m1 == m2 == 4
    prog[2] = ("SUB", 0)
    a3, m3 = s.program(prog)
    assert m3 == 4 and a3[2].op == s.OPS["SUB"] and a1[2].op == s.OPS["ADD"]
    prog.append(("VEC", 2))
    a4, m4 = s.program(prog)
    assert m4 == 5 and a4[4].op == s.OPS["VEC"] and a4[4].arg == 2
    # the same instructions in a fresh list or a tuple give the same codes
    a5, m5 = s.program(tuple(prog))
    assert m5 == 5 and [(a5[i].op, a5[i].arg) for i in range(5)] == [(a4[i].op, a4[i].arg) for i in range(5)]


def test_binding_operand_checks(saltlib):
    """The binding's one-pass operand marshalling: mixed dtypes and unequal
    lengths are rejected before the library is called; an explicit n skips
    the length check (the library then sees the call)."""
    torch = pytest.importorskip("torch")
    s = saltlib
    a32 = torch.zeros(8, dtype=torch.float32)
    b32 = torch.zeros(8, dtype=torch.float32)
    c64 = torch.zeros(8, dtype=torch.float64)
    short = torch.zeros(5, dtype=torch.float32)
    prog = [("VEC", 0), ("VEC", 1), ("ADD", 0), ("STORE", 2)]
    with pytest.raises(s.SaltError) as ei:
        s.salt_eval(prog, [a32, b32, c64])
    assert ei.value.status == s.ERR_DTYPE
    with pytest.raises(s.SaltError) as ei:
        s.salt_eval(prog, [a32, b32, short])
    assert ei.value.status == s.ERR_ARG
    with pytest.raises(s.SaltError) as ei:
        s.salt_dot(a32, short, torch.zeros(1, dtype=torch.float64))
    assert ei.value.status == s.ERR_ARG
    with pytest.raises(s.SaltError) as ei:
        s.salt_axpby(1.0, a32, 2.0, c64)
    assert ei.value.status == s.ERR_DTYPE
    dt, n, ptrs, contiguous = s._operands([a32, None, short], same_length=False)
    assert dt == s.F32 and n == 8 and ptrs[1] is None and contiguous
    assert s._operands([a32[::2]])[3] is False


def test_wait_limits(saltlib):
    """The poll limits of the bounded device waits: defaults, round trip,
    argument errors (no GPU needed)."""
    s = saltlib
    for which in (s.WAIT_STAGED, s.WAIT_CG_BARRIER, s.WAIT_SERVE):
        assert s.salt_get_wait_limit(which) == s.WAIT_DEFAULT_POLLS
        s.salt_set_wait_limit(which, 0)
        assert s.salt_get_wait_limit(which) == 0
        s.salt_set_wait_limit(which, s.WAIT_DEFAULT_POLLS)
        assert s.salt_get_wait_limit(which) == s.WAIT_DEFAULT_POLLS
    assert s.lib.salt_set_wait_limit(4, 5) == s.ERR_ARG
    assert s.lib.salt_set_wait_limit(s.WAIT_STAGED, -1) == s.ERR_ARG
    assert s.lib.salt_set_wait_limit(s.WAIT_STAGED, 1 << 32) == s.ERR_ARG
    assert s.lib.salt_get_wait_limit(s.WAIT_STAGED, None) == s.ERR_ARG
    # without a GPU the status query fails like every device call
    assert s.lib.salt_cg_status(None) == s.ERR_CUDA


def test_tune_cache_environment(tmp_path):
    """SALT_TUNE_CACHE: a saved tuning table is merged into a fresh process's
    table on first use (no GPU needed: the table lives on the host)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    child = (
        "import json\n"
        "from paper_1109_1264_gb300 import salt\n"
        "from paper_1109_1264_gb300.programs import PROG_E\n"
        "import sys\n"
        "if sys.argv[1] == 'save':\n"
        "    salt.salt_tune_set(PROG_E, salt.F64, 1 << 20, 4, 32, 128, 3, 0)\n"
        "    salt.salt_tune_save(sys.argv[2])\n"
        "print(json.dumps(salt.salt_tune_get(PROG_E, salt.F64, 1 << 20)))\n")
    env = dict(os.environ, PYTHONPATH=root)
    env.pop("SALT_TUNE_CACHE", None)
    r = subprocess.run([sys.executable, "-c", child, "save", str(cache)], env=env, cwd=root, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    want = json.loads(r.stdout.strip().splitlines()[-1])
    assert want["unroll"] == 4 and want["blocks_per_sm"] == 3
    r = subprocess.run([sys.executable, "-c", child, "load"], env=dict(env, SALT_TUNE_CACHE=str(cache)), cwd=root,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert json.loads(r.stdout.strip().splitlines()[-1]) == want
    # without the variable the default shape is back
    r = subprocess.run([sys.executable, "-c", child, "load"], env=env, cwd=root, capture_output=True, text=True,
                       timeout=120)
    assert json.loads(r.stdout.strip().splitlines()[-1]) != want


def test_serve_config_persistent_fields(saltlib):
    """The server configuration's persistent-mode fields: defaults and the
    checks made before any device is touched (no GPU needed)."""
    import ctypes
    s = saltlib
    cfg = s.serve_default_config()
    assert cfg.persistent == 0 and cfg.idle_us == 10000
    h = ctypes.c_void_p()
    for field, bad in (("persistent", 2), ("persistent", -1), ("idle_us", 0), ("idle_us", 10_000_001)):
        c = s.serve_default_config()
        setattr(c, field, bad)
        assert s.lib.salt_serve_start(ctypes.byref(h), ctypes.byref(c)) == s.ERR_ARG, (field, bad)
    assert s.lib.salt_serve_launches(None, None, None) == s.ERR_ARG


def test_fp64_rate_argument_errors(saltlib):
    """The FP64 issue-rate probe checks its arguments before touching a device."""
    import ctypes
    s = saltlib
    g = ctypes.c_double()
    assert s.lib.salt_fp64_rate(3, ctypes.byref(g), None) == s.ERR_ARG
    assert s.lib.salt_fp64_rate(-1, ctypes.byref(g), None) == s.ERR_ARG
    assert s.lib.salt_fp64_rate(s.FP64_FMA, None, None) == s.ERR_ARG
