"""Batch API on the host only: item validation, capacity, configuration and
the cross-item overlap check all run before any CUDA call."""
import pytest

from paper_1109_1264_gb300 import programs as P

BASE = 0x7F0000000000


@pytest.fixture
def batch(saltlib):
    b = saltlib.Batch(4)
    yield b
    b.close()


def _add_raw(salt, b, prog, dtype, n, ptrs, scalars=()):
    import ctypes
    arr, m = salt.program(prog)
    p = (ctypes.c_void_p * max(len(ptrs), 1))(*ptrs)
    sc = (ctypes.c_double * max(len(scalars), 1))(*scalars)
    idx = ctypes.c_int32(-7)
    st = salt.lib.salt_batch_add(b.handle, arr, m, dtype, n, p, len(ptrs), sc, len(scalars), ctypes.byref(idx))
    return st, idx.value


def test_add_validates_like_eval(saltlib, batch):
    s = saltlib
    assert _add_raw(s, batch, P.PROG_D, 2, 10, [BASE, BASE + 4096, BASE + 8192, BASE + 12288])[0] == s.ERR_DTYPE
    assert _add_raw(s, batch, P.PROG_D, 0, 10, [BASE, BASE + 4100, BASE + 8192, BASE + 12288])[0] == s.ERR_ALIGN
    assert _add_raw(s, batch, P.PROG_D, 0, 100, [BASE, BASE + 4096, BASE + 8192, BASE + 16])[0] == s.ERR_ALIAS
    # not a compiled shape: cannot be batched
    odd = [("VEC", 0), ("NEG", 0), ("STORE", 1)]
    st, _ = _add_raw(s, batch, odd, 0, 10, [BASE, BASE + 4096])
    assert st == s.ERR_PROGRAM and "batched" in s.salt_last_error()


def test_result_slots_capacity_and_info(saltlib, batch):
    s = saltlib
    st, i0 = _add_raw(s, batch, P.PROG_CG, 1, 100, [BASE, BASE + 4096, BASE + 8192], [0.5, 0.25])
    assert st == s.OK and i0 == 0
    st, i1 = _add_raw(s, batch, P.PROG_D, 1, 50, [BASE + 2 ** 20, BASE + 2 ** 21, BASE + 2 ** 22, BASE + 2 ** 23])
    assert st == s.OK and i1 == -1
    st, i2 = _add_raw(s, batch, P.PROG_DOT, 0, 30, [BASE + 2 ** 24, BASE + 2 ** 25])
    assert st == s.OK and i2 == 1
    import ctypes
    idx = ctypes.c_int32()
    assert s.lib.salt_batch_add_nrm2(batch.handle, 0, 30, BASE + 2 ** 26, ctypes.byref(idx)) == s.OK
    assert idx.value == 2
    assert s.lib.salt_batch_add_nrm2(batch.handle, 0, 30, BASE + 2 ** 26, ctypes.byref(idx)) == s.ERR_BUDGET
    info = batch.info()
    # CG: 3 loads + 2 stores, D: 3 + 1, DOT: 2, nrm2: 1
    assert info == {"items": 4, "results": 3, "bytes": 5 * 8 * 100 + 4 * 8 * 50 + 2 * 4 * 30 + 4 * 30}
    batch.clear()
    assert batch.info()["items"] == 0


def test_config_validation(saltlib, batch):
    batch.set_config(4, 128, 2, 32768)
    assert batch.get_config() == {"unroll": 4, "block": 128, "blocks_per_sm": 2, "tile_bytes": 32768,
                                  "vec_bytes": 32}
    batch.set_vec_bytes(16)
    assert batch.get_config()["vec_bytes"] == 16
    for bad in ((3, 128, 2, 32768), (2, 96, 2, 32768), (2, 512, 2, 32768), (2, 128, 33, 32768),
                (2, 128, 2, 1000), (2, 128, 2, 512)):
        with pytest.raises(saltlib.SaltError):
            batch.set_config(*bad)
    for bad in (0, 8, 24, 64):
        with pytest.raises(saltlib.SaltError):
            batch.set_vec_bytes(bad)


def test_cross_item_overlap_rejected_at_launch(saltlib, batch):
    """Two items that are each valid but write memory the other reads."""
    s = saltlib
    assert _add_raw(s, batch, P.PROG_SCALE, 1, 100, [BASE, BASE + 4096], [2.0])[0] == s.OK
    assert _add_raw(s, batch, P.PROG_SCALE, 1, 100, [BASE + 4096 + 64, BASE + 2 ** 20], [2.0])[0] == s.OK
    assert s.lib.salt_batch_launch(batch.handle, None, None) == s.ERR_ALIAS
    assert "overlap" in s.salt_last_error()
    # read-only sharing between items is fine: fails only later, on the missing GPU (or succeeds)
    batch.clear()
    assert _add_raw(s, batch, P.PROG_SCALE, 1, 100, [BASE, BASE + 4096], [2.0])[0] == s.OK
    assert _add_raw(s, batch, P.PROG_SCALE, 1, 100, [BASE, BASE + 8192], [2.0])[0] == s.OK
    import torch
    if not torch.cuda.is_available():
        assert s.lib.salt_batch_launch(batch.handle, None, None) == s.ERR_CUDA
