"""Scalar subexpressions, elementwise DIV and device scalars on the host
(no GPU): program typing, hoisting limits, which programs keep a compiled
instantiation once their scalar subtrees are hoisted, and the argument
checks of salt_eval_ex (all made before any launch)."""
import ctypes
import random

import pytest

from oracle_pins import CG_P, CG_P0, CG_PQ, CG_Q_PQ, CG_R0, CG_XR_RHO, random_program

BASE = 0x7F0000000000  # fake device addresses: the host rejects before any use

AXPY_DS = [("DSCAL", 0), ("DSCAL", 1), ("DIV", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("ADD", 0),
           ("STORE", 1)]


def test_hoisted_programs_keep_compiled_shapes(saltlib):
    s = saltlib
    # (rho / pq) * x + y is y = a*x + y once the quotient is a slot
    assert s.salt_check_program(AXPY_DS, 2, 0) == (0, True)
    folded = [("SCAL", 0), ("SCAL", 1), ("MUL", 0), ("NEG", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1),
              ("ADD", 0), ("STORE", 1)]
    assert s.salt_check_program(folded, 2, 2) == (0, True)
    # the two equal quotients of the CG update share one slot: 4 vectors, 1
    # scalar, the compiled second pass of a CG iteration
    assert s.salt_check_program(CG_XR_RHO, 5, 0) == (1, True)
    for prog in (CG_R0, CG_P0, CG_PQ):
        assert s.salt_check_program(prog, 6, 0) == (1, True), prog
    assert s.salt_check_program(CG_Q_PQ, 5, 0) == (1, False)
    assert s.salt_check_program(CG_P, 5, 0) == (0, False)
    # elementwise division has no compiled instantiation
    assert s.salt_check_program([("VEC", 0), ("VEC", 1), ("DIV", 0), ("STORE", 2)], 3, 0) == (0, False)


@pytest.mark.parametrize("prog,nv,ns", [
    ([("VEC", 0), ("SCAL", 0), ("ADD", 0), ("STORE", 0)], 1, 1),        # vector + scalar
    ([("SCAL", 0), ("VEC", 0), ("DIV", 0), ("STORE", 0)], 1, 1),        # scalar / vector
    ([("DSCAL", 8), ("VEC", 0), ("SMUL", 0), ("STORE", 0)], 1, 0),      # device scalar index >= 8
    ([("DSCAL", 0), ("SUMSQ", 0)], 1, 0),                               # reduction of a scalar
    ([("DSCAL", 0), ("STORE", 0)], 1, 0),                               # storing a scalar
    ([("DSCAL", 0), ("DSCAL", 1), ("DOT", 0)], 1, 0),                   # dot of scalars
    ([("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("SCAL", 0)] + [("NEG", 0)] + [("VEC", 0), ("SMUL", 0), ("ADD", 0)]
     + [("STORE", 0)], 1, 8),                                           # 8 scalars + 1 hoisted slot
])
def test_scalar_typing_rejects(saltlib, prog, nv, ns):
    with pytest.raises(saltlib.SaltError) as ei:
        saltlib.salt_check_program(prog, nv, ns)
    assert ei.value.status == saltlib.ERR_PROGRAM, ei.value


def test_equal_subexpressions_share_a_slot(saltlib):
    """7 user scalars leave room for one hoisted slot: two equal
    subexpressions fit, two different ones do not."""
    s = saltlib
    q = [("DSCAL", 0), ("DSCAL", 1), ("DIV", 0)]
    same = q + [("VEC", 0), ("SMUL", 0)] + q + [("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 0)]
    assert s.salt_check_program(same, 2, 7)[0] == 0
    other = q + [("VEC", 0), ("SMUL", 0)] + [("DSCAL", 1), ("DSCAL", 0), ("DIV", 0)] + \
        [("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 0)]
    with pytest.raises(s.SaltError):
        s.salt_check_program(other, 2, 7)
    assert s.salt_check_program(other, 2, 6)[0] == 0


def test_oracle_and_library_agree_on_typing(saltlib):
    """Every random extended program the oracle accepts (within the
    library's size limits) is accepted by the library's checker."""
    rng = random.Random(21)
    checked = 0
    for _ in range(600):
        nv, ns, nd = rng.randint(1, 5), rng.randint(0, 3), rng.randint(1, 3)
        prog = random_program(rng, nv, ns, max_len=12, ndscal=nd, ext=True)
        depth = peak = 0
        for op, _ in prog:
            depth += {"VEC": 1, "SCAL": 1, "DSCAL": 1, "NEG": 0, "DOT": -2}.get(op, -1)
            peak = max(peak, depth)
        nred = sum(1 for op, _ in prog if op in ("DOT", "SUMSQ"))
        if len(prog) > 32 or peak > 8 or nred > 4:
            continue
        try:
            saltlib.salt_check_program(prog, nv, ns)
        except saltlib.SaltError as e:
            assert "scalar slots" in e.message, (prog, e)  # hoisting limit only
            continue
        checked += 1
    assert checked > 200


def _eval_ex(s, prog, dtype, n, ptrs, dptrs, ndscal=None, red=None, scalars=()):
    arr, m = s.program(prog)
    p = (ctypes.c_void_p * max(len(ptrs), 1))(*ptrs)
    sc = (ctypes.c_double * max(len(scalars), 1))(*scalars)
    ds = None if dptrs is None else (ctypes.c_void_p * max(len(dptrs), 1))(*dptrs)
    nd = len(dptrs or ()) if ndscal is None else ndscal
    return s.lib.salt_eval_ex(arr, m, dtype, n, p, None, len(ptrs), sc, len(scalars), ds, nd, red, None)


def test_eval_ex_argument_errors(saltlib):
    s = saltlib
    x, y, d0, d1 = BASE, BASE + 2 ** 20, BASE + 2 ** 22, BASE + 2 ** 22 + 8
    assert _eval_ex(s, AXPY_DS, 1, 10, [x, y], [d0]) == s.ERR_PROGRAM      # DSCAL 1 >= ndscal
    assert _eval_ex(s, AXPY_DS, 1, 10, [x, y], None, ndscal=2) == s.ERR_ARG
    assert _eval_ex(s, AXPY_DS, 1, 10, [x, y], [d0, None]) == s.ERR_ARG
    assert _eval_ex(s, AXPY_DS, 1, 10, [x, y], [d0, d1 + 4]) == s.ERR_ALIGN
    assert _eval_ex(s, AXPY_DS, 1, 10, [x, y], [d0, d1], ndscal=9) == s.ERR_ARG
    # a device scalar inside the stored vector y
    assert _eval_ex(s, AXPY_DS, 1, 10, [x, y], [d0, y + 72]) == s.ERR_ALIAS
    # ... but inside the read-only x it is fine (fails later, on the missing GPU)
    assert _eval_ex(s, AXPY_DS, 1, 10, [x, y], [d0, x + 72]) == s.ERR_CUDA
    # a device scalar where this call's reduction result goes
    prog = [("DSCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1), ("VEC", 1), ("SUMSQ", 0)]
    assert _eval_ex(s, prog, 1, 10, [x, y], [d0], red=d0) == s.ERR_ALIAS
    assert _eval_ex(s, prog, 1, 10, [x, y], [d0], red=d1) == s.ERR_CUDA
    # by-value scalar subexpressions need no device scalars at all
    folded = [("SCAL", 0), ("SCAL", 1), ("DIV", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)]
    assert _eval_ex(s, folded, 0, 10, [x, y], [], scalars=(1.0, 3.0)) == s.ERR_CUDA


def test_hoisting_preserves_the_oracle_result(saltlib):
    """The program the kernels run (scalar subtrees hoisted to slots whose
    values the host computes, one operation per node in the dtype) gives,
    under the oracle, the same bits as the original program -- including
    subtrees interleaved with statements (VEC k SUMSQ between their
    tokens)."""
    import numpy as np
    import oracle
    s = saltlib
    rng = random.Random(22)
    nrng = np.random.default_rng(22)
    checked = hoisted = 0
    for t in range(400):
        dt = np.float64 if t % 2 else np.float32
        nv, ns, nd = rng.randint(1, 5), rng.randint(0, 3), rng.randint(0, 3)
        prog = random_program(rng, nv, ns, max_len=12, ndscal=nd, ext=True)
        try:
            s.salt_check_program(prog, nv, ns)
        except s.SaltError:
            continue
        n = 17
        vecs = [(nrng.uniform(0.5, 2.0, n) * nrng.choice([-1.0, 1.0], n)).astype(dt) for _ in range(nv)]
        scalars = list(nrng.uniform(-2.0, 2.0, ns))
        dvals = list(nrng.uniform(-2.0, 2.0, nd))
        hp, slots, _ = s.salt_explain(prog, nv, scalars, s.F32 if dt == np.float32 else s.F64, dvals)
        assert all(op != "DSCAL" for op, _ in hp)
        assert len(hp) <= len(prog) and slots[:ns] == scalars
        want = [v.copy() for v in vecs]
        red_w = oracle.eval_program(prog, want, scalars, dscalars=dvals)
        got = [v.copy() for v in vecs]
        red_g = oracle.eval_program(hp, got, slots)
        for w, g in zip(want, got):
            assert np.array_equal(w.view(np.uint32 if dt == np.float32 else np.uint64),
                                  g.view(np.uint32 if dt == np.float32 else np.uint64)), (prog, hp)
        assert np.array_equal(np.array(red_w), np.array(red_g), equal_nan=True), (prog, hp)
        checked += 1
        hoisted += len(slots) > ns
    assert checked > 150 and hoisted > 60, (checked, hoisted)


def test_explain_shows_the_cse_and_folding(saltlib):
    s = saltlib
    hp, slots, comp = s.salt_explain(CG_XR_RHO, 5, (), s.F64, (6.0, 4.0))
    assert slots == [1.5] and comp
    assert hp == [("VEC", 3), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 3),
                  ("VEC", 4), ("SCAL", 0), ("VEC", 2), ("SMUL", 0), ("SUB", 0), ("STORE", 4),
                  ("VEC", 4), ("SUMSQ", 0)]
    # FP32: 1 + 2^-24 rounds to 1 in the scalar node
    hp, slots, comp = s.salt_explain([("SCAL", 0), ("SCAL", 1), ("ADD", 0), ("VEC", 0), ("SMUL", 0),
                                      ("STORE", 1)], 2, (1.0, 2.0 ** -24), s.F32)
    assert slots == [1.0, 2.0 ** -24, 1.0] and comp
    hp, slots, _ = s.salt_explain([("SCAL", 0), ("SCAL", 1), ("ADD", 0), ("VEC", 0), ("SMUL", 0),
                                   ("STORE", 1)], 2, (1.0, 2.0 ** -24), s.F64)
    assert slots[2] == 1.0 + 2.0 ** -24


@pytest.mark.parametrize("entry", ["salt_cg_diag", "salt_cg_diag_persistent"])
def test_cg_argument_errors(saltlib, entry):
    """Both CG entry points check every call of the run on the host before
    the first launch."""
    s = saltlib
    fn = getattr(s.lib, entry)
    v = [BASE + k * (1 << 24) for k in range(6)]  # d, b, x, r, p, q
    rho = BASE + (1 << 30)
    assert fn(1, 100, *v, -1, rho, None) == s.ERR_ARG             # iters < 0
    assert fn(1, 100, *v, 4, None, None) == s.ERR_ARG             # rho NULL
    assert fn(2, 100, *v, 4, rho, None) == s.ERR_DTYPE
    assert fn(1, 100, v[0] + 4, *v[1:], 4, rho, None) == s.ERR_ALIGN   # d not 8-byte aligned
    assert fn(1, 100, v[0], v[1], v[2], v[3], v[2] + 8, v[5], 4, rho, None) == s.ERR_ALIAS  # p overlaps x
    assert fn(1, 100, *v, 4, v[3] + 16, None) == s.ERR_ALIAS      # rho inside r
    assert fn(1, 100, *v, 4, rho, None) == s.ERR_CUDA             # valid: fails only for want of a GPU


@pytest.mark.parametrize("one_reduction", [False, True])
def test_cg_binding_checks_rho_before_the_call(saltlib, one_reduction):
    """The C entry points receive only rho's address, so the binding checks
    its length (2*iters + 1 entries, 2*iters + 2 for the one-reduction form),
    dtype, layout and placement before calling: a buffer one entry short is
    rejected, never written past its end."""
    import torch
    s = saltlib
    n, iters = 64, 5
    vecs = [torch.zeros(n, dtype=torch.float64) for _ in range(6)]
    need = 2 * iters + (2 if one_reduction else 1)
    with pytest.raises(s.SaltError) as e:
        s.salt_cg_diag(*vecs, iters, torch.zeros(need - 1, dtype=torch.float64), one_reduction=one_reduction)
    assert e.value.status == s.ERR_ARG and f"write {need}" in e.value.message
    with pytest.raises(s.SaltError) as e:
        s.salt_cg_diag(*vecs, iters, torch.zeros(need, dtype=torch.float32), one_reduction=one_reduction)
    assert e.value.status == s.ERR_DTYPE
    with pytest.raises(s.SaltError) as e:
        s.salt_cg_diag(*vecs, iters, torch.zeros(2 * need, dtype=torch.float64)[::2], one_reduction=one_reduction)
    assert "contiguous" in e.value.message
    # the right length on the host: rejected for its placement, still before the call
    with pytest.raises(s.SaltError) as e:
        s.salt_cg_diag(*vecs, iters, torch.zeros(need, dtype=torch.float64), one_reduction=one_reduction)
    assert "CUDA tensor" in e.value.message


def test_cg_form_table(saltlib):
    """salt_cg_diag_auto's form table: the measured defaults, pins per dtype
    and log2 bucket, reset, argument errors (no GPU needed)."""
    s = saltlib
    assert s.salt_cg_form_get(s.F32, 1 << 14) == s.CG_ONE_REDUCTION
    assert s.salt_cg_form_get(s.F32, 1 << 20) == s.CG_TWO_PASS
    assert s.salt_cg_form_get(s.F32, 1 << 28) == s.CG_ONE_REDUCTION
    assert s.salt_cg_form_get(s.F64, (1 << 19) - 1) == s.CG_ONE_REDUCTION
    assert s.salt_cg_form_get(s.F64, 1 << 19) == s.CG_TWO_PASS
    s.salt_cg_form_set(s.F64, 5000, s.CG_PERSISTENT)
    assert s.salt_cg_form_get(s.F64, 4096) == s.CG_PERSISTENT  # same bucket [2^12, 2^13)
    assert s.salt_cg_form_get(s.F64, 8192) == s.CG_ONE_REDUCTION
    s.salt_cg_form_set(s.F64, 5000, -1)
    assert s.salt_cg_form_get(s.F64, 4096) == s.CG_ONE_REDUCTION
    assert s.lib.salt_cg_form_set(s.F32, 10, 3) == s.ERR_ARG
    assert s.lib.salt_cg_form_set(7, 10, 0) == s.ERR_DTYPE
    assert s.lib.salt_cg_form_get(s.F32, 10, None) == s.ERR_ARG
