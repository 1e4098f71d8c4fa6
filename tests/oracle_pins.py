"""Pins of the oracle to facts other than itself.

Each ``check_*`` takes the path of an oracle library build and raises
AssertionError when the oracle disagrees with the paper or the mathematics.
``test_oracle_pins.py`` runs them on the real build; ``test_oracle_mutants.py``
runs them on builds with planted mistakes and requires each mistake to be
caught by at least one pin.
"""
from __future__ import annotations

import math
import os
import random
from fractions import Fraction

import numpy as np

import oracle
from oracle import exact
from oracle import PROG_AXPBY, PROG_CG, PROG_D, PROG_E

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U64 = 2.0 ** -53


def _eq_bits_or_nan(a: np.ndarray, b: np.ndarray) -> bool:
    a = np.asarray(a)
    b = np.asarray(b)
    if a.shape != b.shape:
        return False
    both_nan = np.isnan(a) & np.isnan(b)
    same = (a == b) | both_nan
    return bool(np.all(same))


# ------------------------------------------------------------- elementwise --

def check_figure1_golden(path):
    """Figure 1 worked example d = a + (b - c), hand-computed values."""
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "figure1_d_eq_a_plus_b_minus_c.txt"))
            if l.strip() and not l.startswith("#")]
    cols = list(zip(*rows))
    for dt in (np.float64, np.float32):
        a, b, c, want = (np.array(col, dtype=dt) for col in cols)
        d = np.zeros_like(a)
        oracle.eval_program(PROG_D, [a, b, c, d], path=path)
        assert _eq_bits_or_nan(d, want), (dt, d, want)


def check_d_integer_identity(path):
    """Integers below 2^50 (FP64) / 2^22 (FP32): every node is exact, so the
    result must equal exact integer arithmetic."""
    rng = np.random.default_rng(11)
    for dt, lim in ((np.float64, 2 ** 50), (np.float32, 2 ** 22)):
        n = 10007
        ints = [rng.integers(-lim, lim, n) for _ in range(3)]
        a, b, c = (x.astype(dt) for x in ints)
        d = np.zeros(n, dtype=dt)
        oracle.eval_program(PROG_D, [a, b, c, d], path=path)
        want = ints[0] + (ints[1] - ints[2])
        assert np.array_equal(d.astype(np.float64), want.astype(np.float64)), dt


def check_e_and_axpby_exact(path):
    """alpha = 1.5, beta = -0.25 and multiples of 4: e = alpha a + beta b - c d
    and y = alpha x + beta y are exact in both formats."""
    rng = np.random.default_rng(12)
    alpha, beta = 1.5, -0.25
    for dt in (np.float64, np.float32):
        n = 4099
        A = rng.integers(-2 ** 10, 2 ** 10, n) * 4
        B = rng.integers(-2 ** 10, 2 ** 10, n) * 4
        C = rng.integers(-2 ** 10, 2 ** 10, n)
        D = rng.integers(-2 ** 10, 2 ** 10, n)
        a, b, c, d = (x.astype(dt) for x in (A, B, C, D))
        e = np.zeros(n, dtype=dt)
        oracle.eval_program(PROG_E, [a, b, c, d, e], [alpha, beta], path=path)
        want = [Fraction(3, 2) * int(x) - Fraction(1, 4) * int(y) - int(z) * int(w) for x, y, z, w in zip(A, B, C, D)]
        assert all(Fraction(float(g)) == w for g, w in zip(e, want)), dt
        x, y = a.copy(), b.copy()
        oracle.eval_program(PROG_AXPBY, [x, y], [alpha, beta], path=path)
        want = [Fraction(3, 2) * int(p) - Fraction(1, 4) * int(q) for p, q in zip(A, B)]
        assert all(Fraction(float(g)) == w for g, w in zip(y, want)), dt
        assert np.array_equal(x, a), "x must be left untouched"


def random_program(rng: random.Random, nvecs: int, nscal: int, max_len: int = 20,
                   ndscal: int = 0, ext: bool = False):
    """A random well-typed postfix program over nvecs vectors / nscal scalars
    (and ndscal device scalars).  With ``ext`` it also draws elementwise DIV
    and scalar-typed ADD/SUB/MUL/DIV/NEG nodes.  Keeps stack depth <= 6,
    ends with an empty stack and has >= 1 output."""
    prog = []
    stack = []  # 'v' or 's'
    outputs = 0
    while True:
        can_finish = len(stack) == 0 and outputs > 0
        if can_finish and (len(prog) >= max_len or rng.random() < 0.15):
            return prog
        choices = []
        if len(stack) < 6:
            choices += ["VEC"] * 3
            if nscal:
                choices += ["SCAL"]
            if ndscal:
                choices += ["DSCAL"]
        if len(stack) >= 2 and stack[-1] == "v" and stack[-2] == "v":
            choices += ["ADD", "SUB", "MUL", "DOT"]
            if ext:
                choices += ["DIV"]
        if ext and len(stack) >= 2 and stack[-1] == "s" and stack[-2] == "s":
            choices += ["S_ADD", "S_SUB", "S_MUL", "S_DIV"]
        if ext and stack and stack[-1] == "s":
            choices += ["S_NEG"]
        if len(stack) >= 2 and stack[-1] == "v" and stack[-2] == "s":
            choices += ["SMUL"] * 3
        if stack and stack[-1] == "v":
            choices += ["NEG", "STORE", "STORE", "SUMSQ"]
        if not choices:
            # scalar on top with no vector to scale: push a vector to consume it
            choices = ["VEC"]
        op = rng.choice(choices)
        if op == "VEC":
            prog.append(("VEC", rng.randrange(nvecs))); stack.append("v")
        elif op == "SCAL":
            prog.append(("SCAL", rng.randrange(nscal))); stack.append("s")
        elif op == "DSCAL":
            prog.append(("DSCAL", rng.randrange(ndscal))); stack.append("s")
        elif op in ("ADD", "SUB", "MUL", "DIV"):
            prog.append((op, 0)); stack.pop()
        elif op in ("S_ADD", "S_SUB", "S_MUL", "S_DIV"):
            prog.append((op[2:], 0)); stack.pop()
        elif op == "S_NEG":
            prog.append(("NEG", 0))
        elif op == "SMUL":
            prog.append((op, 0)); stack.pop(); stack.pop(); stack.append("v")
        elif op == "NEG":
            prog.append((op, 0))
        elif op == "STORE":
            prog.append(("STORE", rng.randrange(nvecs))); stack.pop(); outputs += 1
        elif op == "DOT":
            prog.append((op, 0)); stack.pop(); stack.pop(); outputs += 1
        elif op == "SUMSQ":
            prog.append((op, 0)); stack.pop(); outputs += 1
        if len(prog) > 40:
            # force termination: drain the stack
            while stack:
                if stack[-1] == "s":
                    prog.append(("VEC", 0)); prog.append(("SMUL", 0)); stack[-1] = "v"
                    continue
                prog.append(("STORE", rng.randrange(nvecs))); stack.pop(); outputs += 1
            return prog


def _check_against_exact(prog, vecs, scalars, dt, path, dscalars=()):
    ours = [v.copy() for v in vecs]
    red = oracle.eval_program(prog, ours, scalars, path=path, dscalars=dscalars)
    want, red_exact, red_abs = exact.exact_program(prog, vecs, scalars, dt, dscalars)
    for k, (got, w) in enumerate(zip(ours, want)):
        assert _eq_bits_or_nan(got.astype(np.float64), np.array(w, dtype=np.float64)), (prog, k)
    # Reductions: a sequential FP64 sum obeys |err| <= gamma_n sum|terms|
    # (Higham, Eq. 3.5), with the exact terms as reference.
    n = len(vecs[0]) if vecs else 0
    assert len(red) == len(red_exact)
    for r, re, ra in zip(red, red_exact, red_abs):
        err = abs(Fraction(r) - re)
        bound = Fraction(exact.gamma(n + 1, U64)) * ra
        assert err <= bound, (prog, float(err), float(bound))


def check_brute_force_random_programs(path, count=60):
    """Random well-typed programs on tiny n, against per-element exact
    rational arithmetic with one rounding per node."""
    rng = random.Random(5)
    nrng = np.random.default_rng(5)
    for t in range(count):
        dt = np.float64 if t % 2 == 0 else np.float32
        nvecs = rng.randint(1, 6)
        nscal = rng.randint(0, 3)
        prog = random_program(rng, nvecs, nscal)
        n = rng.choice([0, 1, 2, 3, 5, 7, 8, 9, 15, 16, 17, 31, 33, 63, 64, 71])
        vecs = [nrng.uniform(-1, 1, n).astype(dt) for _ in range(nvecs)]
        scalars = list(nrng.uniform(-2, 2, nscal))
        _check_against_exact(prog, vecs, scalars, dt, path)


def _finite_exact(prog, vecs, scalars, dt, dscalars):
    """True when exact evaluation stays finite (no zero denominator, no
    overflow), i.e. when the rational reference is defined."""
    try:
        want, _, _ = exact.exact_program(prog, vecs, scalars, dt, dscalars)
    except (ZeroDivisionError, OverflowError):
        return False
    return all(math.isfinite(t) for w in want for t in w)


def check_brute_force_extended_programs(path, count=80):
    """Random programs with elementwise DIV, scalar-typed nodes and device
    scalars, on tiny n, against exact rational arithmetic with one rounding
    per node (scalar nodes included: Section 4.2 init/load_once values are
    computed once, in the program's dtype)."""
    rng = random.Random(11)
    nrng = np.random.default_rng(11)
    checked = 0
    for t in range(count):
        dt = np.float64 if t % 2 == 0 else np.float32
        nvecs = rng.randint(1, 5)
        nscal = rng.randint(0, 3)
        ndscal = rng.randint(1, 3)
        prog = random_program(rng, nvecs, nscal, ndscal=ndscal, ext=True)
        n = rng.choice([0, 1, 3, 8, 17, 33, 64])
        # magnitudes in [0.5, 2): quotients of inputs stay in range
        vecs = [(nrng.uniform(0.5, 2.0, n) * nrng.choice([-1.0, 1.0], n)).astype(dt)
                for _ in range(nvecs)]
        scalars = list(nrng.uniform(0.5, 2.0, nscal) * nrng.choice([-1.0, 1.0], nscal))
        dscalars = list(nrng.uniform(0.5, 2.0, ndscal) * nrng.choice([-1.0, 1.0], ndscal))
        if not _finite_exact(prog, vecs, scalars, dt, dscalars):
            continue
        _check_against_exact(prog, vecs, scalars, dt, path, dscalars)
        checked += 1
    assert checked >= count // 2, checked


def check_div_exact(path):
    """a / b with a = q * b for small integers q and b: the quotient is q
    exactly (both operands and q representable, IEEE division correctly
    rounded); and 1 / 3 is the correctly rounded third in each precision."""
    rng = np.random.default_rng(12)
    for dt in (np.float64, np.float32):
        n = 333
        q = rng.integers(-1000, 1000, n)
        b = rng.integers(1, 1000, n) * rng.choice([-1, 1], n)
        a = (q * b).astype(dt)
        out = np.zeros(n, dtype=dt)
        oracle.eval_program([("VEC", 0), ("VEC", 1), ("DIV", 0), ("STORE", 2)],
                            [a, b.astype(dt), out], path=path)
        assert np.array_equal(out.astype(np.int64), q), dt
        ones = np.ones(4, dtype=dt)
        threes = np.full(4, 3.0, dtype=dt)
        oracle.eval_program([("VEC", 0), ("VEC", 1), ("DIV", 0), ("STORE", 2)],
                            [ones, threes, out[:4]], path=path)
        assert np.all(out[:4] == exact.round_to(Fraction(1, 3), dt)), dt


def check_scalar_nodes(path):
    """Scalar-typed nodes are one operation each, in the program's dtype,
    with operands in postfix order: (s0 - s1), (s0 / s1), -(s0), (s0 * s1)
    scaled onto a vector of ones; in FP32 the scalar node result is rounded
    to float: 1 + 2^-24 rounds to 1 (ties to even), so the product with
    1 + 2^-23 is 1 + 2^-23, where an unrounded FP64 scalar would give
    1 + 2^-22."""
    for dt in (np.float64, np.float32):
        ones = np.ones(5, dtype=dt)
        out = np.zeros(5, dtype=dt)
        cases = [("SUB", 3.0, 1.0, 2.0), ("DIV", 1.0, 4.0, 0.25), ("MUL", -3.0, 0.5, -1.5),
                 ("ADD", 1.25, 2.0, 3.25)]
        for op, s0, s1, want in cases:
            oracle.eval_program([("SCAL", 0), ("SCAL", 1), (op, 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)],
                                [ones, out], [s0, s1], path=path)
            assert np.all(out == want), (dt, op, out)
            oracle.eval_program([("DSCAL", 0), ("DSCAL", 1), (op, 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)],
                                [ones, out], dscalars=[s0, s1], path=path)
            assert np.all(out == want), (dt, op, "dscal", out)
        oracle.eval_program([("DSCAL", 1), ("NEG", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)],
                            [ones, out], dscalars=[7.0, 2.5], path=path)
        assert np.all(out == -2.5), (dt, out)
    v = np.full(3, 1.0 + 2.0 ** -23, dtype=np.float32)
    out = np.zeros(3, dtype=np.float32)
    oracle.eval_program([("SCAL", 0), ("SCAL", 1), ("ADD", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)],
                        [v, out], [1.0, 2.0 ** -24], path=path)
    assert np.all(out == np.float32(1.0 + 2.0 ** -23)), out
    # a device scalar is rounded to float once: 1 + 2^-24 + 2^-40 -> 1 + 2^-23
    oracle.eval_program([("DSCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)],
                        [np.ones(3, dtype=np.float32), out], dscalars=[1.0 + 2.0 ** -24 + 2.0 ** -40], path=path)
    assert np.all(out == np.float32(1.0 + 2.0 ** -23)), out


# Conjugate gradients (Hestenes-Stiefel) as three fused programs whose
# scalars alpha = rho / (p.q) and beta = rho' / rho are scalar subtrees over
# device-resident reduction results.  Slots: 0 d (diagonal of A), 1 p, 2 q,
# 3 x, 4 r.
CG_Q_PQ = [("VEC", 0), ("VEC", 1), ("MUL", 0), ("STORE", 2), ("VEC", 1), ("VEC", 2), ("DOT", 0)]
CG_XR_RHO = [("VEC", 3), ("DSCAL", 0), ("DSCAL", 1), ("DIV", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0),
             ("STORE", 3),
             ("VEC", 4), ("DSCAL", 0), ("DSCAL", 1), ("DIV", 0), ("VEC", 2), ("SMUL", 0), ("SUB", 0),
             ("STORE", 4),
             ("VEC", 4), ("SUMSQ", 0)]
CG_P = [("VEC", 4), ("DSCAL", 0), ("DSCAL", 1), ("DIV", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0),
        ("STORE", 1)]


def cg_diagonal(evalp, d, b, iters):
    """Runs ``iters`` CG iterations for diag(d) x = b from x = 0 with the
    three programs above through ``evalp(prog, vecs, dscalars)``; returns x
    and the residual norms sqrt(rho_k)."""
    dt = d.dtype
    n = d.shape[0]
    p, q, x, r = b.copy(), np.zeros(n, dt), np.zeros(n, dt), b.copy()
    vecs = [d, p, q, x, r]
    rho = evalp([("VEC", 4), ("SUMSQ", 0)], vecs, [])[0]
    hist = [math.sqrt(rho)]
    for _ in range(iters):
        pq = evalp(CG_Q_PQ, vecs, [])[0]
        rho_new = evalp(CG_XR_RHO, vecs, [rho, pq])[0]
        evalp(CG_P, vecs, [rho_new, rho])
        rho = rho_new
        hist.append(math.sqrt(rho))
    return x, hist


# The same iteration as two passes (the search-direction update fused into
# the next matrix-vector product), started from any x; slot 5 holds b.
CG_R0 = [("VEC", 5), ("VEC", 0), ("VEC", 3), ("MUL", 0), ("SUB", 0), ("STORE", 4), ("VEC", 4), ("SUMSQ", 0)]
CG_P0 = [("VEC", 4), ("STORE", 1), ("VEC", 0), ("VEC", 1), ("MUL", 0), ("STORE", 2), ("VEC", 1), ("VEC", 2),
         ("DOT", 0)]
CG_PQ = [("VEC", 4), ("DSCAL", 0), ("DSCAL", 1), ("DIV", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 1),
         ("VEC", 0), ("VEC", 1), ("MUL", 0), ("STORE", 2), ("VEC", 1), ("VEC", 2), ("DOT", 0)]


def cg_diagonal_two_pass(evalp, d, b, x0, iters):
    """CG from x0 with two programs per iteration; returns x and the history
    [rho_0, pq_0, rho_1, pq_1, ..., rho_iters]."""
    n = d.shape[0]
    dt = d.dtype
    p, q, r = np.zeros(n, dt), np.zeros(n, dt), np.zeros(n, dt)
    x = x0.copy()
    vecs = [d, p, q, x, r, b]
    hist = [evalp(CG_R0, vecs, [])[0]]
    for k in range(iters):
        if k == 0:
            hist.append(evalp(CG_P0, vecs, [])[0])
        else:
            hist.append(evalp(CG_PQ, vecs, [hist[2 * k], hist[2 * k - 2]])[0])
        hist.append(evalp(CG_XR_RHO, vecs, [hist[2 * k], hist[2 * k + 1]])[0])
    return x, hist


# Conjugate gradients with one reduction phase per iteration (Chronopoulos
# and Gear 1989): with w = A r kept implicit (diag(d) o r), each iteration
# updates p = r + beta p and s = A r + beta s (s = A p in exact arithmetic),
# then x = x + alpha p, r = r - alpha s, and reduces gamma = r.r and
# delta = (A r).r of the new residual in the same pass; the scalars are
# beta = gamma_k / gamma_{k-1} and alpha_k = gamma_k / (delta_k - beta_k
# gamma_k / alpha_{k-1}), alpha_0 = gamma_0 / delta_0.  In exact arithmetic
# the iterates are those of Hestenes-Stiefel CG.  Slots: 0 d, 1 p, 2 s, 3 x,
# 4 r, 5 b; device scalars: 0 beta, 1 alpha (values in T, so exact).
CGC_START = [("VEC", 5), ("VEC", 0), ("VEC", 3), ("MUL", 0), ("SUB", 0), ("STORE", 4),
             ("VEC", 4), ("SUMSQ", 0), ("VEC", 0), ("VEC", 4), ("MUL", 0), ("VEC", 4), ("DOT", 0)]
_CGC_TAIL = [("VEC", 3), ("DSCAL", 1), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 3),
             ("VEC", 4), ("DSCAL", 1), ("VEC", 2), ("SMUL", 0), ("SUB", 0), ("STORE", 4),
             ("VEC", 4), ("SUMSQ", 0), ("VEC", 0), ("VEC", 4), ("MUL", 0), ("VEC", 4), ("DOT", 0)]
CGC_FIRST = [("VEC", 4), ("STORE", 1), ("VEC", 0), ("VEC", 4), ("MUL", 0), ("STORE", 2)] + _CGC_TAIL
CGC_STEP = [("VEC", 4), ("DSCAL", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 1),
            ("VEC", 0), ("VEC", 4), ("MUL", 0), ("DSCAL", 0), ("VEC", 2), ("SMUL", 0), ("ADD", 0),
            ("STORE", 2)] + _CGC_TAIL


def cg_diagonal_one_reduction(evalp, d, b, x0, iters):
    """The one-reduction-phase CG from x0 with one program per iteration;
    the scalars are computed in the vectors' precision from the reductions
    rounded to it (as a DSCAL node reads them).  Returns x and the history
    [gamma_0, delta_0, gamma_1, delta_1, ..., gamma_iters, delta_iters]."""
    n = d.shape[0]
    dt = d.dtype.type
    p, s, r = np.zeros(n, d.dtype), np.zeros(n, d.dtype), np.zeros(n, d.dtype)
    x = x0.copy()
    vecs = [d, p, s, x, r, b]
    hist = list(evalp(CGC_START, vecs, []))
    alpha = None
    for k in range(iters):
        g, dl = dt(hist[2 * k]), dt(hist[2 * k + 1])
        if k == 0:
            alpha = g / dl
            out = evalp(CGC_FIRST, vecs, [0.0, float(alpha)])
        else:
            beta = g / dt(hist[2 * k - 2])
            alpha = g / (dl - beta * g / alpha)
            out = evalp(CGC_STEP, vecs, [float(beta), float(alpha)])
        hist.extend(out)
    return x, hist


def check_cg_distinct_eigenvalues(path):
    """CG on an SPD matrix with k distinct eigenvalues reaches the solution
    in at most k iterations in exact arithmetic (Hestenes and Stiefel 1952;
    Nocedal and Wright, Numerical Optimization, Thm. 5.4).  A diagonal A
    with k = 4 distinct entries in [1, 8]: after 4 iterations x equals b / d
    to a few ulps of the condition number, while after 3 it does not."""
    rng = np.random.default_rng(13)

    def evalp(prog, vecs, ds):
        return oracle.eval_program(prog, vecs, dscalars=ds, path=path)

    for dt, tol in ((np.float64, 1e-13), (np.float32, 2e-6)):
        n = 1001
        d = rng.choice([1.0, 2.0, 5.0, 8.0], n).astype(dt)
        b = rng.uniform(-1, 1, n).astype(dt)
        xs = b.astype(np.float64) / d.astype(np.float64)
        x3, _ = cg_diagonal(evalp, d, b, 3)
        x4, hist = cg_diagonal(evalp, d, b, 4)
        err3 = np.linalg.norm(x3 - xs) / np.linalg.norm(xs)
        err4 = np.linalg.norm(x4 - xs) / np.linalg.norm(xs)
        assert err4 < tol, (dt, err4)
        assert err3 > 1e-3, (dt, err3)
        assert hist[-1] < tol * hist[0], (dt, hist)
        # the two-pass form performs the same operations: the same bits
        x2, h2 = cg_diagonal_two_pass(evalp, d, b, np.zeros(n, dt), 4)
        assert np.array_equal(x2, x4), dt
        assert [math.sqrt(v) for v in h2[0::2]] == hist, dt
        # from a nonzero start it converges to the same solution
        x0 = rng.uniform(-3, 3, n).astype(dt)
        x5, _ = cg_diagonal_two_pass(evalp, d, b, x0, 4)
        assert np.linalg.norm(x5 - xs) / np.linalg.norm(xs) < 10 * tol, dt
        # the one-reduction form: the same termination in 4 iterations (not 3),
        # from zero and from x0
        for start in (np.zeros(n, dt), x0):
            xc3, _ = cg_diagonal_one_reduction(evalp, d, b, start, 3)
            xc4, hc = cg_diagonal_one_reduction(evalp, d, b, start, 4)
            assert np.linalg.norm(xc4 - xs) / np.linalg.norm(xs) < 10 * tol, dt
            assert np.linalg.norm(xc3 - xs) / np.linalg.norm(xs) > 1e-3, dt
            assert hc[-2] < (10 * tol) ** 2 * hc[0] * 100, (dt, hc)


def check_cg_one_reduction_matches_cg(path):
    """In exact arithmetic the one-reduction CG produces the Hestenes-Stiefel
    iterates: on a well-conditioned diagonal system (d in [1, 4]) the two
    oracles' x after k iterations agree to rounding, for every k, while the
    residual falls by orders of magnitude; and gamma_k = r_k.r_k matches the
    two-pass rho_k."""
    rng = np.random.default_rng(29)

    def evalp(prog, vecs, ds):
        return oracle.eval_program(prog, vecs, dscalars=ds, path=path)

    for dt, tol in ((np.float64, 1e-12), (np.float32, 1e-4)):
        n = 777
        d = rng.uniform(1.0, 4.0, n).astype(dt)
        b = rng.uniform(-1, 1, n).astype(dt)
        x0 = rng.uniform(-1, 1, n).astype(dt)
        for k in (1, 2, 5, 12):
            xh, hh = cg_diagonal_two_pass(evalp, d, b, x0, k)
            xc, hc = cg_diagonal_one_reduction(evalp, d, b, x0, k)
            scale = max(np.linalg.norm(xh.astype(np.float64)), 1.0)
            assert np.linalg.norm(xc.astype(np.float64) - xh) / scale < tol, (dt, k)
            for j in range(k + 1):
                assert abs(hc[2 * j] - hh[2 * j]) <= tol * hh[0] + 1e-300, (dt, k, j, hc[2 * j], hh[2 * j])
        _, hc = cg_diagonal_one_reduction(evalp, d, b, x0, 12)
        assert hc[-2] < 1e-6 * hc[0], (dt, hc[-2], hc[0])


def check_tail_lengths(path):
    """Every n in 0..64 and 2^k + 7 (k <= 9): the body/tail split of the
    paper's loop template must not matter (Listing 2: the tail elements get
    the same scalar operation)."""
    nrng = np.random.default_rng(6)
    sizes = list(range(0, 65)) + [2 ** k + 7 for k in range(3, 10)]
    for n in sizes:
        for dt in (np.float64, np.float32):
            vecs = [nrng.uniform(-1, 1, n).astype(dt) for _ in range(5)]
            _check_against_exact(PROG_E if n % 2 else PROG_D, vecs, [1.5, -0.25], dt, path)


def check_cg_store_then_load(path):
    """STORE k followed by VEC k reads the stored value (r is updated before
    rho = r.r and p = r + beta p), exact on small integers."""
    rng = np.random.default_rng(7)
    for dt in (np.float64, np.float32):
        n = 777
        R = rng.integers(-100, 100, n)
        Q = rng.integers(-100, 100, n)
        P = rng.integers(-100, 100, n)
        r, q, p = (x.astype(dt) for x in (R, Q, P))
        red = oracle.eval_program(PROG_CG, [r, q, p], [2.0, -0.5], path=path)
        Rn = R - 2 * Q
        assert np.array_equal(r.astype(np.int64), Rn)
        assert np.array_equal(p.astype(np.float64), (Rn - 0.5 * P).astype(np.float64))
        assert red[0] == float(int(np.sum(Rn * Rn)))


def check_special_values(path):
    """IEEE special cases: NaN propagates, inf - inf = NaN, -(+0) = -0,
    (-0) + (-0) = -0, FP32 subnormals are kept (no flush to zero)."""
    for dt in (np.float64, np.float32):
        a = np.array([np.nan, np.inf, 0.0, -0.0, 1.0], dtype=dt)
        b = np.array([1.0, np.inf, 0.0, -0.0, np.nan], dtype=dt)
        out = np.zeros(5, dtype=dt)
        oracle.eval_program([("VEC", 0), ("VEC", 1), ("SUB", 0), ("STORE", 2)], [a, b, out], path=path)
        assert np.isnan(out[0]) and np.isnan(out[1]) and np.isnan(out[4])
        assert out[2] == 0 and not np.signbit(out[2])  # 0 - 0 = +0
        assert out[3] == 0 and not np.signbit(out[3])  # -0 - -0 = +0
        oracle.eval_program([("VEC", 0), ("VEC", 1), ("ADD", 0), ("STORE", 2)], [a, b, out], path=path)
        assert np.signbit(out[3]) and out[3] == 0  # -0 + -0 = -0
        z = np.zeros(3, dtype=dt)
        oracle.eval_program([("VEC", 0), ("NEG", 0), ("STORE", 1)], [np.zeros(3, dtype=dt), z], path=path)
        assert np.all(np.signbit(z))
    tiny = np.array([2.0 ** -149] * 4, dtype=np.float32)
    out = np.zeros(4, dtype=np.float32)
    oracle.eval_program([("VEC", 0), ("VEC", 0), ("ADD", 0), ("STORE", 1)], [tiny, out], path=path)
    assert np.all(out == np.float32(2.0 ** -148))


def check_invalid_programs(path):
    bad = [
        [("ADD", 0)],
        [("VEC", 0), ("SCAL", 0), ("SMUL", 0), ("STORE", 0)],  # operands in wrong order
        [("VEC", 0), ("VEC", 0)],  # leftover stack
        [("VEC", 5), ("STORE", 0)],  # vector index out of range
        [("SCAL", 0), ("STORE", 0)],  # storing a scalar
        [("VEC", 0), ("SCAL", 0), ("ADD", 0), ("STORE", 0)],  # vector + scalar
        [("SCAL", 0), ("VEC", 0), ("DIV", 0), ("STORE", 0)],  # scalar / vector
        [("DSCAL", 2), ("VEC", 0), ("SMUL", 0), ("STORE", 0)],  # device scalar out of range
        [("DSCAL", 0), ("SUMSQ", 0)],  # reduction of a scalar
    ]
    for prog in bad:
        v = [np.zeros(4), np.zeros(4)]
        try:
            oracle.eval_program(prog, v, [1.0], path=path, dscalars=[1.0, 2.0])
        except oracle.OracleProgramError:
            continue
        raise AssertionError(f"accepted invalid program {prog}")


# -------------------------------------------------------------- reductions --

def check_dot_closed_forms(path):
    """sum_{i<n} i = n(n-1)/2 and sum i^2 = (n-1)n(2n-1)/6, exact in FP64
    while below 2^53."""
    for n in (0, 1, 2, 7, 1000, 2 ** 16 + 7, 2 ** 20):
        for dt in (np.float64, np.float32):
            if dt == np.float32 and n > 2 ** 24:
                continue
            x = np.arange(n, dtype=dt)
            y = np.ones(n, dtype=dt)
            assert oracle.dot(x, y, path=path) == n * (n - 1) // 2, (n, dt)
            if n <= 2 ** 17:
                s2 = (n - 1) * n * (2 * n - 1) // 6
                assert oracle.dot(x, x, path=path) == s2, (n, dt)
                assert oracle.eval_program([("VEC", 0), ("SUMSQ", 0)], [x], path=path)[0] == s2
                assert oracle.eval_program([("VEC", 0), ("VEC", 1), ("DOT", 0)], [x, y], path=path)[0] == n * (n - 1) // 2


def check_nrm2_closed_forms(path):
    """nrm2(0..n-1) = correctly rounded sqrt of the exact integer sum of
    squares; math.sqrt is correctly rounded (IEEE 754)."""
    for n in (0, 1, 2, 3, 10, 1000, 2 ** 17):
        for dt in (np.float64, np.float32):
            x = np.arange(n, dtype=dt)
            s2 = (n - 1) * n * (2 * n - 1) // 6 if n else 0
            assert oracle.nrm2(x, path=path) == math.sqrt(s2), (n, dt)
            assert oracle.nrm2(-x, path=path) == math.sqrt(s2), (n, dt)


def check_nrm2_scaling(path):
    """c * ones(4^k) has norm c * 2^k exactly, including c = 2^+-600 whose
    squares overflow / underflow FP64 without scaling."""
    for dt, cs in ((np.float64, (2.0 ** 600, 2.0 ** -600, 3.0, 2.0 ** -1000)), (np.float32, (2.0 ** 100, 2.0 ** -100, 3.0))):
        for c in cs:
            for k in (0, 1, 3, 6):
                x = np.full(4 ** k, c, dtype=dt)
                assert oracle.nrm2(x, path=path) == c * 2 ** k, (dt, c, k, oracle.nrm2(x, path=path))


def check_dot_error_bound(path):
    """Plain sequential FP64 dot: |err| <= gamma_n sum|x_i y_i| (Higham,
    Eq. 3.5) against the exactly rounded reference; and FP32 inputs are
    widened, so the same FP64 bound holds."""
    rng = np.random.default_rng(8)
    for n in (1000, 2 ** 16 + 7, 2 ** 20):
        for dt in (np.float64, np.float32):
            x = rng.uniform(-1, 1, n).astype(dt)
            y = rng.uniform(-1, 1, n).astype(dt)
            got = oracle.dot(x, y, path=path)
            ref = exact.exact_dot(x, y)
            bound = exact.gamma(n, U64) * exact.abs_dot(x, y)
            assert abs(got - ref) <= bound, (n, dt, got, ref, bound)
            got_p = oracle.eval_program([("VEC", 0), ("VEC", 1), ("DOT", 0)], [x, y], path=path)[0]
            assert abs(got_p - ref) <= bound
            nr = oracle.nrm2(x, path=path)
            nref = exact.exact_nrm2(x)
            assert abs(nr - nref) <= (exact.gamma(n + 2, U64) + 2 * U64) * nref, (n, dt)


ALL_CHECKS = [
    check_figure1_golden,
    check_d_integer_identity,
    check_e_and_axpby_exact,
    check_brute_force_random_programs,
    check_brute_force_extended_programs,
    check_div_exact,
    check_scalar_nodes,
    check_cg_distinct_eigenvalues,
    check_cg_one_reduction_matches_cg,
    check_tail_lengths,
    check_cg_store_then_load,
    check_special_values,
    check_invalid_programs,
    check_dot_closed_forms,
    check_nrm2_closed_forms,
    check_nrm2_scaling,
    check_dot_error_bound,
]
