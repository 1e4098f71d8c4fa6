"""Exactly rounded references for judging reductions -- TEST INFRASTRUCTURE.

A sequential FP64 dot product is off by up to ``gamma_n * sum|x_i y_i|``
(Higham, *Accuracy and Stability of Numerical Algorithms*, 2nd ed., Eq. 3.5),
which for the large vectors of the BLAS-1 sweep exceeds the 1e-13 relative
tolerance the GPU results are held to.  So tolerances are measured against
the exact value, rounded once:

* Products are made error-free first.  FP32 x FP32 products are exact in
  FP64 (24 + 24 bits <= 53).  FP64 x FP64 products use Dekker's split
  (Dekker 1971, "A floating-point technique for extending the available
  precision"): x = xh + xl with both halves 26 bits wide, so the four partial
  products are exact in FP64.
* The error-free terms are summed exactly with Rump, Ogita and Oishi's
  error-free vector extraction (SIAM J. Sci. Comput. 31(1), 2008, "Accurate
  floating-point summation part I"): with sigma a power of two large enough,
  ``q = (sigma + p) - sigma`` is p rounded to a grid whose every partial sum
  is exact, and ``p - q`` is exact.  Repeating on the remainders until they
  vanish splits the sum into a few exactly computed level sums, which
  ``math.fsum`` (correctly rounded) then combines.

Tiny cases use ``fractions.Fraction``.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

_SPLITTER = 134217729.0  # 2**27 + 1, Dekker's splitting constant for p = 53


def _split(a: np.ndarray):
    """Dekker split of FP64 values into two 26-bit halves (no FMA used)."""
    c = _SPLITTER * a
    hi = c - (c - a)
    lo = a - hi
    return hi, lo


def _level_sums(p: np.ndarray) -> list[float]:
    """Exact decomposition of sum(p) into a short list of FP64 values."""
    p = np.asarray(p, dtype=np.float64).ravel().copy()
    if p.size == 0:
        return [0.0]
    if not np.all(np.isfinite(p)):
        return [float(np.sum(p))]
    out: list[float] = []
    n = p.size
    log2n = max(1, math.ceil(math.log2(n + 1)))
    while True:
        m = float(np.max(np.abs(p)))
        if m == 0.0:
            break
        # sigma = 2^(ceil(log2 n) + ceil(log2 m) + 1): every q below is a
        # multiple of ulp(sigma)/2 and |sum q| < sigma, so the sum is exact.
        e = math.frexp(m)[1]  # m < 2^e
        sigma = math.ldexp(1.0, e + log2n + 1)
        q = (sigma + p) - sigma
        out.append(float(np.sum(q)))
        p = p - q
    return out or [0.0]


def exact_sum(p: np.ndarray) -> float:
    """Correctly rounded sum of FP64 values."""
    return math.fsum(_level_sums(p))


def _exact_products(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    if x.dtype == np.float32 and y.dtype == np.float32:
        return x.astype(np.float64) * y.astype(np.float64)
    x = x.astype(np.float64)
    y = y.astype(np.float64)
    xh, xl = _split(x)
    yh, yl = _split(y)
    return np.concatenate([xh * yh, xh * yl, xl * yh, xl * yl])


def exact_dot(x: np.ndarray, y: np.ndarray) -> float:
    """sum_i x_i*y_i rounded once to FP64."""
    return exact_sum(_exact_products(np.asarray(x), np.asarray(y)))


def exact_sumsq(x: np.ndarray) -> float:
    return exact_dot(x, x)


def abs_dot(x: np.ndarray, y: np.ndarray) -> float:
    """sum_i |x_i*y_i| (the condition scale of a dot product), exactly rounded.
    Taken as the exact dot of |x| and |y|: the absolute values of Dekker's
    partial products would over-count, since the two halves of a split
    value may differ in sign."""
    return exact_dot(np.abs(np.asarray(x)), np.abs(np.asarray(y)))


class FixedPointDot:
    """Exact dot product of two long vectors whose elements are integers
    times one power of two, fed in pieces (so that n = 2^28 and beyond needs
    no more host memory than one piece).

    The counter-based inputs are such vectors: an FP64 value ``2 (h >> 11)
    2^-53 - 1`` is ``a 2^-52`` with an integer |a| <= 2^52, an FP32 value
    ``2 (h >> 40) 2^-24 - 1`` is ``a 2^-23`` with |a| <= 2^23.  Each integer
    is split as ``a = a1 2^26 + a0`` (``a1 = floor(a / 2^26)``,
    0 <= a0 < 2^26), so every partial product of the four ``ai bj`` has
    magnitude below 2^53 and a sum of 2^9 of them stays below 2^63: int64
    arithmetic is exact.  Row sums are then combined in Python integers;
    ``sum_i a_i b_i = S11 2^52 + (S10 + S01) 2^26 + S00`` exactly, and the
    result is rounded once (Python's int -> float conversion is correctly
    rounded) and scaled by ``2^-(fa + fb)``.  The sum of |a_i b_i| -- the
    condition scale -- is formed the same way from |a|, |b|."""

    ROW = 512

    def __init__(self, frac_bits_x: int, frac_bits_y: int):
        self.fx, self.fy = frac_bits_x, frac_bits_y
        self.s = 0
        self.sabs = 0

    @staticmethod
    def _integers(v: np.ndarray, frac_bits: int) -> np.ndarray:
        a = np.ldexp(np.asarray(v, dtype=np.float64), frac_bits)
        ai = a.astype(np.int64)
        if not np.array_equal(ai.astype(np.float64), a) or np.any(np.abs(ai) > 2 ** 52):
            raise ValueError("values are not integers times 2^-frac_bits with |integer| <= 2^52")
        return ai

    @classmethod
    def _int_dot(cls, a: np.ndarray, b: np.ndarray) -> int:
        pad = (-a.size) % cls.ROW
        if pad:
            a = np.concatenate([a, np.zeros(pad, np.int64)])
            b = np.concatenate([b, np.zeros(pad, np.int64)])
        a1, a0 = a >> 26, a & ((1 << 26) - 1)
        b1, b0 = b >> 26, b & ((1 << 26) - 1)
        tot = 0
        for u, v, shift in ((a1, b1, 52), (a1, b0, 26), (a0, b1, 26), (a0, b0, 0)):
            rows = (u * v).reshape(-1, cls.ROW).sum(axis=1)
            tot += sum(int(r) for r in rows) << shift
        return tot

    def add(self, x: np.ndarray, y: np.ndarray) -> None:
        a = self._integers(x, self.fx)
        b = self._integers(y, self.fy)
        if a.size != b.size:
            raise ValueError("pieces of unequal length")
        self.s += self._int_dot(a, b)
        self.sabs += self._int_dot(np.abs(a), np.abs(b))

    @classmethod
    def combine(cls, parts: list["FixedPointDot"]) -> "FixedPointDot":
        """One accumulator holding the sums of several (same scales), e.g.
        pieces accumulated on separate threads."""
        out = cls(parts[0].fx, parts[0].fy)
        for f in parts:
            if (f.fx, f.fy) != (out.fx, out.fy):
                raise ValueError("accumulators of different scales")
            out.s += f.s
            out.sabs += f.sabs
        return out

    def _round(self, v: int) -> float:
        return math.ldexp(float(v), -(self.fx + self.fy))

    def value(self) -> float:
        """sum x_i y_i of every piece added, rounded once to FP64."""
        return self._round(self.s)

    def abs_value(self) -> float:
        """sum |x_i y_i|, rounded once to FP64."""
        return self._round(self.sabs)


def exact_nrm2(x: np.ndarray) -> float:
    """sqrt of the exactly rounded sum of squares (within 1 ulp of the true
    norm).  For FP64 input the vector is first scaled by a power of two so
    that the squares stay in range; the scaling is exact for normal values."""
    x = np.asarray(x)
    if x.size == 0:
        return 0.0
    if x.dtype == np.float32:
        return math.sqrt(exact_sumsq(x))
    m = float(np.max(np.abs(x)))
    if m == 0.0 or not math.isfinite(m):
        return m
    e = math.frexp(m)[1]
    xs = np.ldexp(x.astype(np.float64), -e)
    return math.ldexp(math.sqrt(exact_sumsq(xs)), e)


def fraction_dot(x, y) -> Fraction:
    """Exact rational dot product (tiny n only)."""
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))


def round_to(fr: Fraction, dtype) -> float:
    """Round an exact rational once to FP64, or to FP32.

    ``float(Fraction)`` is correctly rounded.  Going FP64 -> FP32 afterwards
    is a second rounding, which is innocuous for a single +, - or x of two
    FP32 operands because 53 >= 2*24 + 2 (Figueroa, "When is double rounding
    innocuous?", SIGNUM 1995)."""
    d = float(fr)
    if dtype == np.float32:
        return float(np.float32(d))
    return d


def exact_program(prog, vecs, scalars, dtype, dscalars=()):
    """Per-element evaluation of a postfix program with exact rational
    arithmetic and one rounding per node to ``dtype`` (finite values only;
    every DIV denominator nonzero).  Scalar nodes (two scalar operands) are
    rounded like vector nodes; SCAL and DSCAL values are rounded to
    ``dtype`` once.

    Returns (stored vectors as lists of floats keyed by slot, reductions as
    Fractions, and per reduction the exact sum of |terms|, the scale of
    Higham's error bound).  Slow: meant for n up to a few hundred."""
    n = min(len(v) for v in vecs) if vecs else 0
    cur = [[float(t) for t in v] for v in vecs]
    if dtype == np.float32:
        sc = [float(np.float32(s)) for s in scalars]
        dsc = [float(np.float32(s)) for s in dscalars]
    else:
        sc = [float(s) for s in scalars]
        dsc = [float(s) for s in dscalars]
    # reductions: accumulate exactly over elements in order of appearance
    nred = sum(1 for o, _ in prog if o in ("DOT", "SUMSQ"))
    red_exact = [Fraction(0)] * nred
    red_abs = [Fraction(0)] * nred
    for i in range(n):
        stack = []
        r = 0
        for op, k in prog:
            if op == "VEC":
                stack.append(("v", cur[k][i]))
            elif op == "SCAL":
                stack.append(("s", sc[k]))
            elif op == "DSCAL":
                stack.append(("s", dsc[k]))
            elif op in ("ADD", "SUB", "MUL", "DIV"):
                kb, b = stack.pop()
                ka, a = stack.pop()
                fa, fb = Fraction(a), Fraction(b)
                if op == "ADD":
                    ex = fa + fb
                elif op == "SUB":
                    ex = fa - fb
                elif op == "MUL":
                    ex = fa * fb
                else:
                    ex = fa / fb
                kind = "s" if (ka, kb) == ("s", "s") else "v"
                stack.append((kind, round_to(ex, dtype)))
            elif op == "SMUL":
                v = stack.pop()[1]
                s = stack.pop()[1]
                stack.append(("v", round_to(Fraction(s) * Fraction(v), dtype)))
            elif op == "NEG":
                kv, v = stack.pop()
                stack.append((kv, -v))
            elif op == "STORE":
                cur[k][i] = stack.pop()[1]
            elif op == "DOT":
                b = stack.pop()[1]
                a = stack.pop()[1]
                red_exact[r] += Fraction(a) * Fraction(b)
                red_abs[r] += abs(Fraction(a) * Fraction(b))
                r += 1
            elif op == "SUMSQ":
                a = stack.pop()[1]
                red_exact[r] += Fraction(a) * Fraction(a)
                red_abs[r] += Fraction(a) * Fraction(a)
                r += 1
            else:
                raise ValueError(op)
    return cur, red_exact, red_abs


def gamma(n: int, u: float) -> float:
    """Higham's gamma_n = n u / (1 - n u)."""
    return n * u / (1.0 - n * u)
