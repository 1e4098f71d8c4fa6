"""Oracle for the SALT hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product.

* ``oracle.c`` (compiled to ``liboracle.so`` by :func:`build`) evaluates a
  postfix expression program one node at a time, unfused, with every node a
  separate loop into a temporary (Section 2, Figure 1 of the paper: the tree
  for ``d = a + (b - c)``; Section 4.2, Listing 2: the tail elements get the
  same scalar operation as the body).  It also holds the plain BLAS-1 dot and
  norm of Section 5 (xDOT) and Section 2 (dot product / norm as the places
  where lazy evaluation happens).
* :mod:`oracle.exact` holds exactly rounded references (``math.fsum`` over
  error-free product splits, ``fractions.Fraction``) that the reductions are
  judged against, because a sequential FP64 sum is itself off by up to
  ``gamma_n * sum|x_i y_i|``.

Programs are lists of ``(name, arg)`` pairs with names ``VEC, SCAL, DSCAL,
ADD, SUB, MUL, DIV, SMUL, NEG, STORE, DOT, SUMSQ`` (arg used by VEC, SCAL,
DSCAL, STORE).  ADD, SUB, MUL, DIV and NEG act elementwise on vectors or on
two scalars (a loop-invariant scalar node, Section 4.2 init/load_once);
DSCAL is a scalar that the product reads from device memory -- here it is
simply passed in by value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# The oracle's own node numbering (matches the enum in oracle.c).
_CODES = {"VEC": 1, "SCAL": 2, "ADD": 3, "SUB": 4, "MUL": 5, "SMUL": 6,
          "NEG": 7, "STORE": 8, "DOT": 9, "SUMSQ": 10, "DIV": 11, "DSCAL": 12}

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(src: str = _SRC, out: str = _LIB, extra: list[str] | None = None) -> str:
    """Compile ``oracle.c`` with FMA contraction off (required: gcc contracts
    ``a*b + c`` by default on aarch64)."""
    cmd = ["gcc", *CFLAGS, *(extra or []), "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _load(path: str = _LIB) -> ctypes.CDLL:
    if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        build(out=path)
    lib = ctypes.CDLL(path)
    i32p = ctypes.POINTER(ctypes.c_int32)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    for name in ("oracle_eval_f64", "oracle_eval_f32"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(vp),
                      ctypes.c_int32, dp, ctypes.c_int32, dp, ctypes.c_int32, dp]
    for name in ("oracle_dot_f64", "oracle_dot_f32"):
        f = getattr(lib, name)
        f.restype = ctypes.c_double
        f.argtypes = [ctypes.c_int64, vp, vp]
    for name in ("oracle_nrm2_f64", "oracle_nrm2_f32"):
        f = getattr(lib, name)
        f.restype = ctypes.c_double
        f.argtypes = [ctypes.c_int64, vp]
    return lib


_lib_cache: dict[str, ctypes.CDLL] = {}


def lib(path: str = _LIB) -> ctypes.CDLL:
    if path not in _lib_cache:
        _lib_cache[path] = _load(path)
    return _lib_cache[path]


class OracleProgramError(ValueError):
    pass


def _dtype_of(vecs):
    kinds = {v.dtype for v in vecs}
    if len(kinds) != 1:
        raise TypeError("all vectors of one program must share a dtype")
    dt = kinds.pop()
    if dt not in (np.float32, np.float64):
        raise TypeError(f"unsupported dtype {dt}")
    return dt


def eval_program(prog, vecs, scalars=(), n=None, path: str = _LIB, dscalars=()):
    """Evaluate ``prog`` node by node.  ``vecs`` are C-contiguous numpy
    arrays (all float32 or all float64) that STORE overwrites in place;
    ``scalars`` feed SCAL nodes and ``dscalars`` DSCAL nodes.
    Returns the list of reduction results (DOT/SUMSQ, in program order)."""
    dt = _dtype_of(vecs)
    for v in vecs:
        if not v.flags.c_contiguous:
            raise ValueError("vectors must be contiguous")
    if n is None:
        n = min(v.shape[0] for v in vecs) if vecs else 0
    ops = (ctypes.c_int32 * max(len(prog), 1))(*[_CODES[o] for o, _ in prog])
    args = (ctypes.c_int32 * max(len(prog), 1))(*[int(a) for _, a in prog])
    ptrs = (ctypes.c_void_p * max(len(vecs), 1))(*[v.ctypes.data for v in vecs])
    sc = (ctypes.c_double * max(len(scalars), 1))(*[float(s) for s in scalars])
    dsc = (ctypes.c_double * max(len(dscalars), 1))(*[float(s) for s in dscalars])
    nred = sum(1 for o, _ in prog if o in ("DOT", "SUMSQ"))
    red = (ctypes.c_double * max(nred, 1))()
    fn = lib(path).oracle_eval_f64 if dt == np.float64 else lib(path).oracle_eval_f32
    rc = fn(ops, args, len(prog), int(n), ptrs, len(vecs), sc, len(scalars), dsc, len(dscalars),
            red)
    if rc == 1:
        raise OracleProgramError("invalid program")
    if rc != 0:
        raise MemoryError("oracle out of memory")
    return [red[i] for i in range(nred)]


def dot(x: np.ndarray, y: np.ndarray, path: str = _LIB) -> float:
    """Plain sequential FP64 dot product (FP32 inputs widened first)."""
    if x.dtype != y.dtype or x.shape != y.shape:
        raise TypeError("dot operands must match")
    x = np.ascontiguousarray(x)
    y = np.ascontiguousarray(y)
    f = lib(path).oracle_dot_f64 if x.dtype == np.float64 else lib(path).oracle_dot_f32
    return f(x.shape[0], x.ctypes.data, y.ctypes.data)


def nrm2(x: np.ndarray, path: str = _LIB) -> float:
    """Euclidean norm: FP64 sum of widened squares for FP32 input; two-pass
    power-of-two scaled sum for FP64 input."""
    x = np.ascontiguousarray(x)
    f = lib(path).oracle_nrm2_f64 if x.dtype == np.float64 else lib(path).oracle_nrm2_f32
    return f(x.shape[0], x.ctypes.data)


# Named programs of the paper's examples and the BLAS-1 set, in postfix.
# Figure 1: d = a + (b - c)  -> the subtraction node is evaluated first.
PROG_D = [("VEC", 0), ("VEC", 1), ("VEC", 2), ("SUB", 0), ("ADD", 0), ("STORE", 3)]
# Section 5 xAXPY generalised: y = alpha*x + beta*y.
PROG_AXPBY = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("SCAL", 1), ("VEC", 1), ("SMUL", 0),
              ("ADD", 0), ("STORE", 1)]
# e = alpha*a + beta*b - c o d, C++ precedence / left associativity.
PROG_E = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("SCAL", 1), ("VEC", 1), ("SMUL", 0),
          ("ADD", 0), ("VEC", 2), ("VEC", 3), ("MUL", 0), ("SUB", 0), ("STORE", 4)]
# CG-style update: r <- r - alpha*q ; rho = r.r ; p <- r + beta*p
PROG_CG = [("VEC", 0), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("SUB", 0), ("STORE", 0),
           ("VEC", 0), ("SUMSQ", 0),
           ("VEC", 0), ("SCAL", 1), ("VEC", 2), ("SMUL", 0), ("ADD", 0), ("STORE", 2)]
# Section 5 out-of-place scaling (sCOPY + sSCAL as one loop): y = alpha*x.
PROG_SCALE = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)]
PROG_DOT = [("VEC", 0), ("VEC", 1), ("DOT", 0)]
