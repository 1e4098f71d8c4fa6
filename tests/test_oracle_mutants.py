"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each mutant is a copy of oracle.c with one plausible mistake -- a swapped
operand, a dropped term or element, a wrong index or sign, a missing
widening, FMA contraction left on -- compiled to a scratch library.  The pin
checks of ``oracle_pins`` must reject every one of them."""
import os
import platform

import pytest

import oracle
import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, original text, occurrence index, replacement)
MUTANTS = [
    ("f64_sub_swapped", "t[i] = a[i] - b[i];", 0, "t[i] = b[i] - a[i];"),
    ("f32_sub_swapped", "t[i] = a[i] - b[i];", 1, "t[i] = b[i] - a[i];"),
    ("f64_add_drops_last", "for (int64_t i = 0; i < n; ++i) t[i] = a[i] + b[i];", 0,
     "for (int64_t i = 0; i + 1 < n; ++i) t[i] = a[i] + b[i]; if (n > 0) t[n - 1] = 0;"),
    ("f32_wrong_scalar", "st[sp].s = (float)scal[k];", 0, "st[sp].s = (float)scal[0];"),
    ("f64_store_skips_first", "for (int64_t i = 0; i < n; ++i) vecs[k][i] = v[i];", 0,
     "for (int64_t i = 1; i < n; ++i) vecs[k][i] = v[i];"),
    ("f32_load_reversed", "for (int64_t i = 0; i < n; ++i) t[i] = vecs[k][i];", 1,
     "for (int64_t i = 0; i < n; ++i) t[i] = vecs[k][n - 1 - i];"),
    ("f64_mul_is_add", "t[i] = a[i] * b[i];", 0, "t[i] = a[i] + b[i];"),
    ("f32_smul_wrong_operand", "t[i] = s * v[i];", 1, "t[i] = s * s;"),
    ("f64_neg_noop", "v[i] = -v[i];", 0, "v[i] = v[i];"),
    ("f32_neg_noop", "v[i] = -v[i];", 1, "v[i] = v[i];"),
    ("f64_dot_program_uses_a_twice", "acc = acc + a[i] * b[i];", 0, "acc = acc + a[i] * a[i];"),
    ("f32_sumsq_wrong_index", "acc = acc + (double)a[i] * (double)a[i];", 0,
     "acc = acc + (double)a[i] * (double)a[0];"),
    ("dot_f64_drops_last", "for (int64_t i = 0; i < n; ++i) acc = acc + x[i] * y[i];", 0,
     "for (int64_t i = 0; i + 1 < n; ++i) acc = acc + x[i] * y[i];"),
    ("dot_f32_not_widened", "acc = acc + (double)x[i] * (double)y[i];", 0,
     "acc = acc + (double)(x[i] * y[i]);"),
    ("nrm2_f64_scale_sign", "return ldexp(sqrt(acc), e);", 0, "return ldexp(sqrt(acc), -e);"),
    ("nrm2_f64_no_scaling", "double t = ldexp(x[i], -e);", 0, "double t = x[i]; e = 0;"),
    ("nrm2_f32_no_sqrt", "  return sqrt(acc);\n}", 0, "  return acc;\n}"),
    ("f64_div_swapped", "t[i] = a[i] / b[i];", 0, "t[i] = b[i] / a[i];"),
    ("f32_div_is_mul", "t[i] = a[i] / b[i];", 1, "t[i] = a[i] * b[i];"),
    ("f64_scalar_sub_swapped", "else if (op == OR_SUB) r = a - b;", 0, "else if (op == OR_SUB) r = b - a;"),
    ("f32_scalar_div_inverted", "else r = a / b;", 1, "else r = b / a;"),
    ("f32_scalar_add_wrong_operand", "if (op == OR_ADD) r = a + b;", 1, "if (op == OR_ADD) r = a + a;"),
    ("f64_dscal_wrong_index", "st[sp].s = dscal[k];", 0, "st[sp].s = dscal[0];"),
    ("f32_dscal_reads_scal", "st[sp].s = (float)dscal[k];", 0, "st[sp].s = (float)scal[k];"),
    ("f64_scalar_neg_noop", "st[sp - 1].s = -st[sp - 1].s;", 0, "st[sp - 1].s = st[sp - 1].s;"),
    ("f32_scalar_neg_noop", "st[sp - 1].s = -st[sp - 1].s;", 1, "st[sp - 1].s = st[sp - 1].s;"),
]


def _mutate(text, old, occ, new):
    parts = text.split(old)
    assert len(parts) >= occ + 2, f"anchor {old!r} occurrence {occ} missing"
    return old.join(parts[: occ + 1]) + new + old.join(parts[occ + 1:])


def _pins_fail(path):
    for check in oracle_pins.ALL_CHECKS:
        try:
            check(path)
        except Exception:
            return check.__name__
    return None


@pytest.mark.parametrize("name,old,occ,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, occ, new):
    text = open(SRC).read()
    src = tmp_path / f"{name}.c"
    src.write_text(_mutate(text, old, occ, new))
    lib = oracle.build(str(src), str(tmp_path / f"lib{name}.so"))
    assert _pins_fail(lib) is not None, f"mutant {name} passed every pin"


def test_unfused_oracle_is_immune_to_fma_contraction(tmp_path):
    """Every node of the oracle writes its own temporary array, so even a
    build with FMA contraction on (gcc's default on aarch64) has nothing to
    contract between nodes: all pins still pass.  The product build keeps
    contraction off all the same."""
    import subprocess
    extra = ["-ffp-contract=fast"]
    if platform.machine() in ("x86_64", "AMD64"):
        extra.append("-mfma")
    cflags = [f for f in oracle.CFLAGS if f != "-ffp-contract=off"]
    out = str(tmp_path / "libfma.so")
    subprocess.run(["gcc", *cflags, *extra, "-o", out, SRC, "-lm"], check=True)
    assert _pins_fail(out) is None


@pytest.mark.parametrize("mistake", ["alpha_sign", "beta_inverted", "s_uses_new_r"])
def test_one_reduction_cg_mistakes_are_caught(monkeypatch, mistake):
    """Plausible mistakes in the one-reduction CG recurrence (a sign in the
    alpha denominator, beta upside down, the s update reading the updated
    residual) must fail its pins."""
    import numpy as np
    op = oracle_pins
    step = list(op.CGC_STEP)
    if mistake == "s_uses_new_r":
        # the x and r updates before the p and s updates
        step = [("VEC", 4), ("DSCAL", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 1)] + \
            op._CGC_TAIL[:12] + \
            [("VEC", 0), ("VEC", 4), ("MUL", 0), ("DSCAL", 0), ("VEC", 2), ("SMUL", 0), ("ADD", 0), ("STORE", 2)] + \
            op._CGC_TAIL[12:]

    def mutant(evalp, d, b, x0, iters):
        n = d.shape[0]
        dt = d.dtype.type
        p, s, r = np.zeros(n, d.dtype), np.zeros(n, d.dtype), np.zeros(n, d.dtype)
        x = x0.copy()
        vecs = [d, p, s, x, r, b]
        hist = list(evalp(op.CGC_START, vecs, []))
        alpha = None
        for k in range(iters):
            g, dl = dt(hist[2 * k]), dt(hist[2 * k + 1])
            if k == 0:
                alpha = g / dl
                out = evalp(op.CGC_FIRST, vecs, [0.0, float(alpha)])
            else:
                beta = g / dt(hist[2 * k - 2])
                if mistake == "beta_inverted":
                    beta = dt(hist[2 * k - 2]) / g
                den = dl + beta * g / alpha if mistake == "alpha_sign" else dl - beta * g / alpha
                alpha = g / den
                out = evalp(step, vecs, [float(beta), float(alpha)])
            hist.extend(out)
        return x, hist

    monkeypatch.setattr(op, "cg_diagonal_one_reduction", mutant)
    caught = 0
    for check in (op.check_cg_distinct_eigenvalues, op.check_cg_one_reduction_matches_cg):
        try:
            check(oracle._LIB)
        except AssertionError:
            caught += 1
    assert caught >= 1, mistake
