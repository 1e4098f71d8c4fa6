// Program validation, canonicalisation and lowering (host only).
#include <cmath>

#include "host.h"

#include <cstdio>
#include <cstring>

namespace salt {

static const char* op_name(int op) {
  static const char* names[] = {"VEC",   "SCAL", "ADD",   "SUB", "MUL", "SMUL",
                                "NEG",   "STORE", "DOT",  "SUMSQ", "DIV", "DSCAL"};
  return op >= 0 && op < 12 ? names[op] : "?";
}

salt_status analyse(const salt_insn* prog, int nprog, int nvecs, int nscal, Analysis* out,
                    std::string* err, int ndscal) {
  char buf[160];
  auto fail = [&](salt_status st, const char* msg) {
    if (err) *err = msg;
    return st;
  };
  if (!prog) return fail(SALT_ERR_ARG, "program pointer is NULL");
  if (nprog < 1 || nprog > kMaxProg) {
    snprintf(buf, sizeof buf, "program length %d outside 1..%d", nprog, kMaxProg);
    return fail(SALT_ERR_ARG, buf);
  }
  if (nvecs < 0 || nvecs > kMaxVecs || nscal < 0 || nscal > kMaxScals || ndscal < 0 ||
      ndscal > kMaxDscals)
    return fail(SALT_ERR_ARG, "operand counts outside 0..8");
  Analysis a;
  char stack[kMaxProg + 1];  // 'v' vector, 's' scalar
  int sp = 0, outputs = 0;
  for (int pc = 0; pc < nprog; ++pc) {
    const int op = prog[pc].op, arg = prog[pc].arg;
    auto bad = [&](const char* why) {
      snprintf(buf, sizeof buf, "node %d (%s %d): %s", pc, op_name(op), arg, why);
      return fail(SALT_ERR_PROGRAM, buf);
    };
    switch (op) {
      case OP_VEC:
        if (arg >= nvecs) return bad("vector operand index out of range");
        a.used_vecs |= 1u << arg;
        stack[sp++] = 'v';
        break;
      case OP_SCAL:
        if (arg >= nscal) return bad("scalar operand index out of range");
        a.used_scals |= 1u << arg;
        stack[sp++] = 's';
        break;
      case OP_DSCAL:
        if (arg >= ndscal) return bad("device scalar index out of range");
        a.used_dscals |= 1u << arg;
        a.scalar_nodes = true;
        stack[sp++] = 's';
        break;
      case OP_ADD:
      case OP_SUB:
      case OP_MUL:
      case OP_DIV:
        if (sp < 2) return bad("needs two operands");
        if (stack[sp - 1] != stack[sp - 2]) return bad("operands must be two vectors or two scalars");
        if (stack[sp - 1] == 's') a.scalar_nodes = true;
        --sp;  // the result keeps the operands' type
        break;
      case OP_DOT:
        if (sp < 2) return bad("needs two operands");
        if (stack[sp - 1] != 'v' || stack[sp - 2] != 'v') return bad("operands must be vectors");
        sp -= 2;
        ++a.nred;
        ++outputs;
        break;
      case OP_SMUL:
        if (sp < 2) return bad("needs two operands");
        if (stack[sp - 1] != 'v' || stack[sp - 2] != 's')
          return bad("needs a scalar below a vector");
        sp -= 2;
        stack[sp++] = 'v';
        break;
      case OP_NEG:
        if (sp < 1) return bad("needs an operand");
        if (stack[sp - 1] == 's') a.scalar_nodes = true;
        break;
      case OP_STORE:
      case OP_SUMSQ:
        if (sp < 1) return bad("needs an operand");
        if (stack[sp - 1] != 'v') return bad("operand must be a vector");
        if (op == OP_STORE) {
          if (arg >= nvecs) return bad("vector operand index out of range");
          a.used_vecs |= 1u << arg;
          a.stored_vecs |= 1u << arg;
        } else {
          ++a.nred;
        }
        --sp;
        ++outputs;
        break;
      default:
        return bad("unknown opcode");
    }
    if (sp > kMaxStack) return bad("stack deeper than 8");
    if (sp > a.max_depth) a.max_depth = sp;
    if (a.nred > kMaxReds) return bad("more than 4 reductions");
  }
  if (sp != 0) {
    snprintf(buf, sizeof buf, "%d value(s) left on the stack at the end", sp);
    return fail(SALT_ERR_PROGRAM, buf);
  }
  if (outputs == 0) return fail(SALT_ERR_PROGRAM, "program has no STORE, DOT or SUMSQ");
  if (out) *out = a;
  return SALT_OK;
}

void canonicalise(const salt_insn* prog, int nprog, Canonical* c) {
  int vmap[kMaxVecs], smap[kMaxScals];
  for (int k = 0; k < kMaxVecs; ++k) vmap[k] = -1;
  for (int k = 0; k < kMaxScals; ++k) smap[k] = -1;
  Canonical r;
  uint32_t seen = 0;
  for (int pc = 0; pc < nprog; ++pc) {
    const int op = prog[pc].op, arg = prog[pc].arg;
    int carg = 0;
    if (op == OP_VEC || op == OP_STORE) {
      if (vmap[arg] < 0) {
        vmap[arg] = r.nvec;
        r.vec_user[r.nvec++] = arg;
      }
      carg = vmap[arg];
      if (op == OP_VEC && !((seen >> carg) & 1u)) r.load_mask |= 1u << carg;
      seen |= 1u << carg;
      if (op == OP_STORE) r.store_mask |= 1u << carg;
    } else if (op == OP_SCAL) {
      if (smap[arg] < 0) {
        smap[arg] = r.nscal;
        r.scal_user[r.nscal++] = arg;
      }
      carg = smap[arg];
    }
    if (op == OP_DOT || op == OP_SUMSQ) ++r.nred;
    r.code[r.len++] = pack(op, carg);
  }
  *c = r;
}

namespace {
struct ShapeCode {
  int len;
  int code[kMaxProg];
};
#define SALT_SHAPE_CODE(name, ...) {Prog_##name::len, {__VA_ARGS__}},
const ShapeCode kShapeCodes[NUM_SHAPES] = {SALT_SHAPE_LIST(SALT_SHAPE_CODE)};
#undef SALT_SHAPE_CODE
}  // namespace

int find_shape(const Canonical& c) {
  for (int s = 0; s < NUM_SHAPES; ++s) {
    const ShapeCode& sc = kShapeCodes[s];
    if (sc.len != c.len) continue;
    bool eq = true;
    for (int i = 0; i < c.len && eq; ++i) eq = sc.code[i] == c.code[i];
    if (eq) return s;
  }
  return -1;
}

bool lower(const Canonical& c, RegInsn* code, int* len) {
  // Symbolic stack: each entry names the register holding its value (an
  // operand register 0..7 as long as the value is an unmodified operand, or
  // the depth register 8 + d), or a scalar index.
  struct Ent {
    bool scalar;
    int reg;
  };
  Ent st[kMaxStack + 1];
  int sp = 0, n = 0, r = 0;
  auto emit = [&](uint8_t op, int dst, int a, int b) {
    if (n >= kMaxRegCode) return false;
    code[n++] = RegInsn{op, (uint8_t)dst, (uint8_t)a, (uint8_t)b};
    return true;
  };
  for (int pc = 0; pc < c.len; ++pc) {
    const int op = c.code[pc] / 16, arg = c.code[pc] % 16;
    switch (op) {
      case OP_VEC: st[sp++] = {false, arg}; break;
      case OP_SCAL: st[sp++] = {true, arg}; break;
      case OP_ADD:
      case OP_SUB:
      case OP_MUL:
      case OP_DIV: {
        const Ent b = st[--sp], a = st[--sp];
        const uint8_t io = op == OP_ADD ? I_ADD : op == OP_SUB ? I_SUB : op == OP_MUL ? I_MUL : I_DIV;
        if (!emit(io, 8 + sp, a.reg, b.reg)) return false;
        st[sp] = {false, 8 + sp};
        ++sp;
        break;
      }
      case OP_SMUL: {
        const Ent v = st[--sp], s = st[--sp];
        if (!emit(I_SMUL, 8 + sp, v.reg, s.reg)) return false;
        st[sp] = {false, 8 + sp};
        ++sp;
        break;
      }
      case OP_NEG: {
        const Ent a = st[--sp];
        if (!emit(I_NEG, 8 + sp, a.reg, 0)) return false;
        st[sp] = {false, 8 + sp};
        ++sp;
        break;
      }
      case OP_STORE: {
        const Ent a = st[--sp];
        // Entries still on the stack that alias operand `arg` must keep the
        // old value: copy them to their depth register first.
        for (int d = 0; d < sp; ++d) {
          if (!st[d].scalar && st[d].reg == arg) {
            if (!emit(I_COPY, 8 + d, arg, 0)) return false;
            st[d].reg = 8 + d;
          }
        }
        if (a.reg != arg && !emit(I_COPY, arg, a.reg, 0)) return false;
        break;
      }
      case OP_DOT: {
        const Ent b = st[--sp], a = st[--sp];
        if (!emit(I_DOT, r++, a.reg, b.reg)) return false;
        break;
      }
      case OP_SUMSQ: {
        const Ent a = st[--sp];
        if (!emit(I_SUMSQ, r++, a.reg, a.reg)) return false;
        break;
      }
    }
  }
  *len = n;
  return true;
}

// ------------------------------------------------- scalar subexpressions --

salt_status hoist_scalars(const salt_insn* prog, int nprog, int nscal, Hoisted* h, std::string* err) {
  Hoisted r;
  // Per stack entry, the tokens of its subtree (bit pc).  A scalar subtree
  // need not be contiguous: a statement (VEC k SUMSQ, VEC k STORE j) may sit
  // between its tokens, above its partial values on the stack.
  uint32_t st[kMaxProg + 1];
  int sp = 0;
  uint32_t skip = 0;       // tokens of hoisted occurrences
  int slot_at[kMaxProg];   // hoisted slot whose subtree has its root at pc, or -1
  for (int pc = 0; pc < nprog; ++pc) slot_at[pc] = -1;
  auto same = [&](uint32_t ma, uint32_t mb) {  // equal token sequences
    int i = 0, j = 0;
    for (;;) {
      while (i < nprog && !((ma >> i) & 1u)) ++i;
      while (j < nprog && !((mb >> j) & 1u)) ++j;
      if (i >= nprog || j >= nprog) return i >= nprog && j >= nprog;
      if (prog[i].op != prog[j].op || prog[i].arg != prog[j].arg) return false;
      ++i;
      ++j;
    }
  };
  for (int pc = 0; pc < nprog; ++pc) {
    const uint32_t bit = 1u << pc;
    switch (prog[pc].op) {
      case OP_VEC:
      case OP_SCAL:
      case OP_DSCAL: st[sp++] = bit; break;
      case OP_NEG: st[sp - 1] |= bit; break;
      case OP_STORE:
      case OP_SUMSQ: --sp; break;
      case OP_DOT: sp -= 2; break;
      case OP_SMUL: {
        const uint32_t mv = st[--sp], ms = st[--sp];
        int root = -1;  // last token of the scalar operand
        for (int t = 0; t < nprog; ++t)
          if ((ms >> t) & 1u) root = t;
        const bool bare = (ms & (ms - 1)) == 0 && prog[root].op == OP_SCAL;
        if (!bare) {
          int j = -1;
          for (int q = 0; q < r.nhoist && j < 0; ++q)
            if (same(r.mask[q], ms)) j = q;
          if (j < 0) {
            if (nscal + r.nhoist >= kMaxScals) {
              if (err) *err = "more than 8 scalar slots after hoisting the scalar subexpressions";
              return SALT_ERR_PROGRAM;
            }
            j = r.nhoist++;
            r.mask[j] = ms;
            for (int t = 0; t < nprog; ++t)
              if (((ms >> t) & 1u) && prog[t].op == OP_DSCAL) r.device = true;
          }
          skip |= ms;
          slot_at[root] = j;
        }
        st[sp++] = ms | mv | bit;
        break;
      }
      default: {  // ADD SUB MUL DIV, on two vectors or two scalars
        const uint32_t mb = st[--sp];
        st[sp - 1] |= mb | bit;
        break;
      }
    }
  }
  for (int pc = 0; pc < nprog; ++pc) {
    if (slot_at[pc] >= 0) {
      r.prog[r.nprog++] = salt_insn{(uint8_t)OP_SCAL, (uint8_t)(nscal + slot_at[pc])};
    } else if (!((skip >> pc) & 1u)) {
      r.prog[r.nprog++] = prog[pc];
    }
  }
  r.nscal = nscal + r.nhoist;
  *h = r;
  return SALT_OK;
}

template <typename T>
static double host_scalar_value(const salt_insn* prog, const Hoisted& h, int j, const double* scalars,
                                const double* dvals) {
  T st[kMaxProg + 1];
  int sp = 0;
  for (int pc = 0; pc < kMaxProg; ++pc) {
    if (!((h.mask[j] >> pc) & 1u)) continue;
    const int op = prog[pc].op;
    if (op == OP_SCAL) {
      st[sp++] = (T)scalars[prog[pc].arg];
    } else if (op == OP_DSCAL) {
      st[sp++] = (T)(dvals ? dvals[prog[pc].arg] : 0.0);
    } else if (op == OP_NEG) {
      st[sp - 1] = -st[sp - 1];
    } else {
      const T a = st[sp - 2], b = st[sp - 1];
      T v;
      if (op == OP_ADD) v = a + b;
      else if (op == OP_SUB) v = a - b;
      else if (op == OP_MUL) v = a * b;
      else v = a / b;
      st[sp - 2] = v;
      --sp;
    }
  }
  return (double)st[0];
}

double host_scalar_value_f32(const salt_insn* prog, const Hoisted& h, int j, const double* scalars,
                             const double* dvals) {
  return host_scalar_value<float>(prog, h, j, scalars, dvals);
}
double host_scalar_value_f64(const salt_insn* prog, const Hoisted& h, int j, const double* scalars,
                             const double* dvals) {
  return host_scalar_value<double>(prog, h, j, scalars, dvals);
}

bool build_scalar_code(const salt_insn* prog, const Hoisted& h, const Canonical& c, int user_nscal,
                       const double* scalars, const double* const* dscal, ScalarCode* out) {
  ScalarCode sc;
  memset(&sc, 0, sizeof sc);
  for (int k = 0; k < user_nscal && k < kMaxScals; ++k) sc.cval[k] = scalars ? scalars[k] : 0.0;
  for (int k = 0; k < kMaxDscals; ++k) sc.ds[k] = dscal ? dscal[k] : nullptr;
  int n = 0;
  for (int k = 0; k < c.nscal; ++k) {
    const int j = c.scal_user[k] - user_nscal;
    if (j < 0) continue;  // a user scalar, passed by value
    for (int pc = 0; pc < kMaxProg; ++pc) {
      if (!((h.mask[j] >> pc) & 1u)) continue;
      const int op = prog[pc].op, arg = prog[pc].arg;
      const int sop = op == OP_SCAL ? S_SC : op == OP_DSCAL ? S_DS : op == OP_ADD ? S_ADD
                    : op == OP_SUB ? S_SUB : op == OP_MUL ? S_MUL : op == OP_DIV ? S_DIV : S_NEG;
      if (n >= kMaxScalarCode) return false;
      sc.code[n++] = (uint8_t)(sop * 16 + (sop == S_SC || sop == S_DS ? arg : 0));
    }
    if (n >= kMaxScalarCode) return false;
    sc.code[n++] = (uint8_t)(S_OUT * 16 + k);
  }
  sc.len = n;
  *out = sc;
  return true;
}

bool exact_pow2(double s, int* e) {
  if (s == 0.0 || !std::isfinite(s)) return false;
  int ex = 0;
  const double m = std::frexp(s, &ex);  // s = m 2^ex, 0.5 <= |m| < 1
  if (std::fabs(m) != 0.5) return false;
  ex -= 1;
  if (ex < -1022 || ex > 1023) return false;
  *e = ex;
  return true;
}

Pow2Info pow2_info(const double* sc, int nscal) {
  Pow2Info p{};
  for (int k = 0; k < nscal && k < kMaxScals; ++k) {
    int e = 0;
    if (sc && exact_pow2(sc[k], &e)) {
      p.mask |= 1u << k;
      p.exp[k] = (int16_t)e;
    }
  }
  return p;
}

// Which node pairs the kernels take as one scaled add (Prog::scaled_add /
// scaled_add_load), pinned at compile time.
namespace {
constexpr int V(int k) { return pack(OP_VEC, k); }
constexpr int S(int k) { return pack(OP_SCAL, k); }
constexpr int ST(int k) { return pack(OP_STORE, k); }
constexpr int ADD = pack(OP_ADD, 0), SUB = pack(OP_SUB, 0), MUL = pack(OP_MUL, 0), SMUL = pack(OP_SMUL, 0),
              NEG = pack(OP_NEG, 0);
// e = alpha*a + beta*b - c o d: only beta*b is added at once (alpha*a is not
// followed by an add).
using ProgE = Prog<S(0), V(0), SMUL, S(1), V(1), SMUL, ADD, V(2), V(3), MUL, SUB, ST(4)>;
static_assert(!ProgE::scaled_add(2) && !ProgE::scaled_add_load(2), "alpha*a");
static_assert(ProgE::scaled_add(5) && ProgE::scaled_add_slot(5) == 1, "+ beta*b");
// r - alpha*q, then r + beta*p
using ProgCg = Prog<V(0), S(0), V(1), SMUL, SUB, ST(0), V(0), S(1), V(2), SMUL, ADD, ST(2)>;
static_assert(ProgCg::scaled_add(3) && ProgCg::scaled_add_slot(3) == 0, "r - alpha*q");
static_assert(ProgCg::scaled_add(9) && ProgCg::scaled_add_slot(9) == 1, "r + beta*p");
// s*v - w, the next load subtracted
using ProgSvw = Prog<S(0), V(0), SMUL, V(1), SUB, ST(2)>;
static_assert(ProgSvw::scaled_add_load(2) && !ProgSvw::scaled_add(2) && ProgSvw::scaled_add_slot(2) == 0, "s*v - w");
// a scale computed from two slots, or negated, is not a by-value slot
using ProgProd = Prog<V(0), S(0), S(1), MUL, V(1), SMUL, ADD, ST(2)>;
static_assert(ProgProd::producer(5, 1) == 3 && !ProgProd::scaled_add(5), "(s0*s1)*v");
using ProgNeg = Prog<V(0), S(0), NEG, V(1), SMUL, ADD, ST(2)>;
static_assert(ProgNeg::producer(4, 1) == 2 && !ProgNeg::scaled_add(4), "(-s0)*v");
// x*v + w with x a vector is a plain MUL, never a scaled add
using ProgVv = Prog<V(0), V(1), MUL, V(2), ADD, ST(3)>;
static_assert(!ProgVv::scaled_add_load(2), "a o b + c");
// v must be an operand as loaded: not a computed value, not one stored before
using ProgSum = Prog<V(0), S(0), V(1), V(2), ADD, SMUL, ADD, ST(3)>;
static_assert(ProgSum::producer(5, 2) == 4 && !ProgSum::scaled_add(5), "s*(b+c)");
using ProgStored = Prog<V(0), V(1), ADD, ST(1), V(2), S(0), V(1), SMUL, ADD, ST(2)>;
static_assert(!ProgStored::scaled_add(7) && ProgStored::stored_before(7, 1), "s*b after b is stored");
static_assert(ProgE::any_scaled_add() && !ProgVv::any_scaled_add(), "any");
}  // namespace

}  // namespace salt
