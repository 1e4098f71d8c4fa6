// Compile-time expression programs: the GPU form of the paper's expression
// templates (Section 2, Figure 1; Section 4.2, Listing 1).
//
// A program is a postfix sequence of opcodes packed as op * 16 + arg into a
// template parameter pack.  Everything the paper's node classes expose as
// types and per-node methods -- which operands are loaded, which are stored,
// the stack depth at each node, how many reductions there are -- is derived
// here by constexpr functions, so the kernel body that walks the program is
// fully resolved at compile time: every stack slot and operand lives in a
// register, exactly as the paper's Storage / TemporaryStorage composites do.
#pragma once

namespace salt {

enum : int {
  OP_VEC = 0,
  OP_SCAL = 1,
  OP_ADD = 2,
  OP_SUB = 3,
  OP_MUL = 4,
  OP_SMUL = 5,
  OP_NEG = 6,
  OP_STORE = 7,
  OP_DOT = 8,
  OP_SUMSQ = 9,
  OP_DIV = 10,   // elementwise a / b (two scalars: a scalar node, hoisted)
  OP_DSCAL = 11  // scalar read from device memory (hoisted, never in a kernel program)
};

constexpr int kMaxProg = 32;
constexpr int kMaxVecs = 8;
constexpr int kMaxScals = 8;
constexpr int kMaxStack = 8;
constexpr int kMaxReds = 4;
constexpr int kMaxDscals = 8;

__host__ __device__ constexpr int pack(int op, int arg) { return op * 16 + arg; }

// Stack effect of one opcode.
__host__ __device__ constexpr int stack_delta(int op) {
  return op == OP_VEC || op == OP_SCAL || op == OP_DSCAL ? 1
       : op == OP_NEG ? 0
       : op == OP_STORE || op == OP_SUMSQ ? -1
       : op == OP_DOT ? -2
       : -1;  // ADD SUB MUL DIV SMUL
}

template <int... C>
struct Prog {
  static constexpr int len = sizeof...(C);
  __host__ __device__ static constexpr int at(int i) {
    const int c[] = {C..., 0};
    return c[i];
  }
  __host__ __device__ static constexpr int op(int i) { return at(i) / 16; }
  __host__ __device__ static constexpr int arg(int i) { return at(i) % 16; }
  // Stack depth before node i.
  __host__ __device__ static constexpr int depth_before(int i) {
    int d = 0;
    for (int k = 0; k < i; ++k) d += stack_delta(op(k));
    return d;
  }
  // Index of the reduction result produced by node i (DOT / SUMSQ).
  __host__ __device__ static constexpr int red_index(int i) {
    int r = 0;
    for (int k = 0; k < i; ++k) r += (op(k) == OP_DOT || op(k) == OP_SUMSQ) ? 1 : 0;
    return r;
  }
  __host__ __device__ static constexpr int nred() { return red_index(len); }
  // The stack slot node k writes its result to, or -1 (STORE, DOT, SUMSQ
  // only pop).
  __host__ __device__ static constexpr int writes_slot(int k) {
    return op(k) == OP_VEC || op(k) == OP_SCAL || op(k) == OP_DSCAL ? depth_before(k)
         : op(k) == OP_NEG ? depth_before(k) - 1
         : op(k) == OP_STORE || op(k) == OP_DOT || op(k) == OP_SUMSQ ? -1
         : depth_before(k) - 2;  // ADD SUB MUL DIV SMUL
  }
  // The node whose result stack slot `slot` holds when node i runs (the slot
  // is live there): the last node k < i that wrote that slot.
  __host__ __device__ static constexpr int producer(int i, int slot) {
    int p = -1;
    for (int k = 0; k < i; ++k)
      if (writes_slot(k) == slot) p = k;
    return p;
  }
  // Operand a is stored by a node before node i.
  __host__ __device__ static constexpr bool stored_before(int i, int a) {
    for (int k = 0; k < i; ++k)
      if (op(k) == OP_STORE && arg(k) == a) return true;
    return false;
  }
  // Node i is a scalar-times-vector s*v with s a by-value scalar slot (a SCAL
  // token) and v an operand as loaded (a VEC token of an operand not stored
  // before node i), so both are known before the element's nodes run.
  __host__ __device__ static constexpr bool scaled_vec(int i) {
    if (i >= len || op(i) != OP_SMUL) return false;
    const int d = depth_before(i);
    const int ks = producer(i, d - 2), kv = producer(i, d - 1);
    return ks >= 0 && op(ks) == OP_SCAL && kv >= 0 && op(kv) == OP_VEC && !stored_before(i, arg(kv));
  }
  // A scaled_vec node whose result is at once added to, or subtracted from,
  // the value below it (node i + 1 is ADD or SUB): X + s*v, X - s*v.
  __host__ __device__ static constexpr bool scaled_add(int i) {
    return scaled_vec(i) && depth_before(i) >= 3 && (op(i + 1) == OP_ADD || op(i + 1) == OP_SUB);
  }
  // A scaled_vec node whose result is at once added to, or has subtracted
  // from it, the next vector load (nodes i + 1, i + 2: VEC, ADD / SUB):
  // s*v + w, s*v - w.
  __host__ __device__ static constexpr bool scaled_add_load(int i) {
    return scaled_vec(i) && i + 2 < len && op(i + 1) == OP_VEC && (op(i + 2) == OP_ADD || op(i + 2) == OP_SUB);
  }
  // The scalar slot and the vector operand of a scaled_vec node i.
  __host__ __device__ static constexpr int scaled_add_slot(int i) { return arg(producer(i, depth_before(i) - 2)); }
  __host__ __device__ static constexpr int scaled_add_vec(int i) { return arg(producer(i, depth_before(i) - 1)); }
  // Some node of the program is a scaled add.
  __host__ __device__ static constexpr bool any_scaled_add() {
    for (int i = 0; i < len; ++i)
      if (scaled_add(i) || scaled_add_load(i)) return true;
    return false;
  }
  // Vector operands whose first reference is a read: loaded from memory.
  __host__ __device__ static constexpr unsigned load_mask() {
    unsigned seen = 0, m = 0;
    for (int k = 0; k < len; ++k) {
      const int o = op(k), a = arg(k);
      if (o == OP_VEC && !((seen >> a) & 1u)) m |= 1u << a;
      if (o == OP_VEC || o == OP_STORE) seen |= 1u << a;
    }
    return m;
  }
  // Vector operands assigned by a STORE: written back to memory.
  __host__ __device__ static constexpr unsigned store_mask() {
    unsigned m = 0;
    for (int k = 0; k < len; ++k)
      if (op(k) == OP_STORE) m |= 1u << arg(k);
    return m;
  }
  __host__ __device__ static constexpr int nvec() {
    int n = 0;
    for (int k = 0; k < len; ++k)
      if ((op(k) == OP_VEC || op(k) == OP_STORE) && arg(k) + 1 > n) n = arg(k) + 1;
    return n;
  }
  __host__ __device__ static constexpr int nscal() {
    int n = 0;
    for (int k = 0; k < len; ++k)
      if (op(k) == OP_SCAL && arg(k) + 1 > n) n = arg(k) + 1;
    return n;
  }
  __host__ __device__ static constexpr int nloads() {
    int c = 0;
    for (int s = 0; s < kMaxVecs; ++s) c += (load_mask() >> s) & 1u;
    return c;
  }
  __host__ __device__ static constexpr int nstores() {
    int c = 0;
    for (int s = 0; s < kMaxVecs; ++s) c += (store_mask() >> s) & 1u;
    return c;
  }
};

}  // namespace salt
