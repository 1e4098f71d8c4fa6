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
