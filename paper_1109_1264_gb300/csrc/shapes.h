// Programs with a compile-time instantiation (the fast path), in canonical
// form: vector operands numbered in order of first appearance (VEC or
// STORE), scalars likewise.  The host canonicalises a caller's program and
// looks it up here; anything else runs on the generic interpreter kernel.
//
//  D      d = a + (b - c)                     Section 2, Figure 1
//  AXPBY  y = alpha x + beta y                Section 5 xAXPY, generalised
//  AXPBYZ z = alpha x + beta y
//  AXPY   y = alpha x + y                     Section 5 xAXPY
//  E      e = alpha a + beta b - c o d        fused 4-operand expression
//  SCAL   x = alpha x                         Section 5 xSCAL
//  SCALE  y = alpha x                         Section 5 out-of-place scaling
//  COPY   y = x
//  CG     r = r - alpha q; rho = r.r; p = r + beta p   (map + reduce)
//  DOT    sum x_i y_i                         Section 5 xDOT
//  SUMSQ  sum x_i^2
// and two shapes that only single calls take (not the batch kernel), the
// two passes of a conjugate-gradient iteration for a diagonal operator
// A = diag(d) (Hestenes and Stiefel 1952), with their scalars usually
// hoisted device-scalar quotients:
//  CGR0   r = b - d o x; rho = r.r             (start)
//  CGP0   p = r; q = d o p; pq = p.q            (first pass of iteration 0)
//  CGPQ   p = r + beta p; q = d o p; pq = p.q   (first pass of iteration k)
//  CGXR   x = x + alpha p; r = r - alpha q; rho = r.r   (second pass)
#pragma once

#include "prog.cuh"

#define SALT_V(k) ::salt::pack(::salt::OP_VEC, k)
#define SALT_S(k) ::salt::pack(::salt::OP_SCAL, k)
#define SALT_ST(k) ::salt::pack(::salt::OP_STORE, k)
#define SALT_ADD ::salt::pack(::salt::OP_ADD, 0)
#define SALT_SUB ::salt::pack(::salt::OP_SUB, 0)
#define SALT_MUL ::salt::pack(::salt::OP_MUL, 0)
#define SALT_SMUL ::salt::pack(::salt::OP_SMUL, 0)
#define SALT_NEG ::salt::pack(::salt::OP_NEG, 0)
#define SALT_DOT ::salt::pack(::salt::OP_DOT, 0)
#define SALT_SUMSQ ::salt::pack(::salt::OP_SUMSQ, 0)

#define SALT_BATCH_SHAPE_LIST(X)                                                                 \
  X(D, SALT_V(0), SALT_V(1), SALT_V(2), SALT_SUB, SALT_ADD, SALT_ST(3))                          \
  X(AXPBY, SALT_S(0), SALT_V(0), SALT_SMUL, SALT_S(1), SALT_V(1), SALT_SMUL, SALT_ADD, SALT_ST(1)) \
  X(AXPBYZ, SALT_S(0), SALT_V(0), SALT_SMUL, SALT_S(1), SALT_V(1), SALT_SMUL, SALT_ADD, SALT_ST(2)) \
  X(AXPY, SALT_S(0), SALT_V(0), SALT_SMUL, SALT_V(1), SALT_ADD, SALT_ST(1))                      \
  X(E, SALT_S(0), SALT_V(0), SALT_SMUL, SALT_S(1), SALT_V(1), SALT_SMUL, SALT_ADD, SALT_V(2),     \
    SALT_V(3), SALT_MUL, SALT_SUB, SALT_ST(4))                                                    \
  X(SCAL, SALT_S(0), SALT_V(0), SALT_SMUL, SALT_ST(0))                                            \
  X(SCALE, SALT_S(0), SALT_V(0), SALT_SMUL, SALT_ST(1))                                           \
  X(COPY, SALT_V(0), SALT_ST(1))                                                                  \
  X(CG, SALT_V(0), SALT_S(0), SALT_V(1), SALT_SMUL, SALT_SUB, SALT_ST(0), SALT_V(0), SALT_SUMSQ, \
    SALT_V(0), SALT_S(1), SALT_V(2), SALT_SMUL, SALT_ADD, SALT_ST(2))                             \
  X(DOT, SALT_V(0), SALT_V(1), SALT_DOT)                                                          \
  X(SUMSQ, SALT_V(0), SALT_SUMSQ)

#define SALT_SHAPE_LIST(X)                                                                        \
  SALT_BATCH_SHAPE_LIST(X)                                                                        \
  X(CGR0, SALT_V(0), SALT_V(1), SALT_V(2), SALT_MUL, SALT_SUB, SALT_ST(3), SALT_V(3), SALT_SUMSQ) \
  X(CGP0, SALT_V(0), SALT_ST(1), SALT_V(2), SALT_V(1), SALT_MUL, SALT_ST(3), SALT_V(1), SALT_V(3), \
    SALT_DOT)                                                                                     \
  X(CGPQ, SALT_V(0), SALT_S(0), SALT_V(1), SALT_SMUL, SALT_ADD, SALT_ST(1), SALT_V(2), SALT_V(1),  \
    SALT_MUL, SALT_ST(3), SALT_V(1), SALT_V(3), SALT_DOT)                                         \
  X(CGXR, SALT_V(0), SALT_S(0), SALT_V(1), SALT_SMUL, SALT_ADD, SALT_ST(0), SALT_V(2), SALT_S(0),  \
    SALT_V(3), SALT_SMUL, SALT_SUB, SALT_ST(2), SALT_V(2), SALT_SUMSQ)

namespace salt {

#define SALT_COUNT_ENTRY(name, ...) +1
#define SALT_ENUM_ENTRY(name, ...) SHAPE_##name,
enum ShapeId : int { SALT_SHAPE_LIST(SALT_ENUM_ENTRY) NUM_SHAPES };
enum : int { NUM_BATCH_SHAPES = 0 SALT_BATCH_SHAPE_LIST(SALT_COUNT_ENTRY) };
#undef SALT_ENUM_ENTRY
#undef SALT_COUNT_ENTRY

#define SALT_PROG_TYPE(name, ...) using Prog_##name = Prog<__VA_ARGS__>;
SALT_SHAPE_LIST(SALT_PROG_TYPE)
#undef SALT_PROG_TYPE

// Unroll depths and vector widths that are instantiated.
constexpr int kUnrolls[] = {1, 2, 4};
constexpr int kNumUnroll = 3;
constexpr int kVecBytes[] = {16, 32};
constexpr int kNumVB = 2;

}  // namespace salt
