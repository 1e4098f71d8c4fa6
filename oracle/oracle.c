/*
 * Oracle for the SALT hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, unfused CPU restatement of what the paper's expression
 * templates compute.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library; the product
 * path never does.  It shares no code, header or constant with the CUDA
 * library.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (contraction must stay off: every node is one correctly rounded IEEE
 * operation, exactly as written in the expression).
 *
 * Semantics followed, one node at a time (no fusion, no reordering):
 *  - Section 2 and Figure 1: an expression such as d = a + (b - c) is a tree
 *    whose inner nodes are elementwise operations; the Store node at the root
 *    assigns the tree's value to the destination vector.  Here the tree is
 *    given in postfix order; each node becomes one full loop over all n
 *    elements into a freshly allocated temporary, the way a non-template
 *    vector library would evaluate it (the "individual loops" that Section 2
 *    says expression templates fuse away).
 *  - Section 4.2 (Listing 2): the tail elements get the same scalar operation
 *    as the vector body, so the result is a function of the element only.
 *  - Section 4.2: init / load_once compute, once per loop, what does not
 *    depend on the element (the TemporaryStorage).  Scalar subexpressions --
 *    ADD, SUB, MUL, DIV, NEG of two scalars, scalar operands given by value
 *    (SCAL) or living in device memory (DSCAL, here passed in by value) --
 *    are such loop invariants; each is one operation rounded to the
 *    program's dtype, like a vector node.
 *  - Section 2 (lazy evaluation in dot product and norm) and Section 5
 *    (xDOT, xSCAL, xAXPY): reductions are plain sums of elementwise products,
 *    accumulated here sequentially in index order in FP64.
 *
 * Precision: an FP32 program performs every elementwise node in FP32
 * (round to nearest even, no FMA), an FP64 program in FP64.  Scalars arrive
 * as doubles and an FP32 program rounds each one to float once.  Reductions
 * always accumulate in FP64 (FP32 values widened first, so FP32 products are
 * exact).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Node kinds of the postfix program (the oracle's own numbering). */
enum {
  OR_VEC = 1,   /* push vector operand k            */
  OR_SCAL = 2,  /* push scalar operand k            */
  OR_ADD = 3,   /* a + b                            */
  OR_SUB = 4,   /* a - b                            */
  OR_MUL = 5,   /* a * b (elementwise)              */
  OR_SMUL = 6,  /* s * v (scalar times vector)      */
  OR_NEG = 7,   /* -v                               */
  OR_STORE = 8, /* assign top of stack to vector k  */
  OR_DOT = 9,   /* sum_i a_i * b_i                  */
  OR_SUMSQ = 10, /* sum_i a_i * a_i                  */
  OR_DIV = 11,   /* a / b (elementwise, or two scalars) */
  OR_DSCAL = 12  /* push device-resident scalar k    */
};

/* Error codes of oracle_eval_*: 0 success. */
enum { OR_OK = 0, OR_BAD_PROGRAM = 1, OR_NOMEM = 2 };

#define OR_MAX_STACK 64

/* ---------------------------------------------------------------- FP64 -- */

typedef struct {
  int is_vec;  /* 1: vector temporary, 0: scalar */
  double s;    /* scalar value                   */
  double* v;   /* owned temporary of n elements  */
} item64;

static void free_stack64(item64* st, int sp) {
  for (int i = 0; i < sp; ++i) free(st[i].v);
}

int oracle_eval_f64(const int32_t* ops, const int32_t* args, int32_t nprog, int64_t n,
                    double* const* vecs, int32_t nvecs, const double* scal, int32_t nscal,
                    const double* dscal, int32_t ndscal, double* red) {
  item64 st[OR_MAX_STACK];
  int sp = 0, nred = 0;
  size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(double);
  for (int pc = 0; pc < nprog; ++pc) {
    int op = ops[pc], k = args[pc];
    if (op == OR_VEC) {
      if (k < 0 || k >= nvecs || sp >= OR_MAX_STACK) goto bad;
      double* t = (double*)malloc(bytes);
      if (!t) goto nomem;
      for (int64_t i = 0; i < n; ++i) t[i] = vecs[k][i];
      st[sp].is_vec = 1; st[sp].v = t; st[sp].s = 0; ++sp;
    } else if (op == OR_SCAL) {
      if (k < 0 || k >= nscal || sp >= OR_MAX_STACK) goto bad;
      st[sp].is_vec = 0; st[sp].v = NULL; st[sp].s = scal[k]; ++sp;
    } else if (op == OR_DSCAL) {
      if (k < 0 || k >= ndscal || sp >= OR_MAX_STACK) goto bad;
      st[sp].is_vec = 0; st[sp].v = NULL; st[sp].s = dscal[k]; ++sp;
    } else if ((op == OR_ADD || op == OR_SUB || op == OR_MUL || op == OR_DIV) && sp >= 2 &&
               !st[sp - 2].is_vec && !st[sp - 1].is_vec) {
      /* scalar node: one FP64 operation */
      double a = st[sp - 2].s, b = st[sp - 1].s, r;
      if (op == OR_ADD) r = a + b;
      else if (op == OR_SUB) r = a - b;
      else if (op == OR_MUL) r = a * b;
      else r = a / b;
      --sp;
      st[sp - 1].s = r;
    } else if (op == OR_ADD || op == OR_SUB || op == OR_MUL || op == OR_DIV) {
      if (sp < 2 || !st[sp - 2].is_vec || !st[sp - 1].is_vec) goto bad;
      double* a = st[sp - 2].v;
      double* b = st[sp - 1].v;
      double* t = (double*)malloc(bytes);
      if (!t) goto nomem;
      if (op == OR_ADD) for (int64_t i = 0; i < n; ++i) t[i] = a[i] + b[i];
      if (op == OR_SUB) for (int64_t i = 0; i < n; ++i) t[i] = a[i] - b[i];
      if (op == OR_MUL) for (int64_t i = 0; i < n; ++i) t[i] = a[i] * b[i];
      if (op == OR_DIV) for (int64_t i = 0; i < n; ++i) t[i] = a[i] / b[i];
      free(a); free(b);
      sp -= 2;
      st[sp].is_vec = 1; st[sp].v = t; ++sp;
    } else if (op == OR_SMUL) {
      if (sp < 2 || st[sp - 2].is_vec || !st[sp - 1].is_vec) goto bad;
      double s = st[sp - 2].s;
      double* v = st[sp - 1].v;
      double* t = (double*)malloc(bytes);
      if (!t) goto nomem;
      for (int64_t i = 0; i < n; ++i) t[i] = s * v[i];
      free(v);
      sp -= 2;
      st[sp].is_vec = 1; st[sp].v = t; ++sp;
    } else if (op == OR_NEG) {
      if (sp < 1) goto bad;
      if (!st[sp - 1].is_vec) {
        st[sp - 1].s = -st[sp - 1].s;
        continue;
      }
      double* v = st[sp - 1].v;
      for (int64_t i = 0; i < n; ++i) v[i] = -v[i];
    } else if (op == OR_STORE) {
      if (k < 0 || k >= nvecs || sp < 1 || !st[sp - 1].is_vec) goto bad;
      double* v = st[sp - 1].v;
      for (int64_t i = 0; i < n; ++i) vecs[k][i] = v[i];
      free(v);
      --sp;
    } else if (op == OR_DOT) {
      if (sp < 2 || !st[sp - 2].is_vec || !st[sp - 1].is_vec) goto bad;
      double* a = st[sp - 2].v;
      double* b = st[sp - 1].v;
      double acc = 0.0;
      for (int64_t i = 0; i < n; ++i) acc = acc + a[i] * b[i];
      red[nred++] = acc;
      free(a); free(b);
      sp -= 2;
    } else if (op == OR_SUMSQ) {
      if (sp < 1 || !st[sp - 1].is_vec) goto bad;
      double* a = st[sp - 1].v;
      double acc = 0.0;
      for (int64_t i = 0; i < n; ++i) acc = acc + a[i] * a[i];
      red[nred++] = acc;
      free(a);
      --sp;
    } else {
      goto bad;
    }
  }
  if (sp != 0) goto bad;
  return OR_OK;
bad:
  free_stack64(st, sp);
  return OR_BAD_PROGRAM;
nomem:
  free_stack64(st, sp);
  return OR_NOMEM;
}

/* ---------------------------------------------------------------- FP32 -- */

typedef struct {
  int is_vec;
  float s;
  float* v;
} item32;

static void free_stack32(item32* st, int sp) {
  for (int i = 0; i < sp; ++i) free(st[i].v);
}

int oracle_eval_f32(const int32_t* ops, const int32_t* args, int32_t nprog, int64_t n,
                    float* const* vecs, int32_t nvecs, const double* scal, int32_t nscal,
                    const double* dscal, int32_t ndscal, double* red) {
  item32 st[OR_MAX_STACK];
  int sp = 0, nred = 0;
  size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(float);
  for (int pc = 0; pc < nprog; ++pc) {
    int op = ops[pc], k = args[pc];
    if (op == OR_VEC) {
      if (k < 0 || k >= nvecs || sp >= OR_MAX_STACK) goto bad;
      float* t = (float*)malloc(bytes);
      if (!t) goto nomem;
      for (int64_t i = 0; i < n; ++i) t[i] = vecs[k][i];
      st[sp].is_vec = 1; st[sp].v = t; st[sp].s = 0; ++sp;
    } else if (op == OR_SCAL) {
      if (k < 0 || k >= nscal || sp >= OR_MAX_STACK) goto bad;
      st[sp].is_vec = 0; st[sp].v = NULL; st[sp].s = (float)scal[k]; ++sp;
    } else if (op == OR_DSCAL) {
      if (k < 0 || k >= ndscal || sp >= OR_MAX_STACK) goto bad;
      st[sp].is_vec = 0; st[sp].v = NULL; st[sp].s = (float)dscal[k]; ++sp;
    } else if ((op == OR_ADD || op == OR_SUB || op == OR_MUL || op == OR_DIV) && sp >= 2 &&
               !st[sp - 2].is_vec && !st[sp - 1].is_vec) {
      /* scalar node: one FP32 operation */
      float a = st[sp - 2].s, b = st[sp - 1].s, r;
      if (op == OR_ADD) r = a + b;
      else if (op == OR_SUB) r = a - b;
      else if (op == OR_MUL) r = a * b;
      else r = a / b;
      --sp;
      st[sp - 1].s = r;
    } else if (op == OR_ADD || op == OR_SUB || op == OR_MUL || op == OR_DIV) {
      if (sp < 2 || !st[sp - 2].is_vec || !st[sp - 1].is_vec) goto bad;
      float* a = st[sp - 2].v;
      float* b = st[sp - 1].v;
      float* t = (float*)malloc(bytes);
      if (!t) goto nomem;
      if (op == OR_ADD) for (int64_t i = 0; i < n; ++i) t[i] = a[i] + b[i];
      if (op == OR_SUB) for (int64_t i = 0; i < n; ++i) t[i] = a[i] - b[i];
      if (op == OR_MUL) for (int64_t i = 0; i < n; ++i) t[i] = a[i] * b[i];
      if (op == OR_DIV) for (int64_t i = 0; i < n; ++i) t[i] = a[i] / b[i];
      free(a); free(b);
      sp -= 2;
      st[sp].is_vec = 1; st[sp].v = t; ++sp;
    } else if (op == OR_SMUL) {
      if (sp < 2 || st[sp - 2].is_vec || !st[sp - 1].is_vec) goto bad;
      float s = st[sp - 2].s;
      float* v = st[sp - 1].v;
      float* t = (float*)malloc(bytes);
      if (!t) goto nomem;
      for (int64_t i = 0; i < n; ++i) t[i] = s * v[i];
      free(v);
      sp -= 2;
      st[sp].is_vec = 1; st[sp].v = t; ++sp;
    } else if (op == OR_NEG) {
      if (sp < 1) goto bad;
      if (!st[sp - 1].is_vec) {
        st[sp - 1].s = -st[sp - 1].s;
        continue;
      }
      float* v = st[sp - 1].v;
      for (int64_t i = 0; i < n; ++i) v[i] = -v[i];
    } else if (op == OR_STORE) {
      if (k < 0 || k >= nvecs || sp < 1 || !st[sp - 1].is_vec) goto bad;
      float* v = st[sp - 1].v;
      for (int64_t i = 0; i < n; ++i) vecs[k][i] = v[i];
      free(v);
      --sp;
    } else if (op == OR_DOT) {
      if (sp < 2 || !st[sp - 2].is_vec || !st[sp - 1].is_vec) goto bad;
      float* a = st[sp - 2].v;
      float* b = st[sp - 1].v;
      double acc = 0.0;
      for (int64_t i = 0; i < n; ++i) acc = acc + (double)a[i] * (double)b[i];
      red[nred++] = acc;
      free(a); free(b);
      sp -= 2;
    } else if (op == OR_SUMSQ) {
      if (sp < 1 || !st[sp - 1].is_vec) goto bad;
      float* a = st[sp - 1].v;
      double acc = 0.0;
      for (int64_t i = 0; i < n; ++i) acc = acc + (double)a[i] * (double)a[i];
      red[nred++] = acc;
      free(a);
      --sp;
    } else {
      goto bad;
    }
  }
  if (sp != 0) goto bad;
  return OR_OK;
bad:
  free_stack32(st, sp);
  return OR_BAD_PROGRAM;
nomem:
  free_stack32(st, sp);
  return OR_NOMEM;
}

/* ------------------------------------------------------------ BLAS-1 ---- */

/* xDOT of Section 5: sum_i x_i y_i, sequential FP64. */
double oracle_dot_f64(int64_t n, const double* x, const double* y) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) acc = acc + x[i] * y[i];
  return acc;
}

/* FP32 inputs widened to FP64; every product is then exact. */
double oracle_dot_f32(int64_t n, const float* x, const float* y) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) acc = acc + (double)x[i] * (double)y[i];
  return acc;
}

/* The norm of Section 2, sqrt(sum_i x_i^2).  FP32 inputs: widened squares
 * can neither overflow nor underflow in FP64, so a plain sum suffices. */
double oracle_nrm2_f32(int64_t n, const float* x) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) acc = acc + (double)x[i] * (double)x[i];
  return sqrt(acc);
}

/* FP64 inputs: two passes.  Pass 1 finds m = max |x_i|; pass 2 sums the
 * squares of x_i * 2^-e with e = ilogb(m), a power-of-two scaling that is
 * exact for every element that stays normal, then the root is scaled back
 * by 2^e.  This keeps the sum away from overflow and underflow. */
double oracle_nrm2_f64(int64_t n, const double* x) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double a = fabs(x[i]);
    if (isnan(a)) return a;
    if (a > m) m = a;
  }
  if (m == 0.0 || isinf(m)) return m;
  int e = ilogb(m);
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t = ldexp(x[i], -e);
    acc = acc + t * t;
  }
  return ldexp(sqrt(acc), e);
}
