/*
 * salt.h -- C ABI of the SALT fused vector-expression library for GB300
 * (sm_103a).
 *
 * The paper (Progsch, Ineichen, Adelmann, "A New Vectorization Technique for
 * Expression Templates in C++", arXiv:1109.1264) builds, at compile time, an
 * expression tree of vector operations (Section 2, Figure 1: d = a + (b - c)
 * as Store<Vector, ExprAdd<Vector, ExprSub<Vector, Vector>>>) and evaluates
 * it lazily in ONE loop over the elements when it is assigned, or when a dot
 * product or norm consumes it (Section 2).  Section 4 assembles that loop from
 * three parts: a vectorizer (Section 3), loop templates that issue bursts of
 * loads, operations and stores (Section 4.3) and the tree's per-node methods
 * (Section 4.2, Listing 1), selected by an execute function (Section 4.1,
 * Figure 2).  Section 5 benchmarks xDOT, xSCAL, xAXPY and an out-of-place
 * scaling.
 *
 * This library takes the expression tree as a postfix PROGRAM at run time,
 * validates and types it on the host, and runs it as one fused GPU kernel:
 * each operand element is read from HBM once and each result element written
 * once.
 *
 * Conventions for every entry point below:
 *  - Vectors are dense, contiguous (salt_eval_strided: strided),
 *    caller-owned DEVICE memory of the call's dtype, aligned at least to the
 *    element size.  When every operand of a call is 16-byte aligned and
 *    contiguous (cudaMalloc / torch allocations are) the kernels use 128- or
 *    256-bit accesses; otherwise element accesses (the paper's scalar
 *    single_op path, Section 4.2, for the whole range).  Batches and the
 *    plain-mode reductions need 16-byte alignment.  The library never frees
 *    or retains the vectors.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream; results are valid once the caller has
 *    synchronised with it.
 *  - Reduction results are written as double to caller-owned DEVICE memory.
 *  - Argument and program errors are detected on the host and returned before
 *    anything is launched.  CUDA failures return SALT_ERR_CUDA; the text of
 *    the last error of the calling thread is available from
 *    salt_last_error().
 *  - The library owns only small per-(device, stream) workspaces for
 *    reduction partials, created on the first reducing call on that stream
 *    (so make that first call before capturing the stream into a CUDA graph)
 *    and kept until salt_release_workspaces() or process exit.  Calls that
 *    reduce on the SAME stream are ordered; calls on different streams use
 *    different workspaces.
 *  - Environment (read once per process):
 *      SALT_TUNE_CACHE  a tuning-table file (salt_tune_save format) merged
 *                       into the launch-shape table on first use and
 *                       rewritten after every salt_autotune, so tuned shapes
 *                       persist across processes; unreadable files are ignored.
 *      SALT_JIT_CACHE   directory of run-time compiled kernels ("0" or "off":
 *                       none; see salt_jit_cache_dir).
 *      SALT_DEBUG       "1": salt_eval, salt_eval_strided, salt_eval_ex,
 *                       salt_axpby, salt_dot, salt_nrm2 and salt_cg_diag
 *                       synchronise their stream before returning and report
 *                       a failure of their kernels as SALT_ERR_CUDA from the
 *                       call that caused it (otherwise such an error surfaces
 *                       at a later synchronisation).
 *  - n == 0 is valid: nothing is written to vectors and every reduction
 *    result is 0.
 */
#ifndef SALT_H
#define SALT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types. */
typedef enum { SALT_F32 = 0, SALT_F64 = 1 } salt_dtype;

/* Status codes. */
typedef enum {
  SALT_OK = 0,
  SALT_ERR_ARG = 1,      /* bad size, count, NULL pointer, bad flag          */
  SALT_ERR_PROGRAM = 2,  /* malformed or ill-typed program                    */
  SALT_ERR_DTYPE = 3,    /* unknown dtype, or operands of different dtypes    */
  SALT_ERR_ALIGN = 4,    /* a pointer is not aligned as the call requires      */
  SALT_ERR_ALIAS = 5,    /* an output overlaps another operand's memory       */
  SALT_ERR_BUDGET = 6,   /* request larger than a budget or capacity          */
  SALT_ERR_TIMEOUT = 7,  /* a bounded host wait ran out                       */
  SALT_ERR_CUDA = 8,     /* a CUDA runtime call failed                        */
  SALT_ERR_NOTFOUND = 9  /* unknown request / handle                          */
} salt_status;

/* Program opcodes (one byte each).  The program is the expression tree in
 * postfix order (Section 2, Figure 1); evaluation is per element, so every
 * node sees element i of its operands only.
 *   VEC k    push vector operand k (reads element i of vecs[k]; after a
 *            STORE k earlier in the program it reads the stored value)
 *   SCAL k   push scalar operand k (a loop constant: the paper's
 *            load_once/TemporaryStorage, Section 4.2)
 *   DSCAL k  push device scalar k: the double at dscalars[k] in device
 *            memory (salt_eval_ex), read when the kernel starts
 *   ADD      pop b, pop a, push a + b        (ExprAdd, Figure 1)
 *   SUB      pop b, pop a, push a - b        (ExprSub, Figure 1)
 *   MUL      pop b, pop a, push a * b        (elementwise product)
 *   DIV      pop b, pop a, push a / b        (elementwise quotient)
 *   SMUL     pop v (vector), pop s (scalar), push s * v   (xSCAL / xAXPY)
 *   NEG      pop a, push -a
 *   STORE k  pop a, assign it to vector k   (Store root, Figure 1)
 *   DOT      pop b, pop a, accumulate sum_i a_i * b_i into the next result
 *   SUMSQ    pop a, accumulate sum_i a_i * a_i into the next result
 * ADD, SUB, MUL, DIV and NEG take two vectors (one vector for NEG) or two
 * scalars (one scalar): a scalar subexpression such as (DSCAL0 DSCAL1 DIV)
 * does not depend on the element, so, like the paper's init / load_once
 * values (Section 4.2), it is computed once per launch -- on the host when
 * it reads only SCAL operands, else by the kernel before its loop -- and
 * equal subexpressions are computed once.  The scalar slots after this
 * hoisting (SCAL operands plus distinct subexpressions) must not exceed
 * SALT_MAX_SCALS.
 * Every node, scalar nodes included, computes in the program's dtype,
 * round-to-nearest-even, with no fused multiply-add, in exactly this order:
 * elementwise results are bit-identical to evaluating the tree one node at a
 * time.  Scalars (SCAL and DSCAL) are doubles, rounded once to float for an
 * F32 program.  Reductions: see salt_dot. */
typedef enum {
  SALT_OP_VEC = 0,
  SALT_OP_SCAL = 1,
  SALT_OP_ADD = 2,
  SALT_OP_SUB = 3,
  SALT_OP_MUL = 4,
  SALT_OP_SMUL = 5,
  SALT_OP_NEG = 6,
  SALT_OP_STORE = 7,
  SALT_OP_DOT = 8,
  SALT_OP_SUMSQ = 9,
  SALT_OP_DIV = 10,
  SALT_OP_DSCAL = 11
} salt_opcode;

typedef struct {
  uint8_t op;  /* salt_opcode                                   */
  uint8_t arg; /* operand index for VEC / SCAL / DSCAL / STORE, else 0 */
} salt_insn;

#define SALT_MAX_PROG 32  /* instructions per program       */
#define SALT_MAX_VECS 8   /* vector operands per program    */
#define SALT_MAX_SCALS 8  /* scalar operands per program    */
#define SALT_MAX_STACK 8  /* evaluation stack depth         */
#define SALT_MAX_REDS 4   /* DOT / SUMSQ results per program */
#define SALT_MAX_DSCALS 8 /* device scalars per program     */

/* Reduction flags. */
#define SALT_DEFAULT 0
/* F32 only: plain FP32 accumulation and FP32 combination, no compensation
 * (a comparison mode; less accurate). */
#define SALT_PLAIN 1

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t salt_version(void);

/* Text of a status code (static storage). */
const char* salt_status_str(int32_t status);

/* Text of the last error reported on the calling thread ("" if none). */
const char* salt_last_error(void);

/* ---------------------------------------------------------------------------
 * salt_check_program -- host-only validation and typing of a program
 * (no GPU needed).  Checks opcodes, operand indices against nvecs / nscal
 * (DSCAL indices against SALT_MAX_DSCALS; salt_eval_ex checks them against
 * its ndscal), operand types (ADD/SUB/MUL/DIV take two vectors or two
 * scalars, NEG one of either, DOT two vectors, SMUL a scalar below a vector,
 * STORE/SUMSQ a vector), stack depth <= SALT_MAX_STACK, an empty stack at
 * the end, at least one STORE or reduction, <= SALT_MAX_REDS reductions, and
 * <= SALT_MAX_SCALS scalar slots after hoisting.
 * Outputs (any may be NULL):
 *   nred_out      number of DOT/SUMSQ results,
 *   compiled_out  1 if the program (after hoisting its scalar
 *                 subexpressions) has a compile-time instantiation (the
 *                 fast path; the paper's expression templates, Section 2),
 *                 0 if it runs on a run-time compiled instantiation (the
 *                 default, see salt_set_jit) or the generic interpreter.
 * Returns SALT_OK or SALT_ERR_PROGRAM / SALT_ERR_ARG. */
salt_status salt_check_program(const salt_insn* prog, int32_t nprog, int32_t nvecs,
                               int32_t nscal, int32_t* nred_out, int32_t* compiled_out);

/* ---------------------------------------------------------------------------
 * salt_eval -- evaluate a fused expression program over n elements
 * (Section 2 lazy evaluation at the Store root / dot / norm; Section 4 loop).
 *   prog, nprog      the postfix program (host memory, read during the call)
 *   dtype            SALT_F32 or SALT_F64, the type of every vector
 *   n                element count (>= 0)
 *   vecs, nvecs      host array of nvecs device pointers; vecs[k] is operand
 *                    k.  Only operands the program names must be non-NULL.
 *   scalars, nscal   host array of scalar operands (read during the call)
 *   red_out          device array of >= nred doubles receiving the DOT/SUMSQ
 *                    results in program order; may be NULL if nred == 0
 *   stream           cudaStream_t
 * Aliasing: an operand that is stored may be read by the same program only
 * through the same operand index (exact in-place update, e.g. y = a*x + b*y).
 * If a stored operand's memory overlaps any other named operand's memory the
 * call returns SALT_ERR_ALIAS.  Two read-only operands may share memory.
 * Errors: SALT_ERR_ARG, SALT_ERR_PROGRAM, SALT_ERR_DTYPE, SALT_ERR_ALIGN,
 * SALT_ERR_ALIAS (nothing launched), SALT_ERR_CUDA. */
salt_status salt_eval(const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                      void* const* vecs, int32_t nvecs, const double* scalars, int32_t nscal,
                      double* red_out, void* stream);

/* salt_eval with strided operands (BLAS incx semantics): element i of operand
 * k is vecs[k][i * strides[k]]; strides is a host array of nvecs element
 * strides, nonzero for the operands the program names (SALT_ERR_ARG
 * otherwise).  A negative stride walks the vector backwards from vecs[k]:
 * for BLAS's incx < 0 over an array starting at x, pass
 * x + (n - 1) * |incx| and the negative incx.  Elements between the strided
 * positions are never read or written.  Aliasing is judged on the whole
 * address range an operand spans, ((n - 1) * |stride| + 1) elements.
 * Otherwise as salt_eval. */
salt_status salt_eval_strided(const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                              void* const* vecs, const int64_t* strides, int32_t nvecs, const double* scalars,
                              int32_t nscal, double* red_out, void* stream);

/* salt_eval with DEVICE-RESIDENT scalars (and optional strides): the DSCAL k
 * nodes of `prog` read the double at dscalars[k], a host array of ndscal
 * (<= SALT_MAX_DSCALS) device pointers, each 8-byte aligned.  The value is
 * read when the kernel starts, in stream order, so a reduction result that
 * an earlier call on the same stream wrote (a DOT / SUMSQ red_out) can
 * steer this call without the host reading it: e.g. conjugate gradients'
 * alpha = rho / (p . q) as  DSCAL0 DSCAL1 DIV  (Hestenes and Stiefel 1952).
 * A device scalar must not lie in memory the same call writes (a stored
 * vector or red_out): SALT_ERR_ALIAS.  strides may be NULL (contiguous) or
 * as salt_eval_strided.  Not part of the paper, whose scalars are host
 * values; with ndscal == 0 this is salt_eval / salt_eval_strided.
 * Errors as salt_eval. */
salt_status salt_eval_ex(const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                         void* const* vecs, const int64_t* strides, int32_t nvecs, const double* scalars,
                         int32_t nscal, const double* const* dscalars, int32_t ndscal, double* red_out,
                         void* stream);

/* salt_cg_diag -- `iters` conjugate-gradient iterations (Hestenes and
 * Stiefel 1952) for diag(d) x = b, with every scalar kept on the device: two
 * fused launches per iteration on `stream` and no host synchronisation.
 *   pass 1  p = r + beta p;  q = d o p;  pq = p . q     (iteration 0: p = r)
 *   pass 2  x = x + alpha p;  r = r - alpha q;  rho' = r . r
 * with beta = rho_k / rho_{k-1} and alpha = rho_k / pq read as DSCAL
 * quotients (salt_eval_ex) from the previous launches' results.  A start
 * launch computes r = b - d o x and rho_0 = r . r.
 *   d, b        inputs, n elements (d > 0 for an SPD operator)
 *   x           in: the initial guess; out: the iterate
 *   r, p, q     work vectors of n elements (out: residual, direction, d o p)
 *   rho         device array of >= 2 * iters + 1 doubles: rho[0] = rho_0,
 *               rho[2k+1] = (p . q) of iteration k, rho[2k+2] = rho_{k+1}
 *               (the squared residual norms: the convergence history)
 * All vectors are distinct and 16-byte aligned for the vector kernels
 * (otherwise the element-access kernels run).  There is no stopping test:
 * once a residual is exactly zero the next quotients are 0 / 0 (NaN), so
 * choose `iters` from the rho history of a shorter run.  The same
 * computation is available piecewise through salt_eval_ex; this is not
 * part of the paper.  Every call is validated before the first launch.
 * Errors as salt_eval. */
salt_status salt_cg_diag(int32_t dtype, int64_t n, const void* d, const void* b, void* x, void* r, void* p,
                         void* q, int32_t iters, double* rho, void* stream);

/* salt_cg_diag in ONE cooperative launch: the blocks stay resident for all
 * iterations and meet at a grid-wide barrier after each reduction (two per
 * iteration), instead of two kernel launches per iteration -- for small n,
 * where launches dominate.  Same arguments, per-element operations and
 * scalar nodes as salt_cg_diag; the reductions use the same accumulators
 * but another partition of the elements, so rho and the iterates agree with
 * salt_cg_diag to the reductions' tolerance, not bit for bit.  The launch
 * uses at most one block per 1024 elements and never more blocks than can
 * be resident (cudaLaunchCooperativeKernel; SALT_ERR_CUDA if the device
 * cannot).  Barrier waits are bounded (a few seconds): a launch that cannot
 * progress ends with NaN in rho[0] instead of hanging.  Not in the paper. */
salt_status salt_cg_diag_persistent(int32_t dtype, int64_t n, const void* d, const void* b, void* x, void* r,
                                    void* p, void* q, int32_t iters, double* rho, void* stream);

/* Conjugate gradients for diag(d) x = b with ONE reduction phase per
 * iteration (Chronopoulos and Gear's recurrence), in one cooperative launch
 * with one grid barrier per iteration (salt_cg_diag_persistent has two).
 * Each iteration is one pass over the elements:
 *   p = r + beta p,  s = d o r + beta s   (s = A p in exact arithmetic)
 *   x = x + alpha p, r = r - alpha s
 *   gamma = r . r,   delta = (d o r) . r  of the new residual
 * with beta = gamma_k / gamma_{k-1} and alpha_k = gamma_k / (delta_k -
 * beta_k gamma_k / alpha_{k-1}) (alpha_0 = gamma_0 / delta_0), every scalar
 * node computed in the vectors' precision from the totals rounded to it.
 * In exact arithmetic the iterates are those of salt_cg_diag; in floating
 * point they differ by rounding.  It moves 9 vectors per iteration (reads
 * d, r, x, p, s; writes p, s, x, r) against 11 for the two-pass form.
 *   d, b, x, r, p as salt_cg_diag; s the work vector in salt_cg_diag's q slot
 *   rho   device array of >= 2 * iters + 2 doubles: rho[0] = gamma_0 (the
 *         squared residual norm of x's start), rho[1] = delta_0, then
 *         rho[2k+2] = gamma_{k+1}, rho[2k+3] = delta_{k+1}
 * Launch, residency, bounded barriers and errors as salt_cg_diag_persistent.
 * Not in the paper. */
salt_status salt_cg_diag_one_reduction(int32_t dtype, int64_t n, const void* d, const void* b, void* x, void* r,
                                       void* p, void* s, int32_t iters, double* rho, void* stream);

/* salt_cg_diag_auto -- the same CG for diag(d) x = b in whichever of the
 * three forms is fastest for the dtype and size: SALT_CG_TWO_PASS
 * (salt_cg_diag), SALT_CG_PERSISTENT (salt_cg_diag_persistent) or
 * SALT_CG_ONE_REDUCTION (salt_cg_diag_one_reduction), looked up per dtype and
 * n's log2 bucket in a table whose defaults come from measurements on GB300
 * (FP32: the one-reduction form, except 2^19 <= n < 2^22 where the forms tie
 * and the two-pass form is kept; FP64: the one-reduction form below 2^19,
 * the two-pass form from 2^19, where the FP64 pipe bounds the
 * one-reduction pass).  Arguments as the chosen form; rho must hold
 * 2 * iters + 2 doubles (the most any form writes); in every form rho[2k]
 * is the squared residual norm after k iterations, and rho[2k+1] is p.q
 * (two-pass, persistent) or delta (one-reduction).  *form_used (may be
 * NULL) receives the form.  Not in the paper.  Errors as the chosen form. */
#define SALT_CG_TWO_PASS 0
#define SALT_CG_PERSISTENT 1
#define SALT_CG_ONE_REDUCTION 2
salt_status salt_cg_diag_auto(int32_t dtype, int64_t n, const void* d, const void* b, void* x, void* r, void* p,
                              void* q, int32_t iters, double* rho, int32_t* form_used, void* stream);
/* Pins the form salt_cg_diag_auto uses for dtype and n's log2 bucket
 * (form < 0: back to the default) / reports it.  Errors: SALT_ERR_DTYPE,
 * SALT_ERR_ARG. */
salt_status salt_cg_form_set(int32_t dtype, int64_t n, int32_t form);
salt_status salt_cg_form_get(int32_t dtype, int64_t n, int32_t* form);
/* Times the three forms (reps runs each after one warm-up, CUDA events on
 * `stream`) on the caller's vectors, every run starting from x as passed (it
 * is saved to a temporary device buffer and restored, and left as passed at
 * the end); r, p, q and rho are overwritten.  Pins the fastest for dtype and
 * n's bucket and returns it (*best_form) with its milliseconds per run
 * (*best_ms); either may be NULL.  Synchronous; allocates.  Errors as the
 * forms, SALT_ERR_ARG (reps outside [1, 1000]), SALT_ERR_CUDA. */
salt_status salt_cg_autotune(int32_t dtype, int64_t n, const void* d, const void* b, void* x, void* r, void* p,
                             void* q, int32_t iters, double* rho, int32_t reps, int32_t* best_form, double* best_ms,
                             void* stream);

/* Status of the last cooperative CG launch (salt_cg_diag_persistent or
 * salt_cg_diag_one_reduction) on `stream`: synchronises the stream, then
 * returns SALT_OK if every grid barrier of that launch completed, or
 * SALT_ERR_TIMEOUT if one ran out of its poll limit (the launch then ended
 * early with NaN in rho[0]; x, r, p and q hold partial updates).  Reads a
 * word of the stream's reduction workspace (created by the first reducing
 * call on the stream).  Not in the paper.  Errors: SALT_ERR_TIMEOUT,
 * SALT_ERR_CUDA. */
salt_status salt_cg_status(void* stream);

/* Limits of the bounded device waits, for tests that make a wait run out on
 * purpose (all are process-wide and read at each launch):
 *   SALT_WAIT_STAGED      polls thread 0 of a staged-loop block spends on a
 *                         tile's bulk copies before it stops staging and
 *                         computes from direct loads (results unchanged;
 *                         counted by salt_staged_timeouts); 0: give up at
 *                         once.  The copies already issued are still waited
 *                         for, with the full bound, before the block exits.
 *   SALT_WAIT_CG_BARRIER  polls of one grid barrier of the cooperative CG
 *                         launches before it records a timeout (see
 *                         salt_cg_status); 0: give up unless already passed.
 *   SALT_WAIT_SERVE       polls of each wait of the persistent serving
 *                         kernel (salt_serve_config.persistent) before it
 *                         ends its launch; a wait other than the idle wait
 *                         for the next step that runs out fails the server
 *                         (its requests report SALT_ERR_CUDA).
 * Default for all: 2^26 polls (besides the staged wait's one-second timer
 * bound).  polls in [0, 2^32); errors: SALT_ERR_ARG (unknown wait, polls
 * out of range or NULL).  Not in the paper. */
/* Per-block timeline of launches, for finding where a kernel's time goes
 * (launch ramp, tail, cross-block combine).  With a buffer set, every
 * launch of the fused kernels (register-tiled and staged loops) and of the
 * norm kernel whose grid has at most `max_blocks` blocks writes, from
 * thread 0 of block b, SALT_TRACE_WORDS 64-bit words at buf + b *
 * SALT_TRACE_WORDS: [0] the global timer (ns) when the block starts, [1]
 * after its whole tiles, [2] before the cross-block combine, [3] at its end,
 * [4] its SM id, [5] 1 if it performed the final combine.  Each launch
 * overwrites the words of its blocks; zero the buffer between launches to
 * tell how many blocks wrote.  buf: caller-owned device memory, 8-byte
 * aligned; NULL turns tracing off (the default; the kernels then skip it).
 * Process-wide.  Errors: SALT_ERR_ARG, SALT_ERR_ALIGN.  Not in the paper. */
#define SALT_TRACE_WORDS 8
salt_status salt_trace_set(void* buf, int64_t max_blocks);

/* salt_fp64_rate -- the FP64 pipe's issue rate of one instruction kind,
 * measured from registers: every thread of 4 blocks of 256 threads per SM
 * runs 8 independent chains of DFMA (SALT_FP64_FMA), DADD or DMUL, timed
 * with events on `stream` after a warm-up launch; *gops receives G
 * instructions per second.  The measured counterpart of the FP64 peak
 * derived from unit counts and the clock, for the roofline of the FP64
 * shapes (on GB300 DFMA issues faster than DADD and DMUL, which is why the
 * kernels issue every FP64 node as an FMA with an exact product).
 * Synchronizes the stream; about 150 ms.  Not in the paper.  Errors:
 * SALT_ERR_ARG, SALT_ERR_CUDA. */
#define SALT_FP64_FMA 0
#define SALT_FP64_ADD 1
#define SALT_FP64_MUL 2
salt_status salt_fp64_rate(int32_t op, double* gops, void* stream);

#define SALT_WAIT_STAGED 1
#define SALT_WAIT_CG_BARRIER 2
#define SALT_WAIT_SERVE 3
#define SALT_WAIT_DEFAULT_POLLS 67108864
salt_status salt_set_wait_limit(int32_t which, int64_t polls);
salt_status salt_get_wait_limit(int32_t which, int64_t* polls);

/* salt_explain -- host only (no GPU): the program the kernels evaluate for
 * `prog`, after its scalar subexpressions are hoisted, with the values of
 * the scalar slots.  Not part of the paper; an inspection aid.
 *   dtype              SALT_F32 or SALT_F64 (the precision of scalar nodes)
 *   scalars, nscal     by-value scalars, as for salt_eval
 *   dvals, ndscal      host values standing in for the device scalars
 *   out, nout          receives the hoisted program (<= nprog insns; SCAL k
 *                      with k >= nscal names a hoisted subexpression)
 *   slots, nslots      receives the slot values (<= SALT_MAX_SCALS): the
 *                      nscal user scalars, then each hoisted subexpression
 *                      computed on the host, one operation per node in dtype
 *   compiled_out       (may be NULL) as salt_check_program
 * For a program without DSCAL these are exactly the program and scalars
 * salt_eval launches.  Errors: as salt_check_program, SALT_ERR_DTYPE. */
salt_status salt_explain(const salt_insn* prog, int32_t nprog, int32_t dtype, int32_t nvecs, const double* scalars,
                         int32_t nscal, const double* dvals, int32_t ndscal, salt_insn* out, int32_t* nout,
                         double* slots, int32_t* nslots, int32_t* compiled_out);

/* ---------------------------------------------------------------------------
 * salt_axpby -- y <- alpha*x + beta*y (Section 5's xAXPY generalised; xSCAL
 * when x is not used is salt_eval's SCAL VEC SMUL STORE).  Same as
 * salt_eval of  SCAL0 VEC0 SMUL SCAL1 VEC1 SMUL ADD STORE1  with
 * vecs = {x, y}: beta*y is always computed (no beta == 0 shortcut, so NaN
 * in y propagates).  x and y must not overlap unless x == y.
 * Errors as salt_eval. */
salt_status salt_axpby(int32_t dtype, int64_t n, double alpha, const void* x, double beta,
                       void* y, void* stream);

/* ---------------------------------------------------------------------------
 * salt_dot -- *out = sum_i x_i * y_i  (Section 5, xDOT; Section 2: the dot
 * product is where the tree is evaluated).
 *   out    device pointer to one double
 *   flags  SALT_DEFAULT or SALT_PLAIN
 * F64: per-thread FP64 fused multiply-add accumulation, FP64 warp / block /
 *      cross-block combination in a fixed order (deterministic for given n).
 * F32 (default): per-thread FP32 TwoProduct + TwoSum compensated
 *      accumulation (Ogita, Rump and Oishi 2005, "Accurate sum and dot
 *      product", Dot2), each thread's (sum, correction) pair widened to FP64,
 *      FP64 combination.  SALT_PLAIN: FP32 accumulation and combination.
 * The summation order differs from a sequential loop (as the paper's own
 * unrolled loop differs: per-unroll accumulators combined by reduction(),
 * Section 4.2); results are reproducible run to run for the same n. */
salt_status salt_dot(int32_t dtype, int64_t n, const void* x, const void* y, double* out,
                     int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * salt_nrm2 -- *out = sqrt(sum_i x_i^2) without overflow or underflow for
 * any finite input (the norm of Section 2).  Per element, |x_i| is sorted
 * into small / medium / big ranges and squared after scaling by a power of
 * two (Blue, ACM TOMS 4(1), 1978, "A portable Fortran program to find the
 * Euclidean norm of a vector"), three accumulators per thread (the medium one
 * compensated in F32), FP64 combination and final square root.
 *   out    device pointer to one double; flags as salt_dot. */
salt_status salt_nrm2(int32_t dtype, int64_t n, const void* x, double* out, int32_t flags,
                      void* stream);

/* ---------------------------------------------------------------------------
 * salt_fill_uniform -- x[i] = element (offset + i) of the counter-based
 * uniform[-1, 1) stream keyed by `key`: z = key + (offset + i + 1) *
 * 0x9E3779B97F4A7C15 (mod 2^64), h = SplitMix64 finaliser of z (Steele, Lea,
 * Flood 2014); F64 value 2*(h >> 11)*2^-53 - 1, F32 value
 * 2*(h >> 40)*2^-24 - 1 (both exact).  Synthetic-input generator so that
 * multi-GB operands need no host upload.  Errors: SALT_ERR_ARG,
 * SALT_ERR_DTYPE, SALT_ERR_ALIGN, SALT_ERR_CUDA. */
salt_status salt_fill_uniform(int32_t dtype, int64_t n, uint64_t key, int64_t offset, void* x,
                              void* stream);

/* ---------------------------------------------------------------------------
 * salt_dot_noalloc -- *out = sum_i x_i * y_i, like salt_dot with
 * SALT_DEFAULT, but without any device allocation.  (The paper has no
 * counterpart: it is an interface for callers of this library.)
 * salt_dot's partial sums live in a workspace the library cudaMalloc's on the
 * first reducing call on a stream.  Callers that cannot allow that -- runtimes
 * that hand out all device memory from a fixed up-front reservation, loops
 * that cannot afford cudaMalloc's implicit device synchronisation -- use this
 * entry point instead.  Its scratch is a static device array of 32 KiB + 256 B that
 * every GPU loading the library holds until process exit; it never calls
 * cudaMalloc, cudaFree or any allocating routine.
 *   n      0 <= n <= 2^28 (268435456); larger n returns SALT_ERR_BUDGET
 *          (the scratch holds one partial per 65536 elements, 4096 in all)
 *   x, y   device, 16-byte aligned, `dtype` elements
 *   out    device pointer to one double
 * Accumulation as salt_dot (F32: compensated Dot2, F64: FMA), partials
 * combined in FP64 in a fixed order, so the result depends on n only.
 * The first call on each device looks up the scratch array's device address
 * (set-up); make that first call before capturing any stream.  Every call
 * shares the one array and clears its ticket word on `stream` before the
 * kernel: calls whose work overlaps on the GPU (two streams at once) race on
 * it, so serialise them.
 * Errors: SALT_ERR_DTYPE, SALT_ERR_ARG, SALT_ERR_ALIGN, SALT_ERR_BUDGET (all
 * before any launch), SALT_ERR_CUDA; text via salt_last_error(). */
salt_status salt_dot_noalloc(int32_t dtype, int64_t n, const void* x, const void* y, double* out,
                             void* stream);

/* ---------------------------------------------------------------------------
 * Run-time compilation of programs without a compile-time instantiation.
 * The paper's expression templates generate each expression's loop at
 * compile time (Section 2); salt_eval does the same at run time for any
 * program that has no compiled instantiation: the program is written out as
 * the template arguments of the same fused kernel and compiled by NVRTC for
 * the current GPU on the first call per (program, dtype, launch shape) --
 * tens to hundreds of milliseconds, so make that call before any stream
 * capture -- then cached for the process and on disk (see
 * salt_jit_cache_dir), so later processes load it in about a millisecond.
 * Results are bit-identical to the interpreter's.
 *   SALT_JIT_AUTO (the default): compile; where NVRTC cannot be loaded or a
 *                 compilation fails, run the program on the interpreter.
 *   SALT_JIT_ON:  compile; salt_eval returns SALT_ERR_CUDA with NVRTC's log
 *                 if compilation fails or NVRTC cannot be loaded.
 *   SALT_JIT_OFF: such programs run on the interpreter kernel.
 * salt_set_jit returns SALT_ERR_ARG for another mode. */
#define SALT_JIT_OFF 0
#define SALT_JIT_ON 1
#define SALT_JIT_AUTO 2
salt_status salt_set_jit(int32_t mode);
/* Current mode, kernels compiled so far and their total compile time (ms);
 * any pointer may be NULL. */
salt_status salt_jit_stats(int32_t* mode, int64_t* kernels, double* compile_ms);
/* The directory of compiled kernels kept on disk: `dir` (created on the
 * first write), or NULL / "" to keep none.  Without this call the
 * directory is $SALT_JIT_CACHE ("0" or "off": none), else
 * $XDG_CACHE_HOME/salt-jit, else $HOME/.cache/salt-jit.  A file is named by
 * a hash of the kernel, the GPU architecture, the NVRTC version and the
 * library's kernel sources, and is checked (magic word, payload hash) before
 * it is loaded; a file that fails the check or does not load is recompiled
 * and rewritten.  Files are written under a temporary name and renamed, so
 * processes may share the directory.  Returns SALT_OK. */
salt_status salt_jit_cache_dir(const char* dir);
/* Kernels loaded from and written to the on-disk cache since the library
 * was loaded, and the directory in use ("" if none; dir may be NULL). */
salt_status salt_jit_cache_stats(int64_t* disk_hits, int64_t* disk_writes, char* dir, int32_t dir_len);

/* Free every workspace the library holds (call with no library work in
 * flight).  Returns SALT_OK or SALT_ERR_CUDA. */
salt_status salt_release_workspaces(void);

/* ---------------------------------------------------------------------------
 * Launch configuration (the paper chose its loop unrolling and the number
 * of instruction packages per loop "by trial", Section 4.3; here an autotuner
 * chooses unroll depth, vector width and block/grid shape per program shape,
 * dtype and size bucket).
 *   unroll        vector accesses per operand per thread per tile (1, 2, 4)
 *   vec_bytes     bytes per vector access (16 or 32)
 *   block         threads per block (64..256, multiple of 32)
 *   blocks_per_sm resident blocks per SM the grid is sized for (1..32; 0:
 *                 as many as fit, from the occupancy calculator)
 *   stage_bytes   0: operands are loaded into registers by vector loads (the
 *                 register-tiled loop, shaped by unroll and vec_bytes).
 *                 4096, 8192 or 16384: the staged loop — each block copies
 *                 tiles of stage_bytes per loaded operand into shared memory
 *                 by bulk asynchronous copies, two stages deep, and computes
 *                 on one stage while the next fills; unroll and vec_bytes are
 *                 not used.  Only programs with a compile-time instantiation
 *                 whose operands are 16-byte aligned and contiguous take it
 *                 (others use their usual kernel).  Element results are
 *                 bit-identical either way; reduction results are summed in
 *                 another order (same error bounds).  The first staged launch
 *                 on a device allocates the 8-byte counter that
 *                 salt_staged_timeouts reads (so it cannot be the first
 *                 library call inside a CUDA-graph capture, like any call that
 *                 first needs a stream's reduction workspace).
 * salt_tune_set pins a configuration for (program, dtype, n bucket) where the
 * bucket is floor(log2(max(n,1))); salt_tune_get reports the configuration a
 * call would use.  Returns SALT_ERR_ARG for an invalid configuration (also
 * stage_bytes != 0 for a program without a compile-time instantiation). */
typedef struct {
  int32_t unroll;
  int32_t vec_bytes;
  int32_t block;
  int32_t blocks_per_sm;
  int32_t stage_bytes;
} salt_launch_cfg;

salt_status salt_tune_set(const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                          const salt_launch_cfg* cfg);
salt_status salt_tune_get(const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                          salt_launch_cfg* cfg);
/* Forget every pinned configuration. */
salt_status salt_tune_clear(void);

/* Kernel families for salt_autotune. */
#define SALT_KERNEL_PROGRAM 0    /* the kernel salt_eval picks for `prog`       */
#define SALT_KERNEL_NRM2 1       /* salt_nrm2, SALT_DEFAULT: vecs = {x}          */
#define SALT_KERNEL_NRM2_PLAIN 2 /* salt_nrm2, SALT_PLAIN (F32): vecs = {x}      */
#define SALT_KERNEL_DOT_PLAIN 3  /* salt_dot, SALT_PLAIN (F32): vecs = {x, y}    */

/* Autotuner: runs the call (arguments as salt_eval; for the other families
 * vecs / red_out as noted above) under every configuration of unroll {1,2,4}
 * x vec_bytes {16,32} x block {128,256} x blocks_per_sm {as many as fit, 2,
 * 4} of the register-tiled loop, and for programs with a compile-time
 * instantiation also the staged loop at stage_bytes {4096, 8192, 16384} x
 * block {128, 256} (as many blocks as fit), `reps` timed runs each after one
 * warm-up, on `stream`, and pins the fastest for (family, dtype, n bucket) in
 * the tuning table (a staged configuration only if it is more than 1% faster
 * than the best register-tiled one).  *best and *best_ms (either may be NULL) receive it and
 * its time per call.  The call runs (reps + 1) times per configuration (42
 * configurations for a compiled shape; 36 for nrm2 and the plain dot; 12 for
 * the interpreter, which has no unroll): in-place programs update their
 * operands each time.  When the operands total less than four times the L2
 * size, each timed call is preceded by a read of a scratch buffer twice the
 * L2 size (allocated for the call and freed at its end), so that the shape
 * is chosen for operands that come from device memory, not from L2. */
salt_status salt_autotune(int32_t kernel, const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                          void* const* vecs, int32_t nvecs, const double* scalars, int32_t nscal, double* red_out,
                          int32_t reps, salt_launch_cfg* best, double* best_ms, void* stream);
/* Writes the tuning table as text (one line per entry) / merges such a file
 * into it (lines without the stage_bytes column read as stage_bytes 0).
 * Errors: SALT_ERR_ARG (unreadable, unwritable or malformed). */
salt_status salt_tune_save(const char* path);
salt_status salt_tune_load(const char* path);

/* Waits of staged-loop launches (stage_bytes != 0) on the current device that
 * ran out of their bound (one second) since the library was loaded: *count.
 * A block whose stage copies did not arrive in time finishes its tiles from
 * direct loads (results unchanged) and counts one here.  Synchronous (reads a
 * device counter).  Errors: SALT_ERR_ARG (count NULL), SALT_ERR_CUDA. */
salt_status salt_staged_timeouts(uint64_t* count);

/* Number of kernel launches this library has issued on the calling process
 * (all threads), for accounting in benchmarks. */
int64_t salt_launch_count(void);

/* ===========================================================================
 * Batches: thousands of independent, uneven-length expressions and
 * reductions in ONE persistent launch, replayed as a CUDA graph.  (The paper
 * evaluates one expression per loop; a batch keeps its per-expression loop --
 * same compiled programs, same per-element results -- and removes the
 * per-call launch cost that dominates short vectors: Section 4.3 notes that
 * the best loop shape for small vectors differs from the one for large ones.)
 *
 * Every item is split into tiles of `tile_bytes` per operand; resident blocks
 * pull tiles from an atomic counter and run the owning item's program on the
 * tile.  An item's DOT / SUMSQ / norm result is the tile partial sums added
 * in tile order by the block that finishes the item's last tile, so it
 * depends only on the item's length and the tile size: the same bits whatever
 * else is in the batch.  Elementwise results are bit-identical to salt_eval.
 * Items must not write memory that another item of the batch reads or writes
 * (checked at launch: SALT_ERR_ALIAS).  A batch object is not thread-safe.
 *
 * The batch owns device memory for its item table, tile counters and
 * partials (allocated on the first launch after items change, freed by
 * salt_batch_destroy).  The first launch after any change uploads the table
 * synchronously (it waits for the stream) and builds the graph; launches
 * with unchanged items and the same red_out replay the graph. */
typedef struct salt_batch salt_batch;

/* capacity: maximum number of items (1 .. 2^20). */
salt_status salt_batch_create(salt_batch** out, int32_t capacity);
salt_status salt_batch_destroy(salt_batch* b);

/* Adds one program item; arguments as salt_eval (device operands, host
 * program and scalars read during the call).  The program must have a
 * compiled instantiation (salt_check_program's compiled_out) among the
 * batch kernel's shapes, at most 5 vector operands and 2 scalars, once its
 * scalar subexpressions (by-value scalars only; no DSCAL) are folded.  *red_index_out (may be NULL) receives the
 * index in the launch's red_out of the item's first DOT/SUMSQ result, or -1.
 * Errors: as salt_eval, SALT_ERR_BUDGET when full. */
salt_status salt_batch_add(salt_batch* b, const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                           void* const* vecs, int32_t nvecs, const double* scalars, int32_t nscal,
                           int32_t* red_index_out);
/* Adds a Euclidean-norm item (as salt_nrm2, SALT_DEFAULT accumulation). */
salt_status salt_batch_add_nrm2(salt_batch* b, int32_t dtype, int64_t n, const void* x, int32_t* red_index_out);
/* Removes every item (the device memory is kept for reuse). */
salt_status salt_batch_clear(salt_batch* b);
/* Item count, result count (red_out entries) and algorithmic bytes (each
 * operand element read once, each result element written once); any output
 * may be NULL. */
salt_status salt_batch_info(const salt_batch* b, int32_t* nitems, int32_t* nresults, int64_t* bytes);

/* Launch shape: unroll 1/2/4, block 64, 128 or 256,
 * blocks_per_sm 0 (as many as fit) .. 32, tile_bytes 1 KiB .. 64 MiB
 * (multiple of 256). */
salt_status salt_batch_set_config(salt_batch* b, int32_t unroll, int32_t block, int32_t blocks_per_sm,
                                  int64_t tile_bytes);
salt_status salt_batch_get_config(const salt_batch* b, int32_t* unroll, int32_t* block, int32_t* blocks_per_sm,
                                  int64_t* tile_bytes);
/* Vector width of the batch's accesses: 32 (the default) lets FP32 items
 * whose operands are all 32-byte aligned use 32-byte accesses (at half the
 * unroll, so the same bytes are in flight); 16 keeps every item on 16-byte
 * accesses.  Elementwise results are the same bits either way; reductions
 * are summed in another order (same error bounds).  Errors: SALT_ERR_ARG. */
salt_status salt_batch_set_vec_bytes(salt_batch* b, int32_t vec_bytes);
salt_status salt_batch_get_vec_bytes(const salt_batch* b, int32_t* vec_bytes);

/* One persistent launch over all items (a CUDA graph: counter reset + kernel)
 * on `stream`.  red_out: device array of >= nresults doubles. */
salt_status salt_batch_launch(salt_batch* b, double* red_out, void* stream);
/* The same items as individual salt_eval / salt_nrm2 calls on `stream`, in
 * item order (the plain per-call path, for comparison). */
salt_status salt_batch_launch_plain(salt_batch* b, double* red_out, void* stream);
/* Times every launch shape over unroll {1,2,4} x block {128,256} x
 * tile_bytes {16,32,64,128} KiB, and vector width {32,16} bytes when the
 * batch has FP32 items (reps launches each, after one warm-up), and keeps
 * the fastest; *best_ms (may be NULL) receives its time per launch.  The
 * items' programs run (1 + reps) x 24 (FP64 only) or x 48 times: in-place
 * programs update their operands each time. */
salt_status salt_batch_autotune(salt_batch* b, double* red_out, int32_t reps, double* best_ms, void* stream);

/* ===========================================================================
 * Serving: continuous batching of expression requests (no counterpart in the
 * paper, which evaluates one expression per call; each request here is still
 * one of its fused loops).
 *
 * A server owns a device arena of `budget_bytes` for request operands, a
 * scheduler thread and `streams` CUDA streams.  Submitted requests are
 * admitted in arrival order while fewer than `max_requests` are resident and
 * the arena can hold their operand vectors; a request stays resident until
 * the client releases it.  Whenever a stream is free, the scheduler launches
 * a step holding every admitted request not yet run (up to `max_batch`):
 * one batched launch fills the requests' input vectors on the device from
 * their keys (the counter-based generator of salt_fill_uniform, standing in
 * for the upload of client data), a second runs their programs (the batch
 * kernel).  Steps on different streams overlap on the GPU; requests arriving
 * meanwhile join the next step.  All requests use one tile size, so a
 * request's results are the same bits alone or in any mix.
 * Latency = host time at which the scheduler observed the step's completion
 * event minus the request's submission time.
 *
 * Persistent mode (`persistent` = 1): one cooperative launch stays resident
 * and runs the steps, which the scheduler posts to a ring of `streams`
 * entries in mapped pinned host memory (no launch, table upload or event
 * per step); the launch polls the ring, copies each step's tables to the
 * device, runs the fill and compute phases with the batch kernel's tile
 * loop and writes the step's completion to host memory.  Every device wait
 * is bounded; the launch ends after `idle_us` microseconds with nothing
 * posted (the GPU is then free for other work) and the scheduler launches
 * it again with the next step.  Results are the same bits as in the default
 * mode.  While a launch is resident it occupies every SM it was given, so
 * other kernels on the device wait for SMs until it ends. */
typedef struct salt_server salt_server;

typedef struct {
  int64_t budget_bytes; /* device arena for request operands (>= 1 MiB)          */
  int32_t max_requests; /* resident requests at once                              */
  int32_t max_batch;    /* requests per step (1 .. 65536)                          */
  int32_t streams;      /* steps in flight (1 .. 8)                                */
  int32_t tile_bytes;   /* bytes per operand per tile (>= 1024, multiple of 256)   */
  int32_t unroll;       /* batch kernel unroll: 1, 2, 4                            */
  int32_t block;        /* batch kernel block: 64, 128, 256                        */
  int64_t max_n;        /* longest request accepted                                */
  int32_t persistent;   /* 1: steps run in one resident launch (see above); 0: one  */
                        /* graph launch per step                                   */
  int32_t idle_us;      /* persistent mode: the resident launch ends after this     */
                        /* long with nothing posted (1 .. 10^7)                    */
} salt_serve_config;

/* Defaults: 8 GiB budget, 4096 resident requests, 256 per step, 2 streams,
 * 64 KiB tiles, unroll 2, 256 threads, n <= 2^24, not persistent, 10 ms
 * idle time. */
salt_status salt_serve_default_config(salt_serve_config* cfg);
/* Allocates the arena and per-stream tables on the current device and starts
 * the scheduler thread.  Errors: SALT_ERR_ARG, SALT_ERR_CUDA. */
salt_status salt_serve_start(salt_server** out, const salt_serve_config* cfg);
/* Drains the steps in flight, stops the scheduler, frees everything
 * (requests not yet complete are dropped). */
salt_status salt_serve_stop(salt_server* s);
/* Persistent mode: *launches = launches of the resident kernel so far (one,
 * plus one after each idle end), *live = 1 while one is running (as the
 * scheduler last saw it); 0 and 0 in the default mode.  Either pointer may
 * be NULL.  Errors: SALT_ERR_ARG. */
salt_status salt_serve_launches(salt_server* s, int64_t* launches, int32_t* live);

/* Submits a request.  prog/nprog: a program with a compiled instantiation
 * among the batch kernel's shapes (<= 5 vector operands, <= 2 scalars) once
 * its by-value scalar subexpressions are folded (no DSCAL; SALT_ERR_PROGRAM
 * otherwise); prog == NULL requests the Euclidean
 * norm of one operand.  keys[k] (nkeys entries, one per operand index) seeds
 * operand k's contents: element i is value i of the counter-based uniform
 * stream `keys[k]` (salt_fill_uniform); keys of output-only operands are
 * ignored.  Scalars are read during the call.  *request_id receives the id.
 * Errors: SALT_ERR_ARG (n beyond max_n, stopped server), SALT_ERR_PROGRAM,
 * SALT_ERR_DTYPE, SALT_ERR_BUDGET (operands larger than the whole arena). */
salt_status salt_serve_submit(salt_server* s, const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                              const uint64_t* keys, int32_t nkeys, const double* scalars, int32_t nscal,
                              int64_t* request_id);
/* salt_serve_submit with caller-owned operands: ptrs (nops entries, may be
 * NULL) gives, per operand index, a DEVICE pointer to n elements of the
 * request's dtype, 16-byte aligned (SALT_ERR_ALIGN otherwise), that the
 * request reads (and, if stored, writes) in place: no arena space, no fill.
 * Operands whose pointer is NULL are server-owned and keyed by keys[k] as in
 * salt_serve_submit (keys may be NULL if every operand has a pointer).  The
 * caller keeps caller-owned memory valid and unmodified until the request
 * is done, and its contents ready when submitting (the server's work is not
 * ordered after the caller's streams: synchronize the writes first); two
 * requests in flight must not write memory another one reads or writes (not
 * checked).  salt_serve_read copies caller-owned operands
 * too. */
salt_status salt_serve_submit_ex(salt_server* s, const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                                 const void* const* ptrs, const uint64_t* keys, int32_t nops,
                                 const double* scalars, int32_t nscal, int64_t* request_id);
/* State: 0 waiting, 1 running, 2 done.  When done: *latency_us and the
 * request's DOT/SUMSQ/norm results in red[0..nred) (host memory); either
 * pointer may be NULL.  SALT_ERR_NOTFOUND for an unknown (or released) id. */
salt_status salt_serve_poll(salt_server* s, int64_t id, int32_t* state, double* latency_us, double* red);
/* Waits (bounded) until the request is done: SALT_ERR_TIMEOUT after
 * timeout_us microseconds. */
salt_status salt_serve_wait(salt_server* s, int64_t id, int64_t timeout_us);
/* Copies operand `operand` (the submit's operand index) of a done request to
 * host memory (bytes >= n * element size). */
salt_status salt_serve_read(salt_server* s, int64_t id, int32_t operand, void* host_dst, int64_t bytes);
/* Frees a done request's operands, or cancels a waiting one.  A running
 * request cannot be released (SALT_ERR_ARG). */
salt_status salt_serve_release(salt_server* s, int64_t id);
/* Completed requests, steps launched, algorithmic bytes of completed
 * requests, arena bytes in use, requests waiting; any pointer may be NULL. */
salt_status salt_serve_stats(salt_server* s, int64_t* completed, int64_t* steps, int64_t* bytes,
                             int64_t* resident_bytes, int32_t* waiting);
/* Load generator: submits `count` requests at host times t0 + arrival_us[i]
 * (t0 = the call's start; arrival_us ascending), each the standard served
 * shape shape[i] -- 0: d = a + (b - c), 1: y = 1.5 x - 0.25 y, 2: e = 1.5 a -
 * 0.25 b - c o d, 3: dot(x, y), 4: nrm2(x) -- with dtype[i] and n[i], operand
 * k keyed seed * 0x100000001B3 + i * 16 + k + 1 (mod 2^64); releases each
 * request as it completes and returns latency_us[i] (measured from its
 * nominal arrival), its first result red_first[i] (may be NULL; 0 if none)
 * and *wall_us, the time from t0 to the last completion. */
salt_status salt_serve_replay(salt_server* s, int32_t count, const double* arrival_us, const int32_t* shape,
                              const int32_t* dtype, const int64_t* n, uint64_t seed, double* latency_us,
                              double* red_first, double* wall_us);
/* salt_serve_replay over a RESIDENT STORE: the input operands that a shape
 * only reads come from caller-owned device vectors (salt_serve_submit_ex)
 * instead of a per-request fill: operand k of request i reads elements
 * [o, o + n[i]) of store vector (5 i + k) mod nstore of its dtype, with
 *   h = (key * 0x9E3779B97F4A7C15 mod 2^64) >> 11,
 *   o = (h mod (len - n[i] + 1)), rounded down to a multiple of 32 bytes
 *       (8 FP32 or 4 FP64 elements),
 * key the operand's key above.  Stored operands (d, y, e) stay server-owned
 * (y, read and written, is filled from its key).  store_f32 / store_f64:
 * nstore_f32 / nstore_f64 device vectors of len_f32 / len_f64 elements,
 * 16-byte aligned (32-byte aligned, as cudaMalloc's are, for 256-bit
 * accesses); every n[i] <= the length of its dtype's vectors. */
salt_status salt_serve_replay_store(salt_server* s, int32_t count, const double* arrival_us, const int32_t* shape,
                                    const int32_t* dtype, const int64_t* n, uint64_t seed,
                                    const void* const* store_f32, int32_t nstore_f32, int64_t len_f32,
                                    const void* const* store_f64, int32_t nstore_f64, int64_t len_f64,
                                    double* latency_us, double* red_first, double* wall_us);

#ifdef __cplusplus
}
#endif

#endif /* SALT_H */
