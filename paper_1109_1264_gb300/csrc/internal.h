// Internal interfaces shared by the C-ABI translation units (not exported).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/salt.h"
#include "host.h"

namespace salt {

struct EvalArgs {
  const salt_insn* prog;
  int nprog;
  int dt;
  int64_t n;
  void* const* vecs;
  int nvecs;
  const double* scalars;
  int nscal;
  double* red_out;
  cudaStream_t stream;
  const int64_t* strides = nullptr;  // per operand, in elements; NULL: all 1
  const double* const* dscal = nullptr;  // device scalars (DSCAL k reads *dscal[k])
  int ndscal = 0;
};

// Records `msg` as the calling thread's salt_last_error() and returns `st`.
salt_status report_error(salt_status st, const std::string& msg);

// Every host-side check of a salt_eval call (dtype, sizes, program, NULL
// operands, alignment, aliasing).  Fills `an` on success.  No CUDA calls.
salt_status validate_eval(const EvalArgs& a, Analysis* an);

// salt_eval and salt_nrm2 without the C wrappers.
salt_status eval_impl(const EvalArgs& a);
salt_status nrm2_impl(int32_t dtype, int64_t n, const void* x, double* out, int32_t flags, cudaStream_t s);

// Conjugate gradients for diag(d) x = b (salt_cg_diag): the programs over
// operand slots 0 d, 1 p, 2 q, 3 x, 4 r, 5 b, one checked or launched call,
// and every check of a run before its first launch.
extern const salt_insn kCgR0[8], kCgP0[9], kCgPQ[15], kCgXR[18];
salt_status cg_call(const salt_insn* prog, int len, int32_t dtype, int64_t n, void* const* vecs, double* red,
                    const double* ds0, const double* ds1, cudaStream_t s, bool check_only);
salt_status cg_validate(int32_t dtype, int64_t n, void* const* vecs, int32_t iters, double* rho, cudaStream_t s);

// The reduction workspace of stream `s`: FP64 partials (capacity doubles)
// and a 256-byte slot of words whose first word is the reduction ticket
// (zero between launches); the others are free for one launch's use.
salt_status stream_workspace(cudaStream_t s, double** partials, unsigned** words, int* capacity);

// SM count of the current device (cached); 0 and an error on failure.
salt_status current_device(int* dev, int* sms);

// Number of kernel launches issued by the library (all threads).
void count_launch();

// Polls one grid barrier of the cooperative CG kernels spends before it
// records a timeout; `set` >= 0 replaces the limit first.  Returns the limit.
unsigned cg_barrier_polls(int64_t set);
// Poll bound of the persistent serving kernel's waits (read at each launch).
unsigned serve_polls(int64_t set);

// Run-time compiled fused kernels (csrc/jit.cu): the current mode
// (SALT_JIT_OFF / SALT_JIT_ON / SALT_JIT_AUTO; SALT_JIT_OFF while this
// thread has suspended run-time compilation) and the kernel for a canonical
// program (compiled, or read from the on-disk cache, on first use).
int32_t jit_mode();
// This thread's record of a failed run-time compilation since the last reset,
// and its suspension of run-time compilation (the SALT_JIT_AUTO fallback).
void jit_failure_reset();
bool jit_failed();
void jit_suspend(bool on);
// ds: the variant that computes scalar slots on the device (fused kernel
// only; the element-access kernel always can).
salt_status jit_kernel(const Canonical& c, int is_f32, int unroll, int vec_bytes, bool ds,
                       const void** kernel_out);

}  // namespace salt
