// Device building blocks shared by the SALT kernels: exact per-node
// arithmetic, 128/256-bit vector memory access (the paper's vectorizer,
// Section 3), reduction accumulators and deterministic block combination.
#pragma once

#ifdef __CUDACC_RTC__
// Compiled at run time by NVRTC (csrc/jit.cu): no system headers there.
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef short int16_t;
typedef unsigned char uint8_t;
typedef decltype(sizeof(0)) size_t;
#else
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "prog.cuh"

namespace salt {

// ---------------------------------------------------------------------------
// Arithmetic of one tree node: one correctly rounded IEEE operation, never
// contracted into an FMA (the _rn intrinsics are exempt from contraction),
// so a fused loop produces the same bits as evaluating node by node.
template <typename T> struct Arith;
template <> struct Arith<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
};
// FP64 nodes issue as FMAs whose product is exact: a + b = fma(a, 1, b),
// a - b = fma(b, -1, a), a * b = fma(a, b, -0) (adding -0 leaves every
// product unchanged, a zero product's sign included; +0 would turn -0 into
// +0).  Each is one rounding of the exact result, the bits of DADD / DSUB /
// DMUL, and on GB300 the FP64 pipe issues DFMA about 19% faster than DADD
// and DMUL (593 against 500 G instructions/s, register-only).  The
// constants live in constant memory, which the host may rewrite, so the
// compiler cannot fold the FMAs back into additions and multiplications;
// DFMA reads a constant-bank operand at no cost.
static __constant__ double kFmaOne = 1.0, kFmaNegOne = -1.0, kFmaNegZero = -0.0;
template <> struct Arith<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __fma_rn(a, kFmaOne, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __fma_rn(b, kFmaNegOne, a); }
  static __device__ __forceinline__ double mul(double a, double b) { return __fma_rn(a, b, kFmaNegZero); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};

// ---------------------------------------------------------------------------
// Scalar subexpressions (the paper's init / load_once values, Section 4.2:
// computed once per loop, not per element).  The host replaces every scalar
// subtree of a program by one scalar slot.  When the subtree reads a scalar
// that lives in device memory, its value is computed on the device at kernel
// start by this small stack code, one operation per node in T, and written
// to the slot; otherwise the host computes it the same way before launch.
enum : uint8_t { S_SC = 0, S_DS, S_ADD, S_SUB, S_MUL, S_DIV, S_NEG, S_OUT };
constexpr int kMaxScalarCode = 48;
struct ScalarCode {
  int32_t len;                   // instructions; 0: every slot is passed by value
  uint8_t code[kMaxScalarCode];  // op * 16 + arg
  double cval[kMaxScals];        // S_SC k pushes cval[k] rounded to T
  const double* ds[kMaxDscals];  // S_DS k pushes *ds[k] rounded to T
};

// Runs `c` in one thread with its stack and slots in shared memory (no
// local memory); S_OUT k pops into sc[k].  The host validated the code, so
// the stack stays within kMaxStack; the bound checks only keep a malformed
// code inside the arrays.
template <typename T>
__device__ __forceinline__ void run_scalar_code(const ScalarCode& c, T* st, T* sc) {
  int sp = 0;
  for (int pc = 0; pc < c.len && pc < kMaxScalarCode; ++pc) {
    const int op = c.code[pc] >> 4, k = c.code[pc] & 15;
    if (op == S_SC || op == S_DS) {
      if (sp > kMaxStack || k >= kMaxScals) return;
      st[sp++] = op == S_SC ? (T)c.cval[k] : (T)(*c.ds[k]);
    } else if (op == S_NEG) {
      if (sp < 1) return;
      st[sp - 1] = -st[sp - 1];
    } else if (op == S_OUT) {
      if (sp < 1 || k >= kMaxScals) return;
      sc[k] = st[--sp];
    } else {
      if (sp < 2) return;
      const T a = st[sp - 2], b = st[sp - 1];
      st[sp - 2] = op == S_ADD ? Arith<T>::add(a, b)
                 : op == S_SUB ? Arith<T>::sub(a, b)
                 : op == S_MUL ? Arith<T>::mul(a, b)
                               : Arith<T>::div(a, b);
      --sp;
    }
  }
}

// The scalar slots of a launch: the by-value slots `psc`, with the slots
// that `c` computes overwritten (thread 0 evaluates, the block shares the
// values through shared memory).  Uniform branch when len == 0.
template <typename T>
__device__ __forceinline__ void load_scalars(const T (&psc)[kMaxScals], const ScalarCode& c,
                                             T (&sc)[kMaxScals]) {
#pragma unroll
  for (int k = 0; k < kMaxScals; ++k) sc[k] = psc[k];
  if (c.len > 0) {
    __shared__ T s_sc[kMaxScals];
    __shared__ T s_st[kMaxStack + 1];
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < kMaxScals; ++k) s_sc[k] = psc[k];
      run_scalar_code<T>(c, s_st, s_sc);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMaxScals; ++k) sc[k] = s_sc[k];
  }
}

// ---------------------------------------------------------------------------
// By-value FP64 scalar slots that are exact powers of two, s = +-2^e (found on
// the host).  For such a slot a node pair X + s*v (or X - s*v) may run as one
// FMA with the same bits: s*v is exact whenever its exponent stays in the
// normal range, and then round(X + round(s*v)) = round(X + s*v).  The kernel
// checks that range per element from the exponent bits of v (integer
// instructions) and otherwise runs the two rounded operations.  On GB300 this
// saves an instruction on the FP64 pipe, which bounds the FP64 shapes with
// several nodes per element.
struct Pow2Info {
  uint32_t mask;              // bit k: slot k is +-2^exp[k]
  int16_t exp[kMaxScals];     // -1022 .. 1023
};

// s*v is exact (s = +-2^e): v is normal, NaN or infinite, and v*2^e keeps a
// biased exponent in 1 .. 2046 -- a normal number (or, for v infinite or
// NaN, the same infinity or NaN; its sign and the NaN-ness are the same on
// both paths).
__device__ __forceinline__ bool exact_pow2_scale(double v, int e) {
  const int be = (__double2hiint(v) >> 20) & 0x7FF;
  const int r = be + e;
  return be >= 1 && r >= 1 && (r <= 2046 || be == 2047);
}

// ---------------------------------------------------------------------------
// The vectorizer: VB-byte vectors of T (VB = 16 or 32).  32-byte accesses are
// the sm_100-family ld/st .v8.b32 / .v4.b64 forms.
template <typename T, int VB>
struct __align__(VB) VecT {
  static constexpr int N = VB / (int)sizeof(T);
  T e[N];
};

// RO: the operand is never written by this kernel, so the non-coherent
// read-only path may be used.
template <bool RO>
__device__ __forceinline__ void vload(VecT<float, 16>& v, const float* p) {
  if (RO)
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(v.e[0]), "=f"(v.e[1]), "=f"(v.e[2]), "=f"(v.e[3]) : "l"(p));
  else
    asm volatile("ld.global.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.e[0]), "=f"(v.e[1]), "=f"(v.e[2]), "=f"(v.e[3]) : "l"(p) : "memory");
}
template <bool RO>
__device__ __forceinline__ void vload(VecT<float, 32>& v, const float* p) {
  if (RO)
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v.e[0]), "=f"(v.e[1]), "=f"(v.e[2]), "=f"(v.e[3]), "=f"(v.e[4]), "=f"(v.e[5]),
          "=f"(v.e[6]), "=f"(v.e[7]) : "l"(p));
  else
    asm volatile("ld.global.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v.e[0]), "=f"(v.e[1]), "=f"(v.e[2]), "=f"(v.e[3]), "=f"(v.e[4]), "=f"(v.e[5]),
                   "=f"(v.e[6]), "=f"(v.e[7]) : "l"(p) : "memory");
}
template <bool RO>
__device__ __forceinline__ void vload(VecT<double, 16>& v, const double* p) {
  if (RO)
    asm("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(v.e[0]), "=d"(v.e[1]) : "l"(p));
  else
    asm volatile("ld.global.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
                 : "=d"(v.e[0]), "=d"(v.e[1]) : "l"(p) : "memory");
}
template <bool RO>
__device__ __forceinline__ void vload(VecT<double, 32>& v, const double* p) {
  if (RO)
    asm("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
        : "=d"(v.e[0]), "=d"(v.e[1]), "=d"(v.e[2]), "=d"(v.e[3]) : "l"(p));
  else
    asm volatile("ld.global.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v.e[0]), "=d"(v.e[1]), "=d"(v.e[2]), "=d"(v.e[3]) : "l"(p) : "memory");
}

__device__ __forceinline__ void vstore(float* p, const VecT<float, 16>& v) {
  asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};"
               :: "l"(p), "f"(v.e[0]), "f"(v.e[1]), "f"(v.e[2]), "f"(v.e[3]) : "memory");
}
__device__ __forceinline__ void vstore(float* p, const VecT<float, 32>& v) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :: "l"(p), "f"(v.e[0]), "f"(v.e[1]), "f"(v.e[2]), "f"(v.e[3]), "f"(v.e[4]),
                  "f"(v.e[5]), "f"(v.e[6]), "f"(v.e[7]) : "memory");
}
__device__ __forceinline__ void vstore(double* p, const VecT<double, 16>& v) {
  asm volatile("st.global.v2.f64 [%0], {%1,%2};" :: "l"(p), "d"(v.e[0]), "d"(v.e[1]) : "memory");
}
__device__ __forceinline__ void vstore(double* p, const VecT<double, 32>& v) {
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};"
               :: "l"(p), "d"(v.e[0]), "d"(v.e[1]), "d"(v.e[2]), "d"(v.e[3]) : "memory");
}

// ---------------------------------------------------------------------------
// Reduction accumulators (the paper's per-unroll Storage with a reduction()
// method, Section 4.2).

// F32, compensated: TwoProduct (via FMA) + TwoSum, i.e. Ogita-Rump-Oishi
// Dot2.  s carries the running sum, c the accumulated rounding errors.
struct AccF32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float ep = __fmaf_rn(a, b, -p);        // a*b - p exactly
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, p);
    const float es = __fadd_rn(__fsub_rn(s, z), __fsub_rn(p, __fsub_rn(t, z)));  // s + p - t exactly
    s = t;
    c = __fadd_rn(c, __fadd_rn(es, ep));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// F32, plain: FP32 fused multiply-add accumulation (the comparison mode).
struct AccF32Plain {
  float s = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) { s = __fmaf_rn(a, b, s); }
  __device__ __forceinline__ float value() const { return s; }
};

// F64: FP64 fused multiply-add accumulation (one FP64 instruction per term).
struct AccF64 {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = __fma_rn(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = AccF32; };
template <> struct AccOf<double> { using type = AccF64; };

// ---------------------------------------------------------------------------
// Per-block timeline of a launch, for diagnosing where a kernel's time goes
// (launch ramp, tail, cross-block combine).  Off unless the caller set a
// trace buffer (salt_trace_set): then thread 0 of block b writes
// kTraceWords words at trace[b * kTraceWords]: the global timer (ns) at
// block start, after the whole tiles, before and after the cross-block
// combine, then the SM id and 1 if the block performed the final combine.
constexpr int kTraceWords = 8;
enum : int { TR_START = 0, TR_TILES = 1, TR_PRE_COMBINE = 2, TR_END = 3, TR_SM = 4, TR_LAST = 5 };

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void trace_mark(unsigned long long* tr, int k) {
  if (tr != nullptr && threadIdx.x == 0) tr[(size_t)blockIdx.x * kTraceWords + k] = global_ns();
}

__device__ __forceinline__ void trace_end(unsigned long long* tr, bool last) {
  if (tr != nullptr && threadIdx.x == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    unsigned long long* w = tr + (size_t)blockIdx.x * kTraceWords;
    w[TR_END] = global_ns();
    w[TR_SM] = sm;
    w[TR_LAST] = last ? 1ull : 0ull;
  }
}

// ---------------------------------------------------------------------------
// Deterministic block sums of NV values at once: a butterfly of warp
// shuffles within each warp, then every thread adds the per-warp sums in
// warp order.  Every lane of a warp ends the butterfly with the same bits
// (each step adds the same two values, in either order), so the sums are
// identical in every thread and depend only on blockDim (a multiple of 32,
// at most kMaxBlock).  Every thread of the block must call it (it holds two
// block barriers -- one pair for all NV values), so all 32 lanes of each
// warp reach the full-mask shuffles; shfl.sync itself waits for every lane
// named in its mask, whatever divergent code precedes the call.
constexpr int kMaxBlock = 256;
constexpr int kWarpSlots = 32;  // buf slots per value (>= warps per block)
template <typename R, int NV>
__device__ __forceinline__ void block_sum_n(R (&v)[NV], R* buf /* >= NV * kWarpSlots entries */) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // buf may still be read by a previous call
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[k * kWarpSlots + warp] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    R t = buf[k * kWarpSlots];
    for (unsigned w = 1; w < nw; ++w) t += buf[k * kWarpSlots + w];
    v[k] = t;
  }
}

template <typename R>
__device__ __forceinline__ R block_sum(R v, R* buf /* >= kWarpSlots entries */) {
  R a[1] = {v};
  block_sum_n<R, 1>(a, buf);
  return a[0];
}

// Ticket increment with release and acquire semantics at GPU scope: the
// caller's earlier writes are visible to whoever observes the increment,
// and the caller observes every write released by earlier increments.
__device__ __forceinline__ unsigned ticket_add_acq_rel(unsigned* t, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(t), "r"(v) : "memory");
  return old;
}

// Cross-block combination: every block deposits NV partial values; the last
// block to finish (atomic ticket, no waiting) adds them up in block order and
// returns the NV totals in vals, then re-arms the ticket.  Thread 0 writes
// the block's partials and takes the ticket with release-acquire semantics,
// so the last block's thread 0 observes every other block's partials, and
// the barrier that follows orders its threads' reads after that.  Returns
// true in the last block.
template <typename R, int NV>
__device__ __forceinline__ bool grid_combine(R (&vals)[NV], R* partials, unsigned* ticket,
                                             R* smem /* >= NV * kWarpSlots entries */) {
  block_sum_n<R, NV>(vals, smem);
  if (gridDim.x == 1) return true;  // one block: its sums are the totals (no partials, ticket or fences)
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)blockIdx.x * NV + k] = vals[k];
    is_last = ticket_add_acq_rel(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  // Thread t adds partials t, t + blockDim.x, ... in that order; four loads
  // are issued before their additions, so the reads overlap.
  const volatile R* part = (const volatile R*)partials;
  const unsigned G = gridDim.x, bd = blockDim.x;
#pragma unroll
  for (int k = 0; k < NV; ++k) vals[k] = R(0);
  unsigned b = threadIdx.x;
  for (; b + 3 * bd < G; b += 4 * bd) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const R p0 = part[(size_t)b * NV + k], p1 = part[(size_t)(b + bd) * NV + k];
      const R p2 = part[(size_t)(b + 2 * bd) * NV + k], p3 = part[(size_t)(b + 3 * bd) * NV + k];
      vals[k] = (((vals[k] + p0) + p1) + p2) + p3;
    }
  }
  for (; b < G; b += bd) {
#pragma unroll
    for (int k = 0; k < NV; ++k) vals[k] += part[(size_t)b * NV + k];
  }
  block_sum_n<R, NV>(vals, smem);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

}  // namespace salt
