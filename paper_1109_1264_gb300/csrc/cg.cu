// Conjugate gradients for diag(d) x = b in ONE cooperative launch
// (salt_cg_diag_persistent): every block stays resident for all iterations
// and the blocks meet at a grid-wide barrier after each reduction, so an
// iteration costs two barriers instead of two kernel launches.
//
// Per element the operations are those of salt_cg_diag's programs, in the
// same order and precision (r = b - d*x; p = r + beta*p; q = d*p;
// x = x + alpha*p; r = r - alpha*q), and alpha = rho / (p.q), beta =
// rho' / rho are the same one-division-in-T scalar nodes.  The reductions
// are the library's accumulators (compensated FP32, FP64 FMA) combined per
// block by the warp-shuffle block sums and across blocks in block order, which
// every block does for itself, so all blocks hold the same scalars.
//
// Barrier: a monotonic arrival counter (zeroed before the launch); barrier
// m is passed when the counter reaches m * gridDim.x.  Waits are bounded:
// after max_polls polls (kMaxSpins unless a test sets a smaller limit) a
// block records a timeout in the status word, writes NaN into rho[0] (block
// 0) and returns, and every other block returns at its next barrier, so a
// launch that cannot make progress ends instead of hanging; salt_cg_status
// reports the status word.  The cooperative launch guarantees that all
// blocks are resident.
//
// salt_cg_diag_one_reduction uses the same launch, barrier and reductions
// for Chronopoulos and Gear's recurrence: one pass and one barrier per
// iteration (cg_one_reduction_kernel below).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "../../include/salt.h"
#include "common.cuh"
#include "internal.h"

namespace salt {

namespace {

constexpr unsigned kMaxSpins = 1u << 26;  // polls of >= 32 ns and an L2 round trip: seconds
constexpr int kCgBlock = 256;
std::atomic<unsigned> g_barrier_polls{kMaxSpins};  // tests lower it to make a barrier run out

template <typename T>
struct CgParams {
  const T* d;
  const T* b;
  T* x;
  T* r;
  T* p;
  T* q;
  int64_t n;
  int32_t iters;
  double* rho;        // history: rho[0], then (p.q, rho') per iteration
  double* partials;   // 2 * gridDim.x values
  unsigned long long* counter;  // barrier arrivals, zero at launch
  unsigned* status;             // 0, or 1 after a barrier timeout
  unsigned max_polls;           // polls of one barrier before it records a timeout
};

// Returns false if the barrier timed out (here or in another block).
__device__ bool grid_barrier(unsigned long long* counter, unsigned* status, unsigned long long target,
                             unsigned max_polls) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(counter, 1ull);
    unsigned spins = 0;
    for (;;) {
      if (*(volatile unsigned*)status != 0u) {
        ok = 0;
        break;
      }
      if (*(volatile unsigned long long*)counter >= target) break;
      if (++spins > max_polls) {
        atomicExch(status, 1u);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block sum of each block's value, written to partials[slot * G + block];
// after the barrier every block adds the G partials in block order.
template <typename T>
__device__ bool grid_sum(double v, double* partials, int slot, unsigned long long* counter, unsigned* status,
                         unsigned long long target, unsigned max_polls, double* smem, double* out) {
  const double bs = block_sum<double>(v, smem);
  if (threadIdx.x == 0) partials[(size_t)slot * gridDim.x + blockIdx.x] = bs;
  if (!grid_barrier(counter, status, target, max_polls)) return false;
  const volatile double* part = (const volatile double*)partials + (size_t)slot * gridDim.x;
  if (gridDim.x <= 32) {
    // few blocks: one thread adds them in block order (one barrier)
    __shared__ double s_tot;
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) a += part[k];
      s_tot = a;
    }
    __syncthreads();
    *out = s_tot;
    return true;
  }
  double a = 0.0;
  for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) a += part[k];
  // the same fixed-order block sum in every block: identical totals
  *out = block_sum<double>(a, smem);
  return true;
}

// Two block sums written to partials[slot0 * G + block] and
// partials[(slot0 + 1) * G + block], then ONE barrier, then every block adds
// each set of G partials in block order (the same fixed-order block sum as
// grid_sum, so every block holds the same totals).
__device__ bool grid_sum2(double v0, double v1, double* partials, int slot0, unsigned long long* counter,
                          unsigned* status, unsigned long long target, unsigned max_polls, double* smem,
                          double* out0, double* out1) {
  double bs[2] = {v0, v1};
  block_sum_n<double, 2>(bs, smem);
  if (threadIdx.x == 0) {
    partials[(size_t)slot0 * gridDim.x + blockIdx.x] = bs[0];
    partials[(size_t)(slot0 + 1) * gridDim.x + blockIdx.x] = bs[1];
  }
  if (!grid_barrier(counter, status, target, max_polls)) return false;
  const volatile double* part0 = (const volatile double*)partials + (size_t)slot0 * gridDim.x;
  const volatile double* part1 = part0 + gridDim.x;
  if (gridDim.x <= 32) {
    __shared__ double s_tot[2];
    if (threadIdx.x == 0) {
      double a0 = 0.0, a1 = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) {
        a0 += part0[k];
        a1 += part1[k];
      }
      s_tot[0] = a0;
      s_tot[1] = a1;
    }
    __syncthreads();
    *out0 = s_tot[0];
    *out1 = s_tot[1];
    __syncthreads();  // s_tot is read before the next call overwrites it
    return true;
  }
  double a[2] = {0.0, 0.0};
  for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
    a[0] += part0[k];
    a[1] += part1[k];
  }
  block_sum_n<double, 2>(a, smem);
  *out0 = a[0];
  *out1 = a[1];
  return true;
}

// W consecutive elements of one operand: one 16-byte access when W > 1.
template <typename T, int W>
__device__ __forceinline__ void load_w(T (&v)[W], const T* src) {
  if constexpr (W == 1) {
    v[0] = *src;
  } else {
    VecT<T, 16> t;
    vload<false>(t, src);
#pragma unroll
    for (int e = 0; e < W; ++e) v[e] = t.e[e];
  }
}
template <typename T, int W>
__device__ __forceinline__ void store_w(T* dst, const T (&v)[W]) {
  if constexpr (W == 1) {
    *dst = v[0];
  } else {
    VecT<T, 16> t;
#pragma unroll
    for (int e = 0; e < W; ++e) t.e[e] = v[e];
    vstore(dst, t);
  }
}

// The three element passes on elements [j, j + W).
template <typename T, int W, class Acc>
__device__ __forceinline__ void start_w(const CgParams<T>& p, int64_t j, Acc& acc) {
  T b[W], d[W], x[W], r[W];
  load_w<T, W>(b, p.b + j);
  load_w<T, W>(d, p.d + j);
  load_w<T, W>(x, p.x + j);
#pragma unroll
  for (int e = 0; e < W; ++e) {
    r[e] = Arith<T>::sub(b[e], Arith<T>::mul(d[e], x[e]));
    acc.add_prod(r[e], r[e]);
  }
  store_w<T, W>(p.r + j, r);
}

template <typename T, int W, class Acc>
__device__ __forceinline__ void pass1_w(const CgParams<T>& p, int64_t j, bool first, T beta, Acc& acc) {
  T r[W], pv[W], d[W], q[W];
  load_w<T, W>(r, p.r + j);
  load_w<T, W>(d, p.d + j);
  if (!first) load_w<T, W>(pv, p.p + j);
#pragma unroll
  for (int e = 0; e < W; ++e) {
    pv[e] = first ? r[e] : Arith<T>::add(r[e], Arith<T>::mul(beta, pv[e]));
    q[e] = Arith<T>::mul(d[e], pv[e]);
    acc.add_prod(pv[e], q[e]);
  }
  store_w<T, W>(p.p + j, pv);
  store_w<T, W>(p.q + j, q);
}

template <typename T, int W, class Acc>
__device__ __forceinline__ void pass2_w(const CgParams<T>& p, int64_t j, T alpha, Acc& acc) {
  T x[W], pv[W], r[W], q[W];
  load_w<T, W>(x, p.x + j);
  load_w<T, W>(pv, p.p + j);
  load_w<T, W>(r, p.r + j);
  load_w<T, W>(q, p.q + j);
#pragma unroll
  for (int e = 0; e < W; ++e) {
    x[e] = Arith<T>::add(x[e], Arith<T>::mul(alpha, pv[e]));
    r[e] = Arith<T>::sub(r[e], Arith<T>::mul(alpha, q[e]));
    acc.add_prod(r[e], r[e]);
  }
  store_w<T, W>(p.x + j, x);
  store_w<T, W>(p.r + j, r);
}

// One-reduction CG (q holds s = A p): the start and the single pass.
template <typename T, int W, class Acc>
__device__ __forceinline__ void cgc_start_w(const CgParams<T>& p, int64_t j, Acc& ag, Acc& ad) {
  T b[W], d[W], x[W], r[W];
  load_w<T, W>(b, p.b + j);
  load_w<T, W>(d, p.d + j);
  load_w<T, W>(x, p.x + j);
#pragma unroll
  for (int e = 0; e < W; ++e) {
    r[e] = Arith<T>::sub(b[e], Arith<T>::mul(d[e], x[e]));
    ag.add_prod(r[e], r[e]);
    ad.add_prod(Arith<T>::mul(d[e], r[e]), r[e]);
  }
  store_w<T, W>(p.r + j, r);
}

template <typename T, int W, class Acc>
__device__ __forceinline__ void cgc_pass_w(const CgParams<T>& p, int64_t j, bool first, T beta, T alpha, Acc& ag,
                                           Acc& ad) {
  T d[W], r[W], pv[W], sv[W], x[W];
  load_w<T, W>(d, p.d + j);
  load_w<T, W>(r, p.r + j);
  load_w<T, W>(x, p.x + j);
  if (!first) {
    load_w<T, W>(pv, p.p + j);
    load_w<T, W>(sv, p.q + j);
  }
#pragma unroll
  for (int e = 0; e < W; ++e) {
    const T dr = Arith<T>::mul(d[e], r[e]);
    pv[e] = first ? r[e] : Arith<T>::add(r[e], Arith<T>::mul(beta, pv[e]));
    sv[e] = first ? dr : Arith<T>::add(dr, Arith<T>::mul(beta, sv[e]));
    x[e] = Arith<T>::add(x[e], Arith<T>::mul(alpha, pv[e]));
    r[e] = Arith<T>::sub(r[e], Arith<T>::mul(alpha, sv[e]));
    ag.add_prod(r[e], r[e]);
    ad.add_prod(Arith<T>::mul(d[e], r[e]), r[e]);
  }
  store_w<T, W>(p.p + j, pv);
  store_w<T, W>(p.q + j, sv);
  store_w<T, W>(p.x + j, x);
  store_w<T, W>(p.r + j, r);
}

// Every element of the thread, the same ones in every pass: 16-byte groups
// of W when `vec` (all operands 16-byte aligned), then single elements.
#define SALT_CG_EACH(CALL)                                                    \
  {                                                                           \
    int64_t done = 0;                                                         \
    if (vec) {                                                                \
      const int64_t nv = n / VW;                                              \
      for (int64_t j = gid; j < nv; j += stride) CALL(VW, j * VW);            \
      done = nv * VW;                                                         \
    }                                                                         \
    for (int64_t i = done + gid; i < n; i += stride) CALL(1, i);              \
  }

template <typename T>
__global__ void __launch_bounds__(kCgBlock) cg_persistent_kernel(const CgParams<T> p, int vec) {
  using Acc = typename AccOf<T>::type;
  constexpr int VW = 16 / (int)sizeof(T);
  __shared__ double smem[kMaxBlock];
  const int64_t n = p.n;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const unsigned long long G = gridDim.x;
  unsigned long long target = 0;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;

  // start: r = b - d*x, rho_0 = r.r
  Acc acc;
#define SALT_CG_START(W, J) start_w<T, W>(p, J, acc)
  SALT_CG_EACH(SALT_CG_START)
#undef SALT_CG_START
  double rho = 0.0, rho_prev = 0.0, pq = 0.0;
  target += G;
  if (!grid_sum<T>(acc.value(), p.partials, 0, p.counter, p.status, target, p.max_polls, smem, &rho)) {
    if (lead) p.rho[0] = NAN;
    return;
  }
  if (lead) p.rho[0] = rho;

  for (int k = 0; k < p.iters; ++k) {
    // pass 1: p = r (k = 0) or r + beta p; q = d*p; pq = p.q
    const bool first = k == 0;
    const T beta = first ? T(0) : Arith<T>::div((T)rho, (T)rho_prev);
    Acc a1;
#define SALT_CG_PASS1(W, J) pass1_w<T, W>(p, J, first, beta, a1)
    SALT_CG_EACH(SALT_CG_PASS1)
#undef SALT_CG_PASS1
    target += G;
    if (!grid_sum<T>(a1.value(), p.partials, 1, p.counter, p.status, target, p.max_polls, smem, &pq)) {
      if (lead) p.rho[0] = NAN;
      return;
    }
    if (lead) p.rho[2 * k + 1] = pq;
    // pass 2: x = x + alpha p; r = r - alpha q; rho' = r.r
    const T alpha = Arith<T>::div((T)rho, (T)pq);
    Acc a2;
#define SALT_CG_PASS2(W, J) pass2_w<T, W>(p, J, alpha, a2)
    SALT_CG_EACH(SALT_CG_PASS2)
#undef SALT_CG_PASS2
    double rho_next = 0.0;
    target += G;
    if (!grid_sum<T>(a2.value(), p.partials, 0, p.counter, p.status, target, p.max_polls, smem, &rho_next)) {
      if (lead) p.rho[0] = NAN;
      return;
    }
    if (lead) p.rho[2 * k + 2] = rho_next;
    rho_prev = rho;
    rho = rho_next;
  }
}
// Conjugate gradients with one reduction phase per iteration (Chronopoulos
// and Gear): each iteration is one pass -- p = r + beta p, s = d o r +
// beta s, x = x + alpha p, r = r - alpha s, and gamma = r.r, delta =
// (d o r).r of the new residual -- and one grid barrier; every block then
// computes beta = gamma / gamma_prev and alpha = gamma / (delta - beta gamma
// / alpha_prev) in T from the totals rounded to T.  The partials of
// consecutive iterations alternate between slots {0, 1} and {2, 3}, so a
// block that has moved on never overwrites sums another block still reads.
// History: rho[0] = gamma_0, rho[1] = delta_0, rho[2k+2] = gamma_{k+1},
// rho[2k+3] = delta_{k+1}.
template <typename T>
__global__ void __launch_bounds__(kCgBlock) cg_one_reduction_kernel(const CgParams<T> p, int vec) {
  using Acc = typename AccOf<T>::type;
  constexpr int VW = 16 / (int)sizeof(T);
  __shared__ double smem[kMaxBlock];
  const int64_t n = p.n;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const unsigned long long G = gridDim.x;
  unsigned long long target = 0;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;

  Acc ag, ad;
#define SALT_CGC_START(W, J) cgc_start_w<T, W>(p, J, ag, ad)
  SALT_CG_EACH(SALT_CGC_START)
#undef SALT_CGC_START
  double gamma = 0.0, delta = 0.0;
  target += G;
  if (!grid_sum2(ag.value(), ad.value(), p.partials, 0, p.counter, p.status, target, p.max_polls, smem, &gamma,
                 &delta)) {
    if (lead) p.rho[0] = NAN;
    return;
  }
  if (lead) {
    p.rho[0] = gamma;
    p.rho[1] = delta;
  }
  T alpha = T(0), beta = T(0);
  double gamma_prev = 0.0;
  for (int k = 0; k < p.iters; ++k) {
    const bool first = k == 0;
    const T g = (T)gamma, dl = (T)delta;
    if (first) {
      alpha = Arith<T>::div(g, dl);
    } else {
      beta = Arith<T>::div(g, (T)gamma_prev);
      alpha = Arith<T>::div(g, Arith<T>::sub(dl, Arith<T>::div(Arith<T>::mul(beta, g), alpha)));
    }
    Acc bg, bd;
#define SALT_CGC_PASS(W, J) cgc_pass_w<T, W>(p, J, first, beta, alpha, bg, bd)
    SALT_CG_EACH(SALT_CGC_PASS)
#undef SALT_CGC_PASS
    double gn = 0.0, dn = 0.0;
    target += G;
    if (!grid_sum2(bg.value(), bd.value(), p.partials, (k & 1) ? 0 : 2, p.counter, p.status, target, p.max_polls,
                   smem, &gn, &dn)) {
      if (lead) p.rho[0] = NAN;
      return;
    }
    if (lead) {
      p.rho[2 * k + 2] = gn;
      p.rho[2 * k + 3] = dn;
    }
    gamma_prev = gamma;
    gamma = gn;
    delta = dn;
  }
}
#undef SALT_CG_EACH

template <typename T>
salt_status launch_cg(int64_t n, void* const* v, int32_t iters, double* rho, cudaStream_t s,
                      bool one_reduction) {
  double* partials = nullptr;
  unsigned* words = nullptr;
  int cap = 0;
  salt_status st = stream_workspace(s, &partials, &words, &cap);
  if (st != SALT_OK) return st;
  int dev = 0, sms = 0;
  st = current_device(&dev, &sms);
  if (st != SALT_OK) return st;
  const void* kern = one_reduction ? (const void*)cg_one_reduction_kernel<T> : (const void*)cg_persistent_kernel<T>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgBlock, 0);
  if (e != cudaSuccess || per_sm < 1) return report_error(SALT_ERR_CUDA, "occupancy of the CG kernel");
  // one block per 4 tiles of the block's width, at most all resident blocks
  int64_t want = (n + 4 * kCgBlock - 1) / (4 * kCgBlock);
  int64_t cap_blocks = (int64_t)sms * per_sm;
  const int slots = one_reduction ? 4 : 2;  // partial slots per block
  if (cap_blocks > cap / slots) cap_blocks = cap / slots;
  const int grid = (int)(want < 1 ? 1 : (want < cap_blocks ? want : cap_blocks));
  // words[0] is the reduction ticket; words[1] = status, words[2..3] = the
  // 64-bit barrier counter (8-byte aligned: the slot is 256-byte aligned)
  e = cudaMemsetAsync(words + 1, 0, 3 * sizeof(unsigned), s);
  if (e != cudaSuccess) return report_error(SALT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  CgParams<T> prm{(const T*)v[0], (const T*)v[5], (T*)v[3], (T*)v[4], (T*)v[1], (T*)v[2],
                  n, iters, rho, partials, (unsigned long long*)(words + 2), words + 1,
                  g_barrier_polls.load()};
  int vec = 1;
  for (int k = 0; k < 6; ++k) vec = vec && ((uintptr_t)v[k] % 16 == 0);
  void* args[] = {&prm, &vec};
  e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kCgBlock), args, 0, s);
  count_launch();
  if (e != cudaSuccess)
    return report_error(SALT_ERR_CUDA, std::string("cooperative CG launch: ") + cudaGetErrorString(e));
  return SALT_OK;
}

}  // namespace

unsigned cg_barrier_polls(int64_t set) {
  if (set >= 0) g_barrier_polls.store((unsigned)set);
  return g_barrier_polls.load();
}

}  // namespace salt

using namespace salt;

extern "C" salt_status salt_cg_status(void* stream) {
  const cudaStream_t s = (cudaStream_t)stream;
  double* partials = nullptr;
  unsigned* words = nullptr;
  int cap = 0;
  salt_status st = stream_workspace(s, &partials, &words, &cap);
  if (st != SALT_OK) return st;
  unsigned status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, words + 1, sizeof status, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report_error(SALT_ERR_CUDA, std::string("reading the CG status: ") + cudaGetErrorString(e));
  if (status != 0u)
    return report_error(SALT_ERR_TIMEOUT, "a grid barrier of the last cooperative CG launch on this stream ran out "
                                          "of its poll limit; rho[0] is NaN and x, r, p, q are not valid");
  return SALT_OK;
}

extern "C" salt_status salt_cg_diag_persistent(int32_t dtype, int64_t n, const void* d, const void* b, void* x,
                                               void* r, void* p, void* q, int32_t iters, double* rho,
                                               void* stream) {
  void* vecs[6] = {const_cast<void*>(d), p, q, x, r, const_cast<void*>(b)};
  const cudaStream_t s = (cudaStream_t)stream;
  salt_status st = cg_validate(dtype, n, vecs, iters, rho, s);
  if (st != SALT_OK) return st;
  return dtype == SALT_F32 ? launch_cg<float>(n, vecs, iters, rho, s, false)
                           : launch_cg<double>(n, vecs, iters, rho, s, false);
}

extern "C" salt_status salt_cg_diag_one_reduction(int32_t dtype, int64_t n, const void* d, const void* b, void* x,
                                                  void* r, void* p, void* s_, int32_t iters, double* rho,
                                                  void* stream) {
  void* vecs[6] = {const_cast<void*>(d), p, s_, x, r, const_cast<void*>(b)};
  const cudaStream_t s = (cudaStream_t)stream;
  salt_status st = cg_validate(dtype, n, vecs, iters, rho, s);
  if (st != SALT_OK) return st;
  return dtype == SALT_F32 ? launch_cg<float>(n, vecs, iters, rho, s, true)
                           : launch_cg<double>(n, vecs, iters, rho, s, true);
}

// ------------------------------------------------------------------------
// salt_cg_diag_auto: the form chosen per (dtype, log2 n) bucket.  Defaults
// from per-iteration times measured on GB300 (100 iterations, n = 2^14 ..
// 2^24, and 16 iterations at 2^28): the one-reduction form wins wherever
// launches or barriers dominate and for FP32 at large n (9 vector passes
// per iteration instead of 11); for FP64 at large n the two-pass form wins,
// because the one-reduction pass needs more FP64 instructions per element
// and FP64 kernels are bound by the FP64 pipe; around n = 2^20 FP32 the
// forms tie and the two-pass form is kept.
namespace salt {
namespace {

std::mutex g_form_mu;
std::map<std::pair<int, int>, int> g_form;  // (dtype, bucket) -> SALT_CG_*

int log2_bucket(int64_t n) {
  int b = 0;
  while (b < 62 && (int64_t(1) << (b + 1)) <= n) ++b;
  return b;
}

int default_form(int32_t dtype, int64_t n) {
  const int b = log2_bucket(n);
  if (dtype == SALT_F64) return b < 19 ? SALT_CG_ONE_REDUCTION : SALT_CG_TWO_PASS;
  return (b >= 19 && b < 22) ? SALT_CG_TWO_PASS : SALT_CG_ONE_REDUCTION;
}

int form_for(int32_t dtype, int64_t n) {
  std::lock_guard<std::mutex> lk(g_form_mu);
  auto it = g_form.find(std::make_pair((int)dtype, log2_bucket(n)));
  return it != g_form.end() ? it->second : default_form(dtype, n);
}

salt_status run_form(int form, int32_t dtype, int64_t n, const void* d, const void* b, void* x, void* r, void* p,
                     void* q, int32_t iters, double* rho, void* stream) {
  if (form == SALT_CG_PERSISTENT) return salt_cg_diag_persistent(dtype, n, d, b, x, r, p, q, iters, rho, stream);
  if (form == SALT_CG_ONE_REDUCTION) return salt_cg_diag_one_reduction(dtype, n, d, b, x, r, p, q, iters, rho, stream);
  return salt_cg_diag(dtype, n, d, b, x, r, p, q, iters, rho, stream);
}

bool form_valid(int32_t form) {
  return form == SALT_CG_TWO_PASS || form == SALT_CG_PERSISTENT || form == SALT_CG_ONE_REDUCTION;
}

}  // namespace
}  // namespace salt

extern "C" salt_status salt_cg_form_set(int32_t dtype, int64_t n, int32_t form) {
  if (dtype != SALT_F32 && dtype != SALT_F64) return report_error(SALT_ERR_DTYPE, "dtype must be SALT_F32 or SALT_F64");
  if (n < 0) return report_error(SALT_ERR_ARG, "n must be >= 0");
  std::lock_guard<std::mutex> lk(g_form_mu);
  const auto key = std::make_pair((int)dtype, log2_bucket(n));
  if (form < 0) {
    g_form.erase(key);  // back to the default
    return SALT_OK;
  }
  if (!form_valid(form)) return report_error(SALT_ERR_ARG, "unknown CG form");
  g_form[key] = form;
  return SALT_OK;
}

extern "C" salt_status salt_cg_form_get(int32_t dtype, int64_t n, int32_t* form) {
  if (dtype != SALT_F32 && dtype != SALT_F64) return report_error(SALT_ERR_DTYPE, "dtype must be SALT_F32 or SALT_F64");
  if (!form) return report_error(SALT_ERR_ARG, "form is NULL");
  *form = form_for(dtype, n < 0 ? 0 : n);
  return SALT_OK;
}

extern "C" salt_status salt_cg_diag_auto(int32_t dtype, int64_t n, const void* d, const void* b, void* x, void* r,
                                         void* p, void* q, int32_t iters, double* rho, int32_t* form_used,
                                         void* stream) {
  if (dtype != SALT_F32 && dtype != SALT_F64) return report_error(SALT_ERR_DTYPE, "dtype must be SALT_F32 or SALT_F64");
  const int form = form_for(dtype, n < 0 ? 0 : n);
  if (form_used) *form_used = form;
  return run_form(form, dtype, n, d, b, x, r, p, q, iters, rho, stream);
}

extern "C" salt_status salt_cg_autotune(int32_t dtype, int64_t n, const void* d, const void* b, void* x, void* r,
                                        void* p, void* q, int32_t iters, double* rho, int32_t reps,
                                        int32_t* best_form, double* best_ms, void* stream) {
  if (dtype != SALT_F32 && dtype != SALT_F64) return report_error(SALT_ERR_DTYPE, "dtype must be SALT_F32 or SALT_F64");
  if (reps < 1 || reps > 1000) return report_error(SALT_ERR_ARG, "reps must be in [1, 1000]");
  if (n < 0) return report_error(SALT_ERR_ARG, "n must be >= 0");
  const cudaStream_t s = (cudaStream_t)stream;
  // every form is validated (and its workspace created) before anything runs
  void* vecs[6] = {const_cast<void*>(d), p, q, x, r, const_cast<void*>(b)};
  salt_status st = cg_validate(dtype, n, vecs, iters, rho, s);
  if (st != SALT_OK) return st;
  const size_t bytes = (size_t)n * (dtype == SALT_F32 ? 4 : 8);
  void* x0 = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = bytes ? cudaMalloc(&x0, bytes) : cudaSuccess;
  if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(x0, x, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int best = -1;
  float best_t = 0.f;
  for (int form = SALT_CG_TWO_PASS; form <= SALT_CG_ONE_REDUCTION && e == cudaSuccess && st == SALT_OK; ++form) {
    float total = 0.f;
    for (int k = 0; k <= reps && e == cudaSuccess && st == SALT_OK; ++k) {  // k = 0: warm-up
      if (bytes) e = cudaMemcpyAsync(x, x0, bytes, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) st = run_form(form, dtype, n, d, b, x, r, p, q, iters, rho, stream);
      if (e == cudaSuccess && st == SALT_OK) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess && st == SALT_OK) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess && st == SALT_OK) e = cudaEventElapsedTime(&ms, e0, e1);
      if (k > 0) total += ms;
    }
    if (e == cudaSuccess && st == SALT_OK && (best < 0 || total < best_t)) {
      best = form;
      best_t = total;
    }
  }
  // x is given back as the caller passed it
  if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(x, x0, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (x0) cudaFree(x0);
  if (st != SALT_OK) return st;
  if (e != cudaSuccess) return report_error(SALT_ERR_CUDA, std::string("CG autotuner: ") + cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lk(g_form_mu);
    g_form[std::make_pair((int)dtype, log2_bucket(n))] = best;
  }
  if (best_form) *best_form = best;
  if (best_ms) *best_ms = best_t / reps;
  return SALT_OK;
}
