// salt_dot_noalloc: a dot product that allocates no device memory.
//
// salt_dot keeps its per-block partial sums in a workspace that the library
// allocates with cudaMalloc on the first reducing call on a stream.  Some
// callers cannot let a library allocate: runtimes that reserve all device
// memory up front under a fixed budget, and latency-critical loops where
// cudaMalloc's implicit device synchronisation is unacceptable.  This entry
// point serves them: its scratch is a file-scope static device array of fixed
// size that exists, on every GPU that loads the library, from module load
// until process exit.  The first call on a device looks up the array's
// device address (set-up); make that call before any stream capture.
//
// The scratch holds a ticket word and one FP64 partial per span of
// kSpan = 65536 elements, kMaxSpans = 4096 spans in all (32 KiB + 256 B), so
// n is limited to kMaxSpans * kSpan = 2^28 elements; larger n is rejected.
// Every call shares the array; calls that overlap on the GPU (e.g. on two
// streams at once) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/salt.h"
#include "common.cuh"

namespace salt {
salt_status report_error(salt_status st, const std::string& msg);  // api.cu: salt_last_error()
namespace {

constexpr int64_t kSpan = 65536;
constexpr int kMaxSpans = 4096;
constexpr int kTicketBytes = 256;
constexpr size_t kScratchBytes = kTicketBytes + sizeof(double) * kMaxSpans;
constexpr int kBlock = 256;

// The scratch: [ticket (first 4 bytes of a 256-byte slot)][partials].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// One block per span of kSpan elements: the block's threads accumulate with
// the same accumulators as salt_dot (compensated FP32 / FP64 FMA), fold into
// one FP64 partial, and the last block adds the partials in span order.
template <typename T>
__global__ void __launch_bounds__(kBlock) dot_span_kernel(const T* __restrict__ x, const T* __restrict__ y,
                                                           int64_t n, double* out, unsigned char* scratch) {
  constexpr int VEC = 16 / (int)sizeof(T);
  using V = VecT<T, 16>;
  using Acc = typename AccOf<T>::type;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + kTicketBytes);
  const int64_t begin = (int64_t)blockIdx.x * kSpan;
  const int64_t end = begin + kSpan < n ? begin + kSpan : n;
  Acc acc;
  for (int64_t i = begin + (int64_t)threadIdx.x * VEC; i < end; i += (int64_t)blockDim.x * VEC) {
    if (i + VEC <= end) {
      V a, b;
      vload<true>(a, x + i);
      vload<true>(b, y + i);
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc.add_prod(a.e[e], b.e[e]);
    } else {
      for (int64_t j = i; j < end; ++j) acc.add_prod(x[j], y[j]);
    }
  }
  __shared__ double smem[kMaxBlock];
  double vals[1] = {acc.value()};
  if (grid_combine<double, 1>(vals, partials, ticket, smem) && threadIdx.x == 0) *out = vals[0];
}

std::mutex g_mu;
void* g_scratch_addr[256];  // per device ordinal, filled at set-up

salt_status fail(salt_status st, const std::string& m) { return report_error(st, m); }

// Set-up, once per device, with that device current: look up the device
// address of the static scratch array (the host-side symbol is only a
// stand-in and must never be handed to a kernel).
salt_status scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 256) return fail(SALT_ERR_ARG, "device ordinal out of range");
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(SALT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SALT_OK;
}

}  // namespace
}  // namespace salt

using namespace salt;

extern "C" salt_status salt_dot_noalloc(int32_t dtype, int64_t n, const void* x, const void* y, double* out,
                                        void* stream) {
  if (dtype != SALT_F32 && dtype != SALT_F64) return fail(SALT_ERR_DTYPE, "dtype must be SALT_F32 or SALT_F64");
  if (n < 0) return fail(SALT_ERR_ARG, "n must be >= 0");
  if (n > (int64_t)kMaxSpans * kSpan)
    return fail(SALT_ERR_BUDGET, "n exceeds the static scratch capacity of salt_dot_noalloc: at most 2^28 "
                                 "(268435456) elements (4096 spans of 65536)");
  if (!out) return fail(SALT_ERR_ARG, "out is NULL");
  if (((uintptr_t)out) % 8) return fail(SALT_ERR_ALIGN, "out must be 8-byte aligned");
  if (n > 0 && (!x || !y)) return fail(SALT_ERR_ARG, "x or y is NULL");
  if (((uintptr_t)x) % 16 || ((uintptr_t)y) % 16) return fail(SALT_ERR_ALIGN, "x and y must be 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SALT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    e = cudaMemsetAsync(out, 0, sizeof(double), s);
    return e == cudaSuccess ? SALT_OK : fail(SALT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  void* scratch = nullptr;
  salt_status st = scratch_address(dev, &scratch);
  if (st != SALT_OK) return st;
  // The ticket must be zero when the kernel starts; the array keeps whatever
  // the previous call (or an interrupted one) left, so clear it first.
  e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return fail(SALT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const int grid = (int)((n + kSpan - 1) / kSpan);
  if (dtype == SALT_F32)
    dot_span_kernel<float><<<grid, kBlock, 0, s>>>((const float*)x, (const float*)y, n, out, (unsigned char*)scratch);
  else
    dot_span_kernel<double><<<grid, kBlock, 0, s>>>((const double*)x, (const double*)y, n, out,
                                                    (unsigned char*)scratch);
  e = cudaGetLastError();
  return e == cudaSuccess ? SALT_OK : fail(SALT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}
