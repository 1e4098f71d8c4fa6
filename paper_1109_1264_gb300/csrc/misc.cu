// Instantiations of the generic interpreter and the input fill kernel.
#include "interp.cuh"
#include "reduce.cuh"
#include "registry.h"

namespace salt {

template <typename T, int VB>
static cudaError_t launch_interp(const void* prm, int grid, int block, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(interp_kernel<T, VB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  interp_kernel<T, VB><<<grid, block, smem, s>>>(*static_cast<const InterpParams<T>*>(prm));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_fill(const void* prm, int grid, int block, size_t smem, cudaStream_t s) {
  const FillParams& p = *static_cast<const FillParams*>(prm);
  fill_kernel<T><<<grid, block, smem, s>>>((T*)p.x, p.n, p.key, p.offset);
  return cudaGetLastError();
}

// Reads `n16` 16-byte words (an L2 flush that leaves clean lines behind);
// the sink is written only for a combination of values that uniformly
// random data essentially never gives, so that the reads are not removed.
__global__ void l2_flush_kernel(const uint4* p, int64_t n16, unsigned* sink) {
  unsigned acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 v = p[i];
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x9E3779B9u) *sink = acc;
}

cudaError_t launch_l2_flush(const void* buf, size_t bytes, unsigned* sink, int sms, cudaStream_t s) {
  l2_flush_kernel<<<sms * 4, 256, 0, s>>>(static_cast<const uint4*>(buf), (int64_t)(bytes / 16), sink);
  return cudaGetLastError();
}

// FP64 issue-rate probe: every thread runs 8 independent chains of one
// instruction kind from registers (0: DFMA, 1: DADD, 2: DMUL).  The sum is
// stored only for a value the chains essentially never reach, so the work
// is not removed.
__device__ double g_fp64_rate_sink;

template <int OP>
__global__ void fp64_rate_kernel(int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (double)threadIdx.x * 1e-9 + (double)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (OP == 0) a[k] = __fma_rn(a[k], b, c);
      else if (OP == 1) a[k] = __dadd_rn(a[k], c);
      else a[k] = __dmul_rn(a[k], b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 1.2345e-300) g_fp64_rate_sink = s;
}

// Times `iters` x 8 instructions per thread on 4 blocks of 256 threads per
// SM (after a short warm-up launch) with events on stream s; *gops receives
// G instructions per second.
cudaError_t fp64_rate(int op, int sms, double* gops, cudaStream_t s) {
  const int grid = sms * 4, block = 256, iters = 60000;
  void (*k)(int, double, double) = op == 0 ? &fp64_rate_kernel<0> : op == 1 ? &fp64_rate_kernel<1> : &fp64_rate_kernel<2>;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k<<<grid, block, 0, s>>>(200, 1.0000001, 1e-7);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    k<<<grid, block, 0, s>>>(iters, 1.0000001, 1e-7);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *gops = (double)grid * block * iters * 8 / (ms * 1e-3) / 1e9;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

void register_misc(Registry& r) {
  r.interp[DT_F32][0] = {&launch_interp<float, 16>, (const void*)&interp_kernel<float, 16>};
  r.interp[DT_F32][1] = {&launch_interp<float, 32>, (const void*)&interp_kernel<float, 32>};
  r.interp[DT_F64][0] = {&launch_interp<double, 16>, (const void*)&interp_kernel<double, 16>};
  r.interp[DT_F64][1] = {&launch_interp<double, 32>, (const void*)&interp_kernel<double, 32>};
  r.fill[DT_F32] = {&launch_fill<float>, (const void*)&fill_kernel<float>};
  r.fill[DT_F64] = {&launch_fill<double>, (const void*)&fill_kernel<double>};
}

}  // namespace salt
