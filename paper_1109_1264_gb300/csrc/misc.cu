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

void register_misc(Registry& r) {
  r.interp[DT_F32][0] = {&launch_interp<float, 16>, (const void*)&interp_kernel<float, 16>};
  r.interp[DT_F32][1] = {&launch_interp<float, 32>, (const void*)&interp_kernel<float, 32>};
  r.interp[DT_F64][0] = {&launch_interp<double, 16>, (const void*)&interp_kernel<double, 16>};
  r.interp[DT_F64][1] = {&launch_interp<double, 32>, (const void*)&interp_kernel<double, 32>};
  r.fill[DT_F32] = {&launch_fill<float>, (const void*)&fill_kernel<float>};
  r.fill[DT_F64] = {&launch_fill<double>, (const void*)&fill_kernel<double>};
}

}  // namespace salt
