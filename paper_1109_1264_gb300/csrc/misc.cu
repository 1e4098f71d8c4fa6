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

void register_misc(Registry& r) {
  r.interp[DT_F32][0] = {&launch_interp<float, 16>, (const void*)&interp_kernel<float, 16>};
  r.interp[DT_F32][1] = {&launch_interp<float, 32>, (const void*)&interp_kernel<float, 32>};
  r.interp[DT_F64][0] = {&launch_interp<double, 16>, (const void*)&interp_kernel<double, 16>};
  r.interp[DT_F64][1] = {&launch_interp<double, 32>, (const void*)&interp_kernel<double, 32>};
  r.fill[DT_F32] = {&launch_fill<float>, (const void*)&fill_kernel<float>};
  r.fill[DT_F64] = {&launch_fill<double>, (const void*)&fill_kernel<double>};
}

}  // namespace salt
