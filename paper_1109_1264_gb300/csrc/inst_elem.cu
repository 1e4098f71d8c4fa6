// Instantiations of the element-access kernels: every shape and dtype, for
// operands that are not 16-byte aligned or not contiguous.
#include "fused.cuh"
#include "reduce.cuh"
#include "registry.h"

namespace salt {

template <class P, typename T>
static cudaError_t launch_strided(const void* prm, int grid, int block, size_t smem, cudaStream_t s) {
  strided_kernel<P, T, kElemUnroll><<<grid, block, smem, s>>>(*static_cast<const MapParams<T>*>(prm));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_nrm2_elem(const void* prm, int grid, int block, size_t smem, cudaStream_t s) {
  nrm2_elem_kernel<T><<<grid, block, smem, s>>>(*static_cast<const NrmParams*>(prm));
  return cudaGetLastError();
}

void register_elementwise(Registry& r) {
#define SALT_REG_STRIDED(name, ...)                                                                       \
  r.strided[SHAPE_##name][DT_F32] = {&launch_strided<Prog_##name, float>,                                 \
                                     (const void*)&strided_kernel<Prog_##name, float, kElemUnroll>};      \
  r.strided[SHAPE_##name][DT_F64] = {&launch_strided<Prog_##name, double>,                                \
                                     (const void*)&strided_kernel<Prog_##name, double, kElemUnroll>};
  SALT_SHAPE_LIST(SALT_REG_STRIDED)
#undef SALT_REG_STRIDED
  r.nrm2_elem[DT_F32] = {&launch_nrm2_elem<float>, (const void*)&nrm2_elem_kernel<float>};
  r.nrm2_elem[DT_F64] = {&launch_nrm2_elem<double>, (const void*)&nrm2_elem_kernel<double>};
}

}  // namespace salt
