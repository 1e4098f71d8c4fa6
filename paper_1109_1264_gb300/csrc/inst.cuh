// Instantiation helpers: one launcher per (program, dtype, unroll, width).
#pragma once

#include "fused.cuh"
#include "reduce.cuh"
#include "registry.h"

namespace salt {

template <class P, typename T, int U, int VB, bool DS = false>
cudaError_t launch_fused(const void* prm, int grid, int block, size_t smem, cudaStream_t s) {
  fused_kernel<P, T, U, VB, DS><<<grid, block, smem, s>>>(*static_cast<const MapParams<T>*>(prm));
  return cudaGetLastError();
}

template <typename T, int U, int VB, bool PLAIN>
cudaError_t launch_nrm2(const void* prm, int grid, int block, size_t smem, cudaStream_t s) {
  nrm2_kernel<T, U, VB, PLAIN><<<grid, block, smem, s>>>(*static_cast<const NrmParams*>(prm));
  return cudaGetLastError();
}

template <int U, int VB>
cudaError_t launch_dot_plain(const void* prm, int grid, int block, size_t smem, cudaStream_t s) {
  dot_plain_kernel<U, VB><<<grid, block, smem, s>>>(*static_cast<const DotParams*>(prm));
  return cudaGetLastError();
}

template <typename T, int U, int VB>
void register_unroll(Registry& r) {
  constexpr int dt = sizeof(T) == 4 ? DT_F32 : DT_F64;
  constexpr int ui = U == 1 ? 0 : U == 2 ? 1 : 2;
  constexpr int vi = VB == 16 ? 0 : 1;
#define SALT_REG_ENTRY(name, ...)                                                           \
  r.fused[SHAPE_##name][dt][ui][vi] = {&launch_fused<Prog_##name, T, U, VB>,                \
                                       (const void*)&fused_kernel<Prog_##name, T, U, VB>};
  SALT_SHAPE_LIST(SALT_REG_ENTRY)
#undef SALT_REG_ENTRY
  if constexpr (U == kDsUnroll<T>) {
#define SALT_REG_DS(name, ...)                                                       \
  r.fused_ds[SHAPE_##name][dt][vi] = {&launch_fused<Prog_##name, T, U, VB, true>,   \
                                      (const void*)&fused_kernel<Prog_##name, T, U, VB, true>};
    SALT_SHAPE_LIST(SALT_REG_DS)
#undef SALT_REG_DS
  }
  r.special[SPECIAL_NRM2][dt][ui][vi] = {&launch_nrm2<T, U, VB, false>,
                                         (const void*)&nrm2_kernel<T, U, VB, false>};
  if constexpr (dt == DT_F32) {
    r.special[SPECIAL_NRM2_PLAIN][dt][ui][vi] = {&launch_nrm2<T, U, VB, true>,
                                                 (const void*)&nrm2_kernel<T, U, VB, true>};
    r.special[SPECIAL_DOT_PLAIN][dt][ui][vi] = {&launch_dot_plain<U, VB>,
                                                (const void*)&dot_plain_kernel<U, VB>};
  }
}

template <typename T, int VB>
void register_width(Registry& r) {
  register_unroll<T, 1, VB>(r);
  register_unroll<T, 2, VB>(r);
  register_unroll<T, 4, VB>(r);
}

}  // namespace salt
