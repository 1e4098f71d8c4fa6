// Table of instantiated kernels: the "execute function" of the paper's
// Section 4.1 / Figure 2 selects one of these loop templates per call.
#pragma once

#include <cuda_runtime.h>

#include "shapes.h"

namespace salt {

// Launches a kernel with a parameter block of the kernel's own type.
using LaunchFn = cudaError_t (*)(const void* params, int grid, int block, size_t smem,
                                 cudaStream_t stream);

struct KernelEntry {
  LaunchFn launch = nullptr;
  const void* kernel = nullptr;  // for occupancy queries
};

enum : int { DT_F32 = 0, DT_F64 = 1 };

// Special (non-program) kernels.
enum SpecialId : int { SPECIAL_NRM2 = 0, SPECIAL_NRM2_PLAIN, SPECIAL_DOT_PLAIN, NUM_SPECIAL };

// Unroll of the element-access kernels (operands unaligned or strided).
constexpr int kElemUnroll = 4;

// Unroll of the fused kernels that compute scalar slots on the device (one
// instantiation per shape, dtype and width; the tuned F32 / F64 defaults).
template <typename T> constexpr int kDsUnroll = sizeof(T) == 4 ? 4 : 2;

struct Registry {
  KernelEntry fused[NUM_SHAPES][2][kNumUnroll][kNumVB];
  KernelEntry fused_ds[NUM_SHAPES][2][kNumVB];  // device scalar slots, unroll kDsUnroll
  KernelEntry special[NUM_SPECIAL][2][kNumUnroll][kNumVB];
  KernelEntry interp[2][kNumVB];
  KernelEntry fill[2];
  KernelEntry strided[NUM_SHAPES][2];  // strided_kernel<P, T, kElemUnroll>
  KernelEntry nrm2_elem[2];            // nrm2_elem_kernel<T>
};

Registry& registry();

// Filled by the instantiation translation units.
void register_f32_vb16(Registry&);
void register_f32_vb32(Registry&);
void register_f64_vb16(Registry&);
void register_f64_vb32(Registry&);
void register_misc(Registry&);
void register_elementwise(Registry&);

inline int unroll_index(int u) { return u == 1 ? 0 : u == 2 ? 1 : u == 4 ? 2 : -1; }
inline int vb_index(int vb) { return vb == 16 ? 0 : vb == 32 ? 1 : -1; }

}  // namespace salt
