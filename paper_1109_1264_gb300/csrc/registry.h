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
  KernelEntry staged[NUM_SHAPES][2];   // staged_kernel<P, T>: params StagedParams<T>
  size_t (*staged_smem[NUM_SHAPES])(int stage_bytes);  // its dynamic shared memory
};

Registry& registry();

// Filled by the instantiation translation units.
void register_f32_vb16(Registry&);
void register_f32_vb32(Registry&);
void register_f64_vb16(Registry&);
void register_f64_vb32(Registry&);
void register_misc(Registry&);
void register_elementwise(Registry&);
void register_staged(Registry&);

// Reads `bytes` of `buf` on `s` (16-byte multiple) so that L2 holds other,
// clean lines afterwards; one word of `sink` may be written.
cudaError_t launch_l2_flush(const void* buf, size_t bytes, unsigned* sink, int sms, cudaStream_t s);
// Register-only FP64 issue rate of one instruction kind (0 DFMA, 1 DADD, 2 DMUL), G instructions/s.
cudaError_t fp64_rate(int op, int sms, double* gops, cudaStream_t s);

// Timed-out stage waits of staged kernels since the library was loaded
// (synchronous read of a device counter).
cudaError_t staged_timeouts(unsigned long long* out);
// Polls a staged-loop block spends on a tile's copies before it falls back to
// direct loads; `set` >= 0 replaces the limit first.  Returns the limit.
unsigned staged_tile_polls(int64_t set);

inline int unroll_index(int u) { return u == 1 ? 0 : u == 2 ? 1 : u == 4 ? 2 : -1; }
inline int vb_index(int vb) { return vb == 16 ? 0 : vb == 32 ? 1 : -1; }
// Stage sizes of the staged schedule (bytes per loaded operand per stage).
inline bool stage_bytes_valid(int sb) { return sb == 0 || sb == 4096 || sb == 8192 || sb == 16384; }

}  // namespace salt
