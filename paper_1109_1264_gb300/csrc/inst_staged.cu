// Instantiations of the staged schedule (staged.cuh): every shape and dtype.
#include <atomic>
#include <mutex>

#include "registry.h"
#include "staged.cuh"

namespace salt {

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_counter_mu;
unsigned long long* g_counter[kMaxDevices];  // per device: timed-out stage waits
std::atomic<unsigned> g_tile_polls{kStageSpins};  // polls of a tile's copies (tests lower it)

// The current device's counter, allocated and zeroed on first use.
cudaError_t counter_address(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_counter_mu);
  if (!g_counter[dev]) {
    void* p = nullptr;
    e = cudaMalloc(&p, sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    e = cudaMemset(p, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
      cudaFree(p);
      return e;
    }
    g_counter[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_counter[dev];
  return cudaSuccess;
}

// The caller has raised the kernel's dynamic shared-memory limit to `smem`.
template <class P, typename T>
cudaError_t launch_staged(const void* prm, int grid, int block, size_t smem, cudaStream_t s) {
  static_assert(kStages * staged_nbuf<P>() * 16384 + 4096 <= 227 * 1024, "stages exceed shared memory");
  StagedParams<T> sp = *static_cast<const StagedParams<T>*>(prm);
  cudaError_t e = counter_address(&sp.timeouts);
  if (e != cudaSuccess) return e;
  sp.tile_polls = g_tile_polls.load();
  staged_kernel<P, T><<<grid, block, smem, s>>>(sp);
  return cudaGetLastError();
}

template <class P>
size_t smem_of(int stage_bytes) {
  return staged_smem<P>(stage_bytes);
}

}  // namespace

void register_staged(Registry& r) {
#define SALT_REG_STAGED(name, ...)                                                                  \
  r.staged[SHAPE_##name][DT_F32] = {&launch_staged<Prog_##name, float>,                             \
                                    (const void*)&staged_kernel<Prog_##name, float>};               \
  r.staged[SHAPE_##name][DT_F64] = {&launch_staged<Prog_##name, double>,                            \
                                    (const void*)&staged_kernel<Prog_##name, double>};              \
  r.staged_smem[SHAPE_##name] = &smem_of<Prog_##name>;
  SALT_SHAPE_LIST(SALT_REG_STAGED)
#undef SALT_REG_STAGED
}

unsigned staged_tile_polls(int64_t set) {
  if (set >= 0) g_tile_polls.store((unsigned)set);
  return g_tile_polls.load();
}

cudaError_t staged_timeouts(unsigned long long* out) {
  unsigned long long* c = nullptr;
  cudaError_t e = counter_address(&c);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(out, c, sizeof *out, cudaMemcpyDeviceToHost);
}

}  // namespace salt
