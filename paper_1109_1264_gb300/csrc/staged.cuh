// Staged schedule of the fused loop: operand tiles arrive in shared memory
// by bulk asynchronous copies (cp.async.bulk, global -> shared, completing
// on an mbarrier) instead of register loads.
//
// Per element the work is exec_chunk's, so element results are bit-identical
// to fused_kernel's; what changes is how bytes reach the SM.  Each block is
// persistent over tiles of `stage_bytes` per loaded operand.  One thread
// issues a tile's copies (one per loaded operand) into one of two stages;
// while the block computes on one stage the copies of its next tile fill
// the other, so the bytes in flight per SM are bounded by shared memory
// rather than by registers.  Results are stored from registers with 16-byte
// vector stores.  Elements after the last whole tile take a per-element
// loop.  The autotuner chooses between this schedule and the register-tiled
// one per shape, dtype and size (Section 4.3: the loop layout is picked by
// trial on the target machine).
//
// Waits on an mbarrier are bounded.  If a tile's copies have not completed
// within kStageWaitNs (or `tile_polls` polls, kStageSpins unless a test sets
// a smaller limit), the block counts a timeout in *timeouts, stops issuing
// copies, computes that tile and every later one from direct global loads
// (so the results do not change), and before it exits waits, with the full
// bound, for the copies it still has in flight.
#pragma once

#include "fused.cuh"

namespace salt {

template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

constexpr int kStages = 2;
constexpr unsigned kStageSpins = 1u << 26;           // polls
constexpr uint64_t kStageWaitNs = 1000000000ull;     // one second of the global timer

template <typename T>
struct StagedParams {
  MapParams<T> m;
  int32_t stage_bytes;            // per loaded operand per stage: 4096, 8192 or 16384
  unsigned tile_polls;            // polls of a tile's copies before the fallback (0: none)
  unsigned long long* timeouts;   // device counter of timed-out waits
};

// Operands read from memory by P (at least one stage buffer is laid out).
template <class P>
__host__ __device__ constexpr int staged_nbuf() {
  return P::nloads() > 0 ? P::nloads() : 1;
}

// Dynamic shared memory of one block of staged_kernel<P, T>.
template <class P>
inline size_t staged_smem(int stage_bytes) {
  return (size_t)kStages * staged_nbuf<P>() * (size_t)stage_bytes;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// One arrival that also announces `bytes` of asynchronous copies to come.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// True once the phase with the given parity has completed (acquire).
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// At most `polls` tests of the phase (none when polls is 0) and at most
// kStageWaitNs of the global timer.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned polls = kStageSpins) {
  if (polls == 0u) return false;
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (unsigned k = 1; k < polls; ++k) {
    if (mbar_test(bar, parity)) return true;
    if (global_ns() - t0 > kStageWaitNs) return false;
  }
  return false;
}

// Global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) that completes its bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <class P, typename T>
__global__ void __launch_bounds__(256) staged_kernel(const StagedParams<T> sp) {
  constexpr unsigned LM = P::load_mask(), SMASK = P::store_mask();
  constexpr int NB = staged_nbuf<P>();
  constexpr int NR = P::nred();
  constexpr int VEC = 16 / (int)sizeof(T);
  using V = VecT<T, 16>;
  using Acc = typename AccOf<T>::type;
  extern __shared__ __align__(128) unsigned char stage_mem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ int s_ok;  // 1: this tile is in shared memory; 0: read it from global memory

  const MapParams<T>& p = sp.m;
  trace_mark(p.trace, TR_START);
  T sc[kMaxScals];
  load_scalars<T>(p.sc, p.scode, sc);
  Acc acc[kMaxReds];
  run_head<P, T, Acc>(p, sc, acc);

  const int64_t n = p.n;
  const int sb = sp.stage_bytes;
  const int64_t te = sb / (int64_t)sizeof(T);  // elements per operand per tile
  const int64_t ntiles = n / te;
  const int64_t gstep = gridDim.x;
  auto buf = [&](int st, int b) -> T* {
    return reinterpret_cast<T*>(stage_mem + ((size_t)st * NB + b) * (size_t)sb);
  };
  // thread 0 only: copies of `tile` into stage st
  auto issue = [&](int st, int64_t tile) {
    mbar_arrive_expect_tx(&bars[st], (unsigned)(P::nloads() * sb));
    int b = 0;
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s) {
      if ((LM >> s) & 1u) {
        bulk_g2s(buf(st, b), p.v[s] + tile * te, (unsigned)sb, &bars[st]);
        ++b;
      }
    }
  };

  // thread 0's bookkeeping: stages with copies in flight, their phase parities
  unsigned pending = 0, parity = 0;
  bool staging = true;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
    for (int st = 0; st < kStages; ++st) {
      const int64_t t = (int64_t)blockIdx.x + st * gstep;
      if (t < ntiles) {
        issue(st, t);
        pending |= 1u << st;
      }
    }
  }
  __syncthreads();

  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gstep, ++it) {
    const int st = it % kStages;
    if (threadIdx.x == 0) {
      bool ok = staging && mbar_wait_bounded(&bars[st], (parity >> st) & 1u, sp.tile_polls);
      if (ok) {
        pending &= ~(1u << st);
        parity ^= 1u << st;
      } else if (staging) {
        atomicAdd(sp.timeouts, 1ull);
        staging = false;
      }
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    // every reader acquires the completed phase for itself (returns at once)
    const bool from_smem = s_ok != 0 && mbar_wait_bounded(&bars[st], (unsigned)(it / kStages) & 1u);

    const int64_t base = tile * te;
    const int nj = (int)(te / VEC);
    // one pass over this thread's elements of the tile; FMA: the scaled adds
    // as FMAs (exec_node)
    auto run = [&](auto fma) {
      constexpr bool FMA = decltype(fma)::value;
      for (int j = threadIdx.x; j < nj; j += blockDim.x) {
        T x[kMaxVecs][VEC];
        int b = 0;
#pragma unroll
        for (int s = 0; s < kMaxVecs; ++s) {
          if ((LM >> s) & 1u) {
            V t;
            if (from_smem) t = *reinterpret_cast<const V*>(buf(st, b) + j * VEC);
            else if ((SMASK >> s) & 1u) vload<false>(t, p.v[s] + base + j * VEC);
            else vload<true>(t, p.v[s] + base + j * VEC);
#pragma unroll
            for (int e = 0; e < VEC; ++e) x[s][e] = t.e[e];
            ++b;
          } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) x[s][e] = T(0);
          }
        }
        exec_chunk<P, T, Acc, VEC, FMA>(x, sc, acc);
#pragma unroll
        for (int s = 0; s < kMaxVecs; ++s) {
          if ((SMASK >> s) & 1u) {
            V t;
#pragma unroll
            for (int e = 0; e < VEC; ++e) t.e[e] = x[s][e];
            vstore(p.v[s] + base + j * VEC, t);
          }
        }
      }
    };
    // FP64 programs without reductions whose by-value scalars include a power
    // of two (exec_chunk_p2): this thread's operands of the tile, already in
    // shared memory, are checked first, and the whole tile then runs one of
    // the two bodies, so no element computes both forms.
    bool fma_ok = false;
    if constexpr (sizeof(T) == 8 && P::nred() == 0 && P::any_scaled_add()) {
      if (from_smem && p.p2.mask != 0u) {
        fma_ok = true;
        for (int j = threadIdx.x; j < nj; j += blockDim.x) {
          T x[kMaxVecs][VEC];
          int b = 0;
#pragma unroll
          for (int s = 0; s < kMaxVecs; ++s) {
            if ((LM >> s) & 1u) {
              const V t = *reinterpret_cast<const V*>(buf(st, b) + j * VEC);
#pragma unroll
              for (int e = 0; e < VEC; ++e) x[s][e] = t.e[e];
              ++b;
            } else {
#pragma unroll
              for (int e = 0; e < VEC; ++e) x[s][e] = T(0);
            }
          }
          fma_ok = fma_ok & pow2_chunk_ok<P, 0, VEC>(x, p.p2);
        }
      }
    }
    if (fma_ok) run(BoolTag<true>{});
    else run(BoolTag<false>{});
    __syncthreads();  // stage st is free again
    if (threadIdx.x == 0 && staging && tile + kStages * gstep < ntiles) {
      issue(st, tile + kStages * gstep);
      pending |= 1u << st;
    }
  }

  // copies still in flight (only after a timeout): let them land before exit
  if (threadIdx.x == 0 && pending != 0u) {
#pragma unroll
    for (int st = 0; st < kStages; ++st)
      if ((pending >> st) & 1u) mbar_wait_bounded(&bars[st], (parity >> st) & 1u);
  }

  trace_mark(p.trace, TR_TILES);
  // elements after the last whole tile
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = gstep * blockDim.x;
  for (int64_t i = ntiles * te + gid; i < n; i += gstride) {
    T x[kMaxVecs][1];
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s) x[s][0] = ((LM >> s) & 1u) ? p.v[s][i] : T(0);
    exec_chunk<P, T, Acc, 1>(x, sc, acc);
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s)
      if ((SMASK >> s) & 1u) p.v[s][i] = x[s][0];
  }

  trace_mark(p.trace, TR_PRE_COMBINE);
  bool last = false;
  if constexpr (NR > 0) {
    __shared__ double smem[kMaxBlock];
    double vals[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) vals[r] = acc[r].value();
    last = grid_combine<double, NR>(vals, (double*)p.partials, p.ticket, smem);
    if (last && threadIdx.x == 0) {
#pragma unroll
      for (int r = 0; r < NR; ++r) p.red_out[r] = vals[r];
    }
  }
  trace_end(p.trace, last);
}

}  // namespace salt
