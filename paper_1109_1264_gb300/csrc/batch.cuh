// Batched persistent evaluation: thousands of independent, uneven-length
// expression items in ONE launch.
//
// The host lays every item out as a run of fixed-size tiles (tile_bytes per
// operand) and writes a table of items with the first global tile of each.
// Resident blocks pull global tile numbers from an atomic counter (no
// waiting), find the owning item by binary search, and run that item's
// compiled program on the tile's element range -- the same per-element
// operations as the single-expression kernels, so elementwise results are
// bit-identical to them.  Reductions: each tile's block folds its partial sum
// into partials[tile]; the block that finishes an item's last tile (per-item
// ticket) adds the item's partials in tile order and writes the result.  The
// summation order therefore depends only on the item's length and the tile
// size, never on which block ran which tile or on the other items in the
// launch.
#pragma once

#include "fused.cuh"
#include "reduce.cuh"
#include "registry.h"
#include "shapes.h"

namespace salt {

constexpr int kBatchOps = 5;       // operands per item (largest shape: E)
constexpr int kBatchPartials = 3;  // FP64 partial values per tile
constexpr int32_t kKindNrm2 = -1;  // item kind: Euclidean norm (else shape id)
constexpr int32_t kKindFill = -2;  // item kind: counter-based uniform fill of v[0]
                                   // with the key stored in the bits of sc[0]

struct BatchItem {
  int32_t kind;       // shape id, or kKindNrm2
  int32_t dtype;      // DT_F32 / DT_F64
  int64_t n;          // elements
  int64_t tile_begin; // first global tile of this item
  int32_t ntiles;     // >= 1 (an empty item still owns one empty tile)
  int32_t red_index;  // first result slot in red_out, or -1
  void* v[kBatchOps]; // canonical operands
  double sc[2];       // scalars (rounded to float for F32 items)
};

struct BatchHeader {
  int32_t nitems;
  int32_t narrow;      // 1: 16-byte accesses only; 0: 32-byte accesses for 32-byte aligned FP32 items
  int64_t total_tiles;
  int64_t tile_bytes;  // bytes per operand per tile (multiple of 16 * block * unroll)
};

struct BatchParams {
  const BatchHeader* hdr;
  const BatchItem* items;
  unsigned* counter;  // global tile counter; zero at launch
  unsigned* exits;    // blocks that have finished; zero at launch
  unsigned* tickets;  // per-item tile tickets; zero at launch
  double* partials;   // kBatchPartials per global tile
  double* red_out;    // device or mapped pinned host memory
};

// One block evaluates program P on elements [lo, hi) of an item: whole
// sub-tiles of U vectors per thread (load burst, op burst, store burst), then
// single vectors, then single elements.
template <class P, typename T, int U, int VB = 16, bool NC = true>
__device__ __forceinline__ void range_eval(T* const* v, const T (&sc)[kMaxScals], int64_t lo, int64_t hi,
                                           typename AccOf<T>::type (&acc)[kMaxReds]) {
  constexpr int VEC = VB / (int)sizeof(T);
  constexpr unsigned LM = P::load_mask(), SMASK = P::store_mask();
  using Acc = typename AccOf<T>::type;
  using V = VecT<T, VB>;
  const int64_t bd = blockDim.x;
  const int64_t SUB = (int64_t)U * bd * VEC;
  const int64_t nsub = (hi - lo) / SUB;
  for (int64_t s = 0; s < nsub; ++s) {
    const int64_t base = lo + s * SUB + (int64_t)threadIdx.x * VEC;
    T x[kMaxVecs][U * VEC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int k = 0; k < kMaxVecs; ++k) {
        if ((LM >> k) & 1u) {
          V t;
          if (NC && !((SMASK >> k) & 1u)) vload<true>(t, v[k] + base + u * bd * VEC);
          else vload<false>(t, v[k] + base + u * bd * VEC);
#pragma unroll
          for (int e = 0; e < VEC; ++e) x[k][u * VEC + e] = t.e[e];
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) x[k][u * VEC + e] = T(0);
        }
      }
    }
    exec_chunk<P, T, Acc, U * VEC>(x, sc, acc);
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int k = 0; k < kMaxVecs; ++k) {
        if ((SMASK >> k) & 1u) {
          V t;
#pragma unroll
          for (int e = 0; e < VEC; ++e) t.e[e] = x[k][u * VEC + e];
          vstore(v[k] + base + u * bd * VEC, t);
        }
      }
    }
  }
  const int64_t rlo = lo + nsub * SUB;
  const int64_t nvr = (hi - rlo) / VEC;
  for (int64_t j = threadIdx.x; j < nvr; j += bd) {
    const int64_t off = rlo + j * VEC;
    T x[kMaxVecs][VEC];
#pragma unroll
    for (int k = 0; k < kMaxVecs; ++k) {
      if ((LM >> k) & 1u) {
        V t;
        if (NC && !((SMASK >> k) & 1u)) vload<true>(t, v[k] + off);
        else vload<false>(t, v[k] + off);
#pragma unroll
        for (int e = 0; e < VEC; ++e) x[k][e] = t.e[e];
      } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) x[k][e] = T(0);
      }
    }
    exec_chunk<P, T, Acc, VEC>(x, sc, acc);
#pragma unroll
    for (int k = 0; k < kMaxVecs; ++k) {
      if ((SMASK >> k) & 1u) {
        V t;
#pragma unroll
        for (int e = 0; e < VEC; ++e) t.e[e] = x[k][e];
        vstore(v[k] + off, t);
      }
    }
  }
  for (int64_t i = rlo + nvr * VEC + threadIdx.x; i < hi; i += bd) {
    T x[kMaxVecs][1];
#pragma unroll
    for (int k = 0; k < kMaxVecs; ++k) x[k][0] = ((LM >> k) & 1u) ? v[k][i] : T(0);
    exec_chunk<P, T, Acc, 1>(x, sc, acc);
#pragma unroll
    for (int k = 0; k < kMaxVecs; ++k)
      if ((SMASK >> k) & 1u) v[k][i] = x[k][0];
  }
}

// Program item: returns the number of partial values produced (its
// reductions) in vals.
// NC = false: no read-only (non-coherent) loads, for a kernel that also
// writes the data it reads (the persistent serving kernel).
template <class P, typename T, int U, bool NC = true>
__device__ __forceinline__ int item_program(const BatchItem& it, int64_t lo, int64_t hi, double (&vals)[kBatchPartials],
                                            bool narrow) {
  T* v[kMaxVecs];
#pragma unroll
  for (int k = 0; k < kMaxVecs; ++k) v[k] = k < kBatchOps ? (T*)it.v[k] : nullptr;
  T sc[kMaxScals];
#pragma unroll
  for (int k = 0; k < kMaxScals; ++k) sc[k] = k < 2 ? (T)it.sc[k] : T(0);
  typename AccOf<T>::type acc[kMaxReds];
  // FP32 items: 32-byte accesses (at half the unroll: the same bytes in
  // flight) when every operand is 32-byte aligned and the batch allows them
  // (its vector width, a tuning parameter), else 16-byte accesses.  (FP64
  // items are bound by the FP64 pipe; 32-byte accesses measured no better
  // there.)
  uintptr_t align = 0;
#pragma unroll
  for (int k = 0; k < kBatchOps; ++k)
    if (k < P::nvec()) align |= (uintptr_t)it.v[k];
  if constexpr (U >= 2 && sizeof(T) == 4) {
    if (!narrow && (align & 31u) == 0) range_eval<P, T, U / 2, 32, NC>(v, sc, lo, hi, acc);
    else range_eval<P, T, U, 16, NC>(v, sc, lo, hi, acc);
  } else {
    range_eval<P, T, U, 16, NC>(v, sc, lo, hi, acc);
  }
  constexpr int NR = P::nred();
#pragma unroll
  for (int r = 0; r < NR && r < kBatchPartials; ++r) vals[r] = acc[r].value();
  return NR;
}

template <typename T, bool NC = true>
__device__ __forceinline__ int item_nrm2(const BatchItem& it, int64_t lo, int64_t hi, double (&vals)[kBatchPartials]) {
  constexpr int VEC = 16 / (int)sizeof(T);
  using V = VecT<T, 16>;
  const T* x = (const T*)it.v[0];
  if constexpr (sizeof(T) == 4) {
    Nrm2F32 acc;
    for (int64_t i = lo + (int64_t)threadIdx.x * VEC; i < hi; i += (int64_t)blockDim.x * VEC) {
      if (i + VEC <= hi) {
        V a;
        vload<NC>(a, x + i);
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc.add(a.e[e]);
      } else {
        for (int64_t j = i; j < hi; ++j) acc.add(x[j]);
      }
    }
    vals[0] = acc.value();
    return 1;
  } else {
    Nrm2F64 acc;
    for (int64_t i = lo + (int64_t)threadIdx.x * VEC; i < hi; i += (int64_t)blockDim.x * VEC) {
      if (i + VEC <= hi) {
        V a;
        vload<NC>(a, x + i);
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc.add(a.e[e]);
      } else {
        for (int64_t j = i; j < hi; ++j) acc.add(x[j]);
      }
    }
    vals[0] = acc.sml;
    vals[1] = acc.med;
    vals[2] = acc.big;
    return 3;
  }
}

// Fill item: element i of v[0] is value i of the counter-based uniform stream
// (the same generator as fill_kernel), standing in for an upload.
template <typename T>
__device__ __forceinline__ int item_fill(const BatchItem& it, int64_t lo, int64_t hi) {
  T* x = (T*)it.v[0];
  const uint64_t key = (uint64_t)__double_as_longlong(it.sc[0]);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const uint64_t h = splitmix64_at(key, (uint64_t)i);
    if constexpr (sizeof(T) == 8) {
      x[i] = __dsub_rn(__dmul_rn(2.0, (double)(h >> 11) * 0x1p-53), 1.0);
    } else {
      x[i] = __fsub_rn(__fmul_rn(2.0f, (float)(uint32_t)(h >> 40) * 0x1p-24f), 1.0f);
    }
  }
  return 0;
}

template <typename T, int U, bool NC = true>
__device__ __forceinline__ int dispatch_item(const BatchItem& it, int64_t lo, int64_t hi, double (&vals)[kBatchPartials],
                                             bool narrow) {
  switch (it.kind) {
#define SALT_BATCH_CASE(name, ...) \
  case SHAPE_##name:               \
    return item_program<Prog_##name, T, U, NC>(it, lo, hi, vals, narrow);
    SALT_BATCH_SHAPE_LIST(SALT_BATCH_CASE)
#undef SALT_BATCH_CASE
    case kKindFill:
      return item_fill<T>(it, lo, hi);
    default:
      return item_nrm2<T, NC>(it, lo, hi, vals);
  }
}

// Index of the item that owns global tile t: the last item whose
// tile_begin <= t.  Warp 0 searches 32 ways at a time (one probe per lane, a
// ballot picks the sub-range), so 4096 items take 3 dependent loads instead
// of 12.  Called by all 32 lanes of warp 0, converged.
__device__ __forceinline__ int find_item(const BatchItem* items, int nitems, int64_t t) {
  const int lane = threadIdx.x & 31;
  int a = 0, b = nitems - 1;  // items[a].tile_begin <= t always holds
  while (a < b) {
    const int step = (b - a + 32) / 32;  // ceil((b - a + 1) / 32)
    const int k = a + lane * step;
    const bool ok = k <= b && items[k].tile_begin <= t;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    const int hi = 31 - __clz((int)m);  // bit 0 is set: k = a satisfies ok
    a += hi * step;
    const int nb = a + step - 1;
    b = nb < b ? nb : b;
  }
  return a;
}

// The tile loop of one batch launch (or of one phase of a step of the
// persistent serving kernel): tiles from p.counter until it passes the
// header's total.  Returns once this block has taken its last tile; the
// counter is then past the total, and the caller zeroes it once every block
// has returned.
template <int U, bool NC = true>
__device__ __forceinline__ void run_tiles(const BatchParams& p) {
  __shared__ int64_t s_tile;
  __shared__ int s_item;
  __shared__ bool s_last;
  __shared__ double smem[kMaxBlock];
  const int64_t total = p.hdr->total_tiles;
  const int nitems = p.hdr->nitems;
  const int64_t tile_bytes = p.hdr->tile_bytes;
  const bool narrow = p.hdr->narrow != 0;
  // Tile numbers come from an atomic counter (no waiting).  Thread 0 asks
  // for the next one when a tile starts and hands it over when the tile
  // ends, so the atomic's latency hides behind the tile's work; warp 0 then
  // finds its item.
  if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(p.counter, 1u);
  __syncthreads();
  for (;;) {
    if (threadIdx.x < 32) {
      const int64_t t = s_tile;
      const int item = t < total ? find_item(p.items, nitems, t) : 0;
      if (threadIdx.x == 0) s_item = item;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= total) break;
    const int item = s_item;
    unsigned next = 0;
    if (threadIdx.x == 0) next = atomicAdd(p.counter, 1u);
    const BatchItem it = p.items[item];
    const int64_t tile_elems = tile_bytes / (it.dtype == DT_F32 ? 4 : 8);
    const int64_t lo = (tile - it.tile_begin) * tile_elems;
    const int64_t hi = lo + tile_elems < it.n ? lo + tile_elems : it.n;
    double vals[kBatchPartials] = {0.0, 0.0, 0.0};
    const int nv = it.dtype == DT_F32 ? dispatch_item<float, U, NC>(it, lo, hi, vals, narrow)
                                      : dispatch_item<double, U, NC>(it, lo, hi, vals, narrow);
    if (nv > 0) {
      double tot[kBatchPartials] = {0.0, 0.0, 0.0};
      for (int r = 0; r < nv; ++r) tot[r] = block_sum<double>(vals[r], smem);
      bool last = true;
      if (it.ntiles == 1) {
        // the item's only tile: its totals are this block's sums, added to
        // 0.0 as the combine below adds a single partial (the same bits)
        for (int r = 0; r < nv; ++r) tot[r] = 0.0 + tot[r];
      } else {
        // this tile's partials, then the per-item ticket
        if (threadIdx.x == 0) {
          for (int r = 0; r < nv; ++r) p.partials[tile * kBatchPartials + r] = tot[r];
          __threadfence();
          const unsigned k = atomicAdd(&p.tickets[item], 1u);
          s_last = (k == (unsigned)it.ntiles - 1u);
        }
        __syncthreads();
        last = s_last;
        if (last) {
          __threadfence();
          for (int r = 0; r < nv; ++r) {
            double a = 0.0;
            for (int64_t k = threadIdx.x; k < it.ntiles; k += blockDim.x)
              a += ((volatile double*)p.partials)[(it.tile_begin + k) * kBatchPartials + r];
            tot[r] = block_sum<double>(a, smem);
          }
        }
      }
      if (last && threadIdx.x == 0) {
        if (it.kind == kKindNrm2) {
          p.red_out[it.red_index] = it.dtype == DT_F32 ? __dsqrt_rn(tot[0]) : blue_finish(tot[0], tot[1], tot[2]);
        } else {
          for (int r = 0; r < nv; ++r) p.red_out[it.red_index + r] = tot[r];
        }
        if (it.ntiles != 1) p.tickets[item] = 0u;
      }
    }
    __syncthreads();  // every thread has read s_tile / s_item / s_last of this tile
    if (threadIdx.x == 0) s_tile = (int64_t)next;
    __syncthreads();
  }
}

template <int U>
__global__ void __launch_bounds__(256) batch_kernel(const BatchParams p) {
  run_tiles<U>(p);
  // Every counter is zero again when the launch ends, so the next launch
  // needs no reset: the tickets are cleared by each item's last tile, and
  // the last block to finish (its tile fetches are all done) clears the tile
  // counter and this count.
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(p.exits, 1u) == gridDim.x - 1u) {
      atomicExch(p.counter, 0u);
      atomicExch(p.exits, 0u);
    }
  }
}

}  // namespace salt
