// The fused loop: the GPU form of the paper's loop templates (Section 4.2,
// Listing 2; Section 4.3).
//
// Each thread walks tiles in grid-stride order.  Per tile it issues, like one
// of the paper's instruction packages, a burst of U vector loads for every
// loaded operand, then the tree's operations on every element in registers,
// then a burst of U vector stores for every stored operand.  Every block
// takes the same number of whole tiles; what is left (less than one tile per
// block) is spread evenly over all threads as whole vectors in one guarded
// burst, then single elements, with the same per-element operations (the
// paper's single_op tail).
#pragma once

#include "common.cuh"

namespace salt {

template <typename T>
struct MapParams {
  T* v[kMaxVecs];       // operand k (canonical numbering); NULL if unused
  T sc[kMaxScals];      // scalar operands, already in T
  int64_t n;            // element count
  double* red_out;      // device, one double per reduction
  void* partials;       // workspace: gridDim.x * NR values
  unsigned* ticket;     // workspace: zero between launches
  int64_t stride[kMaxVecs];  // element strides (strided_kernel only)
  ScalarCode scode;          // scalar slots computed on the device (len 0: none)
  int32_t head;              // elements before the aligned body (fused and staged kernels):
                             // v[k] points at element `head` of operand k, and elements
                             // 0 .. head-1 sit just before it; 0 for the strided kernel
  unsigned long long* trace; // per-block timeline (kTraceWords per block), or NULL
  Pow2Info p2;               // scalar slots that are powers of two (FP64 programs)
};

// Per-element evaluation of program P: node I at compile-time stack depth.
// FMA = true (FP64 only; exec_chunk_p2 decides): every scaled add (X +- s*v,
// or s*v +- w with w the next vector load; Prog::scaled_add /
// scaled_add_load) is one FMA, which gives the rounded nodes' bits when s*v
// is exact (Pow2Info).  FMA = false: every node its own rounded operation.
template <class P, int I, typename T, class Acc, bool FMA = false>
__device__ __forceinline__ void exec_node(T (&st)[kMaxStack + 1], T (&v)[kMaxVecs], const T (&sc)[kMaxScals],
                                          Acc (&acc)[kMaxReds]) {
  if constexpr (I < P::len) {
    constexpr int op = P::op(I), a = P::arg(I), d = P::depth_before(I);
    constexpr bool fuse = FMA && sizeof(T) == 8 && P::scaled_add(I);
    constexpr bool fuse_load = FMA && sizeof(T) == 8 && P::scaled_add_load(I);
    if constexpr (op == OP_VEC) {
      st[d] = v[a];
    } else if constexpr (op == OP_SCAL) {
      st[d] = sc[a];
    } else if constexpr (op == OP_ADD) {
      st[d - 2] = Arith<T>::add(st[d - 2], st[d - 1]);
    } else if constexpr (op == OP_SUB) {
      st[d - 2] = Arith<T>::sub(st[d - 2], st[d - 1]);
    } else if constexpr (fuse) {  // SMUL, then ADD / SUB
      const T s = st[d - 2];
      st[d - 3] = __fma_rn(P::op(I + 1) == OP_SUB ? -s : s, st[d - 1], st[d - 3]);
    } else if constexpr (fuse_load) {  // SMUL, VEC, then ADD / SUB
      const T w = v[P::arg(I + 1)];
      st[d - 2] = __fma_rn(st[d - 2], st[d - 1], P::op(I + 2) == OP_SUB ? -w : w);
    } else if constexpr (op == OP_MUL || op == OP_SMUL) {
      st[d - 2] = Arith<T>::mul(st[d - 2], st[d - 1]);
    } else if constexpr (op == OP_DIV) {
      st[d - 2] = Arith<T>::div(st[d - 2], st[d - 1]);
    } else if constexpr (op == OP_NEG) {
      st[d - 1] = -st[d - 1];
    } else if constexpr (op == OP_STORE) {
      v[a] = st[d - 1];
    } else if constexpr (op == OP_DOT) {
      acc[P::red_index(I)].add_prod(st[d - 2], st[d - 1]);
    } else if constexpr (op == OP_SUMSQ) {
      acc[P::red_index(I)].add_prod(st[d - 1], st[d - 1]);
    }
    exec_node<P, I + (fuse ? 2 : fuse_load ? 3 : 1), T, Acc, FMA>(st, v, sc, acc);
  }
}

template <class P, typename T, class Acc, bool FMA = false>
__device__ __forceinline__ void exec_elem(T (&v)[kMaxVecs], const T (&sc)[kMaxScals], Acc (&acc)[kMaxReds]) {
  T st[kMaxStack + 1];
  exec_node<P, 0, T, Acc, FMA>(st, v, sc, acc);
}

// One thread's work on NE consecutive elements held in per-operand arrays.
template <class P, typename T, class Acc, int NE, bool FMA = false>
__device__ __forceinline__ void exec_chunk(T (&x)[kMaxVecs][NE], const T (&sc)[kMaxScals], Acc (&acc)[kMaxReds]) {
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    T v[kMaxVecs];
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s) v[s] = x[s][e];
    exec_elem<P, T, Acc, FMA>(v, sc, acc);
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s)
      if ((P::store_mask() >> s) & 1u) x[s][e] = v[s];
  }
}

// At every scaled add of P from node I on, the slot is a power of two and s*v
// is exact for every element of the chunk (v as loaded: Prog::scaled_vec).
template <class P, int I, int NE>
__device__ __forceinline__ bool pow2_chunk_ok(const double (&x)[kMaxVecs][NE], const Pow2Info& p2) {
  if constexpr (I >= P::len) {
    return true;
  } else {
    bool ok = true;
    if constexpr (P::scaled_add(I) || P::scaled_add_load(I)) {
      constexpr int k = P::scaled_add_slot(I), a = P::scaled_add_vec(I);
      ok = ((p2.mask >> k) & 1u) != 0u;
#pragma unroll
      for (int e = 0; e < NE; ++e) ok = ok & exact_pow2_scale(x[a][e], p2.exp[k]);
    }
    return ok & pow2_chunk_ok<P, I + 1, NE>(x, p2);
  }
}

// exec_chunk with the scaled adds as FMAs when the whole chunk allows it
// (FP64).  The test runs on the loaded operands before any arithmetic and
// picks one of two complete chunk bodies, so each element runs one form only
// (a test per element let the compiler compute both forms and select, one
// FP64 instruction more instead of one less).  Programs with reductions keep
// one body: the second doubled the register count of the CG-update shape
// (80 to 157 at unroll 4).
template <class P, typename T, class Acc, int NE>
__device__ __forceinline__ void exec_chunk_p2(T (&x)[kMaxVecs][NE], const T (&sc)[kMaxScals], Acc (&acc)[kMaxReds],
                                              const Pow2Info& p2) {
  if constexpr (sizeof(T) == 8 && P::nred() == 0 && P::any_scaled_add()) {
    if (p2.mask != 0u && pow2_chunk_ok<P, 0, NE>(x, p2)) {
      exec_chunk<P, T, Acc, NE, true>(x, sc, acc);
      return;
    }
  }
  exec_chunk<P, T, Acc, NE>(x, sc, acc);
}

// The head of operands that share one misalignment: the host moved every
// operand pointer forward to the next 16-byte boundary, and threads
// 0 .. head-1 of block 0 evaluate the elements it stepped over, one each,
// with the same per-element operations (Section 4.3's single_op, before the
// vectorised loop instead of after it).
template <class P, typename T, class Acc>
__device__ __forceinline__ void run_head(const MapParams<T>& p, const T (&sc)[kMaxScals], Acc (&acc)[kMaxReds]) {
  constexpr unsigned LM = P::load_mask(), SMASK = P::store_mask();
  if (blockIdx.x == 0 && (int)threadIdx.x < p.head) {
    const int64_t i = (int64_t)threadIdx.x - p.head;  // negative: before the body
    T x[kMaxVecs][1];
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s) x[s][0] = ((LM >> s) & 1u) ? p.v[s][i] : T(0);
    exec_chunk<P, T, Acc, 1>(x, sc, acc);
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s)
      if ((SMASK >> s) & 1u) p.v[s][i] = x[s][0];
  }
}

// DS: some scalar slots are computed on the device from p.scode at kernel
// start.  A separate instantiation, because scalars that may come from
// shared memory occupy registers for the whole loop, while by-value
// scalars are re-read from the constant bank at each use.
template <class P, typename T, int U, int VB, bool DS = false>
__global__ void __launch_bounds__(256) fused_kernel(const MapParams<T> p) {
  constexpr int VEC = VB / (int)sizeof(T);
  constexpr unsigned LM = P::load_mask(), SMASK = P::store_mask();
  constexpr int NR = P::nred();
  using Acc = typename AccOf<T>::type;
  using V = VecT<T, VB>;

  trace_mark(p.trace, TR_START);
  T sc[kMaxScals];
  if constexpr (DS) {
    load_scalars<T>(p.sc, p.scode, sc);
  } else {
#pragma unroll
    for (int k = 0; k < kMaxScals; ++k) sc[k] = p.sc[k];
  }
  Acc acc[kMaxReds];
  run_head<P, T, Acc>(p, sc, acc);

  const int64_t n = p.n;
  const int64_t bd = blockDim.x;
  const int64_t TE = (int64_t)U * bd * VEC;  // elements per tile
  // Whole rounds of tiles in grid-stride order: every block takes exactly
  // `rounds` tiles, so no block runs a tile longer than the others.
  const int64_t rounds = (n / TE) / gridDim.x;

  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t tile = blockIdx.x + r * (int64_t)gridDim.x;
    const int64_t base = tile * TE + (int64_t)threadIdx.x * VEC;
    T x[kMaxVecs][U * VEC];
    // load burst
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int s = 0; s < kMaxVecs; ++s) {
        if ((LM >> s) & 1u) {
          V t;
          if ((SMASK >> s) & 1u) vload<false>(t, p.v[s] + base + u * bd * VEC);
          else vload<true>(t, p.v[s] + base + u * bd * VEC);
#pragma unroll
          for (int e = 0; e < VEC; ++e) x[s][u * VEC + e] = t.e[e];
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) x[s][u * VEC + e] = T(0);
        }
      }
    }
    // operation burst
    exec_chunk_p2<P, T, Acc, U * VEC>(x, sc, acc, p.p2);
    // store burst
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int s = 0; s < kMaxVecs; ++s) {
        if ((SMASK >> s) & 1u) {
          V t;
#pragma unroll
          for (int e = 0; e < VEC; ++e) t.e[e] = x[s][u * VEC + e];
          vstore(p.v[s] + base + u * bd * VEC, t);
        }
      }
    }
  }

  trace_mark(p.trace, TR_TILES);
  // The remainder after the whole rounds -- fewer than gridDim.x tiles --
  // spread evenly over every thread of the grid as whole vectors, at most U
  // per thread, in one guarded burst (all loads first, then the operations
  // and stores of the vectors that exist), then single elements.
  const int64_t rbase = rounds * (int64_t)gridDim.x * TE;
  const int64_t nvr = (n - rbase) / VEC;  // < gridDim.x * U * blockDim.x
  const int64_t gid = (int64_t)blockIdx.x * bd + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * bd;
  if (gid < nvr) {
    T x[kMaxVecs][U * VEC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t j = gid + u * gstride;
#pragma unroll
      for (int s = 0; s < kMaxVecs; ++s) {
        if (((LM >> s) & 1u) && j < nvr) {
          V t;
          if ((SMASK >> s) & 1u) vload<false>(t, p.v[s] + rbase + j * VEC);
          else vload<true>(t, p.v[s] + rbase + j * VEC);
#pragma unroll
          for (int e = 0; e < VEC; ++e) x[s][u * VEC + e] = t.e[e];
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) x[s][u * VEC + e] = T(0);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t j = gid + u * gstride;
      if (j < nvr) {
        T xu[kMaxVecs][VEC];
#pragma unroll
        for (int s = 0; s < kMaxVecs; ++s) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) xu[s][e] = x[s][u * VEC + e];
        }
        exec_chunk<P, T, Acc, VEC>(xu, sc, acc);
#pragma unroll
        for (int s = 0; s < kMaxVecs; ++s) {
          if ((SMASK >> s) & 1u) {
            V t;
#pragma unroll
            for (int e = 0; e < VEC; ++e) t.e[e] = xu[s][e];
            vstore(p.v[s] + rbase + j * VEC, t);
          }
        }
      }
    }
  }
  for (int64_t i = rbase + nvr * VEC + gid; i < n; i += gstride) {
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

// Element-wise access variant for operands that are not 16-byte aligned or
// not contiguous: element i of operand k is v[k][i * stride[k]].  Each thread
// takes U elements per pass, U * blockDim apart within a block's stretch, so
// unit-stride operands still coalesce; the load burst / operation / store
// burst shape is kept, and out-of-range elements are neither loaded, stored
// nor reduced.
template <class P, typename T, int U>
__global__ void __launch_bounds__(256) strided_kernel(const MapParams<T> p) {
  constexpr unsigned LM = P::load_mask(), SMASK = P::store_mask();
  constexpr int NR = P::nred();
  using Acc = typename AccOf<T>::type;
  T sc[kMaxScals];
  load_scalars<T>(p.sc, p.scode, sc);
  Acc acc[kMaxReds];
  const int64_t n = p.n;
  const int64_t bd = blockDim.x;
  const int64_t span = (int64_t)U * bd;
  for (int64_t base = (int64_t)blockIdx.x * span; base < n; base += (int64_t)gridDim.x * span) {
    T x[kMaxVecs][U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * bd + threadIdx.x;
#pragma unroll
      for (int s = 0; s < kMaxVecs; ++s)
        x[s][u] = (((LM >> s) & 1u) && i < n) ? p.v[s][i * p.stride[s]] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * bd + threadIdx.x;
      if (i < n) {
        T v[kMaxVecs];
#pragma unroll
        for (int s = 0; s < kMaxVecs; ++s) v[s] = x[s][u];
        exec_elem<P, T, Acc>(v, sc, acc);
#pragma unroll
        for (int s = 0; s < kMaxVecs; ++s)
          if ((SMASK >> s) & 1u) x[s][u] = v[s];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * bd + threadIdx.x;
#pragma unroll
      for (int s = 0; s < kMaxVecs; ++s)
        if (((SMASK >> s) & 1u) && i < n) p.v[s][i * p.stride[s]] = x[s][u];
    }
  }
  if constexpr (NR > 0) {
    __shared__ double smem[kMaxBlock];
    double vals[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) vals[r] = acc[r].value();
    if (grid_combine<double, NR>(vals, (double*)p.partials, p.ticket, smem) && threadIdx.x == 0) {
#pragma unroll
      for (int r = 0; r < NR; ++r) p.red_out[r] = vals[r];
    }
  }
}

}  // namespace salt
