// Generic path: one kernel that runs ANY validated program, for programs
// without a compile-time instantiation.  Same results as the fused kernels
// (same per-node operations in the same order), fewer optimisations.
//
// The host lowers the postfix program to register code over 16 per-thread
// registers: 0..7 hold the vector operands, 8..15 the values at each stack
// depth (register 8 + d for depth d).  Registers live in shared memory, one
// private row per thread, so dynamic register numbers cost no local memory
// and no synchronisation.  Each tile: load burst into the operand registers,
// the register program, store burst -- the same package shape as the fused
// kernels.
#pragma once

#include "common.cuh"

namespace salt {

enum : uint8_t { I_ADD = 0, I_SUB, I_MUL, I_SMUL, I_NEG, I_COPY, I_DOT, I_SUMSQ, I_DIV };
constexpr int kMaxRegCode = 64;
constexpr int kRegs = 16;

struct RegInsn {
  uint8_t op, dst, a, b;  // SMUL: b = scalar index; DOT/SUMSQ: dst = result index
};

template <typename T>
struct InterpParams {
  T* v[kMaxVecs];
  T sc[kMaxScals];
  int64_t n;
  double* red_out;
  void* partials;
  unsigned* ticket;
  uint32_t load_mask, store_mask;
  int32_t len, nred;
  RegInsn code[kMaxRegCode];
  int32_t elementwise;        // 1: operands unaligned or strided, element accesses only
  int64_t stride[kMaxVecs];   // element strides (used when elementwise)
  ScalarCode scode;           // scalar slots computed on the device (len 0: none)
};

template <typename T, class Acc>
__device__ __forceinline__ void acc_add(Acc (&acc)[kMaxReds], int r, T a, T b) {
  switch (r) {
    case 0: acc[0].add_prod(a, b); break;
    case 1: acc[1].add_prod(a, b); break;
    case 2: acc[2].add_prod(a, b); break;
    default: acc[3].add_prod(a, b); break;
  }
}

template <typename T, int VB>
__global__ void __launch_bounds__(256) interp_kernel(const InterpParams<T> p) {
  constexpr int VEC = VB / (int)sizeof(T);
  using V = VecT<T, VB>;
  using Acc = typename AccOf<T>::type;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  T* R = reinterpret_cast<T*>(smem_raw);
  const int64_t bd = blockDim.x;
  auto row = [&](int r) -> T* { return R + ((int64_t)r * bd + threadIdx.x) * VEC; };

  // Scalar slots, shared by the block (dynamic slot numbers read shared
  // memory, not local memory).
  __shared__ T ssc[kMaxScals];
  {
    T sc[kMaxScals];
    load_scalars<T>(p.sc, p.scode, sc);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < kMaxScals; ++k) ssc[k] = sc[k];
    }
    __syncthreads();
  }

  Acc acc[kMaxReds];
  const int64_t n = p.n;
  const int64_t TE = bd * VEC;
  const int64_t ntiles = (n + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * TE + (int64_t)threadIdx.x * VEC;
    const int cnt = base >= n ? 0 : (n - base >= VEC ? VEC : (int)(n - base));
    // load burst
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s) {
      if ((p.load_mask >> s) & 1u) {
        T* r = row(s);
        if (cnt == VEC && !p.elementwise) {
          V t;
          if ((p.store_mask >> s) & 1u) vload<false>(t, p.v[s] + base);
          else vload<true>(t, p.v[s] + base);
          *reinterpret_cast<V*>(r) = t;
        } else {
          const int64_t st = p.elementwise ? p.stride[s] : 1;
          for (int e = 0; e < VEC; ++e) r[e] = e < cnt ? p.v[s][(base + e) * st] : T(0);
        }
      }
    }
    // register program
    for (int pc = 0; pc < p.len; ++pc) {
      const RegInsn in = p.code[pc];
      T* d = row(in.dst);
      const T* a = row(in.a);
      switch (in.op) {
        case I_ADD: {
          const T* b = row(in.b);
#pragma unroll
          for (int e = 0; e < VEC; ++e) d[e] = Arith<T>::add(a[e], b[e]);
        } break;
        case I_SUB: {
          const T* b = row(in.b);
#pragma unroll
          for (int e = 0; e < VEC; ++e) d[e] = Arith<T>::sub(a[e], b[e]);
        } break;
        case I_MUL: {
          const T* b = row(in.b);
#pragma unroll
          for (int e = 0; e < VEC; ++e) d[e] = Arith<T>::mul(a[e], b[e]);
        } break;
        case I_DIV: {
          const T* b = row(in.b);
#pragma unroll
          for (int e = 0; e < VEC; ++e) d[e] = Arith<T>::div(a[e], b[e]);
        } break;
        case I_SMUL: {
          const T s = ssc[in.b];
#pragma unroll
          for (int e = 0; e < VEC; ++e) d[e] = Arith<T>::mul(s, a[e]);
        } break;
        case I_NEG:
#pragma unroll
          for (int e = 0; e < VEC; ++e) d[e] = -a[e];
          break;
        case I_COPY:
#pragma unroll
          for (int e = 0; e < VEC; ++e) d[e] = a[e];
          break;
        case I_DOT: {
          const T* b = row(in.b);
          for (int e = 0; e < cnt; ++e) acc_add<T>(acc, in.dst, a[e], b[e]);
        } break;
        case I_SUMSQ:
          for (int e = 0; e < cnt; ++e) acc_add<T>(acc, in.dst, a[e], a[e]);
          break;
        default:
          break;
      }
    }
    // store burst
#pragma unroll
    for (int s = 0; s < kMaxVecs; ++s) {
      if ((p.store_mask >> s) & 1u) {
        const T* r = row(s);
        if (cnt == VEC && !p.elementwise) {
          vstore(p.v[s] + base, *reinterpret_cast<const V*>(r));
        } else {
          const int64_t st = p.elementwise ? p.stride[s] : 1;
          for (int e = 0; e < cnt; ++e) p.v[s][(base + e) * st] = r[e];
        }
      }
    }
  }

  if (p.nred > 0) {
    __shared__ double smem[kMaxBlock];
    double vals[kMaxReds];
#pragma unroll
    for (int r = 0; r < kMaxReds; ++r) vals[r] = acc[r].value();
    if (grid_combine<double, kMaxReds>(vals, (double*)p.partials, p.ticket, smem) && threadIdx.x == 0) {
      for (int r = 0; r < p.nred; ++r) p.red_out[r] = vals[r];
    }
  }
}

}  // namespace salt
