// Reductions with their own accumulators: the Euclidean norm with Blue's
// three-range scaling, and the plain-FP32 dot product comparison mode.
#pragma once

#include "common.cuh"

namespace salt {

// Blue's thresholds and scale factors (Blue 1978; radix 2).  With t the
// precision, emin / emax the exponent range (x = m * 2^e, 0.5 <= m < 1):
//   tsml = 2^ceil((emin - 1) / 2)       squares of values >= tsml are normal
//   tbig = 2^floor((emax - t + 1) / 2)  squares of values <= tbig, summed up to
//                                       2^t times, stay finite
//   ssml = 2^-floor((emin - t) / 2)     small values are scaled up by ssml
//   sbig = 2^-ceil((emax + t - 1) / 2)  big values are scaled down by sbig
// F32: t = 24, emin = -125, emax = 128.  F64: t = 53, emin = -1021, emax = 1024.
template <typename T> struct Blue;
template <> struct Blue<float> {
  static constexpr float tsml = 0x1p-63f, tbig = 0x1p52f, ssml = 0x1p75f, sbig = 0x1p-76f;
  // powers of two that undo the scaling of the squares, used in FP64
  static constexpr double unsml = 0x1p-150, unbig = 0x1p152;
};
template <> struct Blue<double> {
  static constexpr double tsml = 0x1p-511, tbig = 0x1p486, ssml = 0x1p537, sbig = 0x1p-538;
};

// Per-thread state of the F32 norm: compensated medium sum, plain small and
// big sums of scaled squares.
struct Nrm2F32 {
  AccF32 med;
  float sml = 0.f, big = 0.f;
  // x^2 added to the medium sum, error-free: the square by TwoProduct (FMA)
  // and, because both addends are non-negative, the sum by Fast2Sum with the
  // larger addend first (exact whenever |a| >= |b|; Dekker 1971) -- two
  // min/max instead of TwoSum's three extra additions.  Same error bound as
  // the general compensated product (Ogita, Rump and Oishi's Dot2).
  __device__ __forceinline__ void add_sq(float x) {
    const float p = __fmul_rn(x, x);
    const float ep = __fmaf_rn(x, x, -p);  // x*x - p exactly
    const float t = __fadd_rn(med.s, p);
    const float hi = fmaxf(med.s, p), lo = fminf(med.s, p);
    const float es = __fadd_rn(__fsub_rn(hi, t), lo);  // med.s + p - t exactly
    med.s = t;
    med.c = __fadd_rn(med.c, __fadd_rn(es, ep));
  }
  __device__ __forceinline__ void add(float x) {
    const float ax = fabsf(x);
    if (ax > Blue<float>::tbig) {
      const float t = __fmul_rn(ax, Blue<float>::sbig);
      big = __fmaf_rn(t, t, big);
    } else if (ax < Blue<float>::tsml) {
      const float t = __fmul_rn(ax, Blue<float>::ssml);
      sml = __fmaf_rn(t, t, sml);
    } else {
      add_sq(ax);
    }
  }
  // A whole vector: one range test for all its elements (the largest and
  // smallest magnitude), then the medium path without per-element tests; a
  // vector with any element outside the medium range takes the per-element
  // path.  A NaN (which fmaxf / fminf pass over) reaches add_sq on either
  // path and makes the sum NaN, as the per-element path does.
  template <int N>
  __device__ __forceinline__ void add_vec(const float (&v)[N]) {
    float mx = fabsf(v[0]), mn = mx;
#pragma unroll
    for (int e = 1; e < N; ++e) {
      mx = fmaxf(mx, fabsf(v[e]));
      mn = fminf(mn, fabsf(v[e]));
    }
    if (mx <= Blue<float>::tbig && mn >= Blue<float>::tsml) {
#pragma unroll
      for (int e = 0; e < N; ++e) add_sq(v[e]);
    } else {
#pragma unroll
      for (int e = 0; e < N; ++e) add(v[e]);
    }
  }
  // The whole sum of squares in FP64, where it cannot overflow for F32 data.
  __device__ __forceinline__ double value() const {
    return med.value() + (double)big * Blue<float>::unbig + (double)sml * Blue<float>::unsml;
  }
};

struct Nrm2F32Plain {
  float s = 0.f;
  __device__ __forceinline__ void add(float x) { s = __fmaf_rn(x, x, s); }
};

// F64: the range of |x| is read from the biased exponent with integer
// instructions -- on GB300 the FP64 pipe (about 2 instructions per clock per
// SM) is the scarce resource, and a medium element then costs exactly one
// FP64 instruction (the FMA).  Medium: 2^-511 <= |x| < 2^486 (biased exponent
// 512..1508); big: |x| >= 2^486, Inf and NaN (exponent >= 1509); small:
// |x| < 2^-511, zeros and subnormals (exponent < 512).
struct Nrm2F64 {
  double sml = 0.0, med = 0.0, big = 0.0;
  __device__ __forceinline__ void add(double x) {
    const unsigned bexp = ((unsigned)__double2hiint(x) >> 20) & 0x7FFu;
    if (bexp - 512u < 997u) {
      med = __fma_rn(x, x, med);
    } else if (bexp >= 1509u) {
      const double t = __dmul_rn(fabs(x), Blue<double>::sbig);
      big = __fma_rn(t, t, big);
    } else {
      const double t = __dmul_rn(fabs(x), Blue<double>::ssml);
      sml = __fma_rn(t, t, sml);
    }
  }
};

// Final combination of Blue's three FP64 sums into the norm.
__device__ __forceinline__ double blue_finish(double sml, double med, double big) {
  if (isnan(sml) || isnan(med) || isnan(big)) return sml + med + big;
  if (big > 0.0) {
    // medium contributions are folded into the big scale; small ones are
    // below its rounding
    const double tot = __dadd_rn(big, __dmul_rn(__dmul_rn(med, Blue<double>::sbig), Blue<double>::sbig));
    return __dsqrt_rn(tot) / Blue<double>::sbig;
  }
  if (sml > 0.0) {
    if (med > 0.0) {
      const double ymed = __dsqrt_rn(med);
      const double ysml = __dsqrt_rn(sml) / Blue<double>::ssml;
      const double ymax = fmax(ymed, ysml), ymin = fmin(ymed, ysml);
      const double r = ymin / ymax;
      return ymax * __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(r, r)));
    }
    return __dsqrt_rn(sml) / Blue<double>::ssml;
  }
  return __dsqrt_rn(med);
}

struct NrmParams {
  const void* x;
  int64_t n;
  double* out;
  void* partials;
  unsigned* ticket;
  unsigned long long* trace = nullptr;  // per-block timeline (kTraceWords per block), or NULL
};

// Tile loop shared by the norm and plain-dot kernels: calls fv(vector of x,
// vector of y) on whole vectors and f1 on single elements.  As in the fused
// loop, every block takes the same number of whole tiles, and the remainder
// (less than a tile per block) goes to every thread of the grid as at most U
// whole vectors in one guarded burst.
template <typename T, int U, int VB, int NIN, class FV, class F1>
__device__ __forceinline__ void reduce_loop(const T* x, const T* y, int64_t n, FV fv, F1 f1,
                                            unsigned long long* trace) {
  constexpr int VEC = VB / (int)sizeof(T);
  using V = VecT<T, VB>;
  const int64_t bd = blockDim.x;
  const int64_t TE = (int64_t)U * bd * VEC;
  const int64_t rounds = (n / TE) / gridDim.x;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t base = (blockIdx.x + r * (int64_t)gridDim.x) * TE + (int64_t)threadIdx.x * VEC;
    V a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      vload<true>(a[u], x + base + u * bd * VEC);
      if (NIN == 2) vload<true>(b[u], y + base + u * bd * VEC);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) fv(a[u], b[u]);
  }
  trace_mark(trace, TR_TILES);
  const int64_t rbase = rounds * (int64_t)gridDim.x * TE;
  const int64_t nvr = (n - rbase) / VEC;  // < gridDim.x * U * blockDim.x
  const int64_t gid = (int64_t)blockIdx.x * bd + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * bd;
  if (gid < nvr) {
    V a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t j = gid + u * gstride;
      if (j < nvr) {
        vload<true>(a[u], x + rbase + j * VEC);
        if (NIN == 2) vload<true>(b[u], y + rbase + j * VEC);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (gid + u * gstride < nvr) fv(a[u], b[u]);
  }
  for (int64_t i = rbase + nvr * VEC + gid; i < n; i += gstride) f1(x[i], NIN == 2 ? y[i] : T(0));
}

template <typename T, int U, int VB, bool PLAIN>
__global__ void __launch_bounds__(256) nrm2_kernel(const NrmParams p) {
  using V = VecT<T, VB>;
  constexpr int VEC = VB / (int)sizeof(T);
  const T* x = (const T*)p.x;
  trace_mark(p.trace, TR_START);
  bool last = false;
  if constexpr (sizeof(T) == 4 && PLAIN) {
    Nrm2F32Plain acc;
    reduce_loop<T, U, VB, 1>(x, nullptr, p.n,
        [&](const V& a, const V&) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc.add(a.e[e]);
        },
        [&](T a, T) { acc.add(a); }, p.trace);
    __shared__ float smem[kMaxBlock];
    float vals[1] = {acc.s};
    trace_mark(p.trace, TR_PRE_COMBINE);
    last = grid_combine<float, 1>(vals, (float*)p.partials, p.ticket, smem);
    if (last && threadIdx.x == 0) *p.out = (double)sqrtf(vals[0]);
  } else if constexpr (sizeof(T) == 4) {
    Nrm2F32 acc;
    reduce_loop<T, U, VB, 1>(x, nullptr, p.n,
        [&](const V& a, const V&) { acc.add_vec<VEC>(a.e); },
        [&](T a, T) { acc.add(a); }, p.trace);
    __shared__ double smem[kMaxBlock];
    double vals[1] = {acc.value()};
    trace_mark(p.trace, TR_PRE_COMBINE);
    last = grid_combine<double, 1>(vals, (double*)p.partials, p.ticket, smem);
    if (last && threadIdx.x == 0) *p.out = __dsqrt_rn(vals[0]);
  } else {
    Nrm2F64 acc;
    reduce_loop<T, U, VB, 1>(x, nullptr, p.n,
        [&](const V& a, const V&) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc.add(a.e[e]);
        },
        [&](T a, T) { acc.add(a); }, p.trace);
    __shared__ double smem[kMaxBlock];
    double vals[3] = {acc.sml, acc.med, acc.big};
    trace_mark(p.trace, TR_PRE_COMBINE);
    last = grid_combine<double, 3>(vals, (double*)p.partials, p.ticket, smem);
    if (last && threadIdx.x == 0) *p.out = blue_finish(vals[0], vals[1], vals[2]);
  }
  trace_end(p.trace, last);
}

// Norm of an operand that is not 16-byte aligned: element loads (consecutive
// threads, consecutive elements), same accumulators and combination as
// nrm2_kernel.
template <typename T>
__global__ void __launch_bounds__(256) nrm2_elem_kernel(const NrmParams p) {
  const T* x = (const T*)p.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  __shared__ double smem[kMaxBlock];
  if constexpr (sizeof(T) == 4) {
    Nrm2F32 acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) acc.add(x[i]);
    double vals[1] = {acc.value()};
    if (grid_combine<double, 1>(vals, (double*)p.partials, p.ticket, smem) && threadIdx.x == 0)
      *p.out = __dsqrt_rn(vals[0]);
  } else {
    Nrm2F64 acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) acc.add(x[i]);
    double vals[3] = {acc.sml, acc.med, acc.big};
    if (grid_combine<double, 3>(vals, (double*)p.partials, p.ticket, smem) && threadIdx.x == 0)
      *p.out = blue_finish(vals[0], vals[1], vals[2]);
  }
}

struct DotParams {
  const void* x;
  const void* y;
  int64_t n;
  double* out;
  void* partials;
  unsigned* ticket;
  unsigned long long* trace = nullptr;  // per-block timeline, or NULL
};

// Plain FP32 dot: FP32 accumulation and FP32 combination.
template <int U, int VB>
__global__ void __launch_bounds__(256) dot_plain_kernel(const DotParams p) {
  using V = VecT<float, VB>;
  constexpr int VEC = VB / 4;
  AccF32Plain acc;
  reduce_loop<float, U, VB, 2>((const float*)p.x, (const float*)p.y, p.n,
      [&](const V& a, const V& b) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc.add_prod(a.e[e], b.e[e]);
      },
      [&](float a, float b) { acc.add_prod(a, b); }, p.trace);
  __shared__ float smem[kMaxBlock];
  float vals[1] = {acc.s};
  if (grid_combine<float, 1>(vals, (float*)p.partials, p.ticket, smem) && threadIdx.x == 0)
    *p.out = (double)vals[0];
}

// Counter-based uniform fill (SplitMix64 finaliser, Steele-Lea-Flood 2014).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t key, uint64_t i) {
  uint64_t z = key + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct FillParams {
  void* x;
  int64_t n;
  uint64_t key;
  int64_t offset;
};

template <typename T>
__global__ void __launch_bounds__(256) fill_kernel(T* x, int64_t n, uint64_t key, int64_t offset) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t h = splitmix64_at(key, (uint64_t)(offset + i));
    if constexpr (sizeof(T) == 8) {
      const double u = (double)(h >> 11) * 0x1p-53;
      x[i] = __dsub_rn(__dmul_rn(2.0, u), 1.0);
    } else {
      const float u = (float)(uint32_t)(h >> 40) * 0x1p-24f;
      x[i] = __fsub_rn(__fmul_rn(2.0f, u), 1.0f);
    }
  }
}

}  // namespace salt
