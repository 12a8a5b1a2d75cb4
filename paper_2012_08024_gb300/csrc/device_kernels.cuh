// Device helpers shared by the solve-phase kernels: read-only loads, aligned
// vector loads of n_p consecutive values, and row i of (A x)_K of a block-sparse
// operator (n_p x n_p row-major blocks, element-major vectors).
#pragma once

#include <cuda_runtime.h>

namespace cdgk {
template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Conversions between binary32 and binary64 built from the IEEE 754 bit
// fields with integer operations.  On this GPU a conversion instruction to or
// from FP64 runs at the rate of the FP64 pipe (about two per clock per SM),
// as slow as an FP64 FMA; the vector kernels of the FP64 CG would spend as
// much time converting as computing.  Both functions give the correctly
// rounded IEEE result; the cases outside the common range (zero is handled
// here; subnormals, infinities and NaN) fall back to the conversion
// instruction.
//
// binary32 -> binary64 is exact: sign, exponent rebiased by 1023 - 127,
// the 23 fraction bits placed at the top of the 52.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  if (e - 1u < 0xFEu)   // 1 <= e <= 254: a normal number
    return __longlong_as_double(
        (long long)(sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
  if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)sgn);   // +-0
  return (double)f;
}

// binary64 -> binary32, round to nearest, ties to even: for a result in the
// normal binary32 range keep the top 23 fraction bits and add one unit when
// the 29 dropped bits exceed half a unit, or equal it with an odd kept part.
// The carry of that addition moves into the exponent field as it should, and
// from the largest finite value into the infinity encoding.
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e >= -126 && e <= 127) {
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const unsigned int kept = (unsigned int)(m >> 29);
    const unsigned int rest = (unsigned int)(m & 0x1FFFFFFFull);
    unsigned int r = ((unsigned int)(e + 127) << 23) | kept;
    if (rest > 0x10000000u || (rest == 0x10000000u && (kept & 1u))) r += 1u;
    return __uint_as_float(sgn | r);
  }
  if ((b << 1) == 0ull) return __uint_as_float(sgn);   // +-0
  return (float)d;
}

template <typename TO, typename TI>
__device__ __forceinline__ TO cvt(TI v) {
  if constexpr (sizeof(TO) == 8 && sizeof(TI) == 4) return f32_to_f64(v);
  else if constexpr (sizeof(TO) == 4 && sizeof(TI) == 8) return f64_to_f32(v);
  else return (TO)v;
}

// NP consecutive values of x as aligned vector loads; CG: through L2 only
// (ld.global.cg: coherent within a kernel whose own phases write x), else
// through the read-only path
template <typename T, int NP, bool CG = false>
struct VecLoad;
template <int NP, bool CG>
struct VecLoad<float, NP, CG> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    if constexpr (NP % 2 == 0) {
#pragma unroll
      for (int j = 0; j < NP; j += 2) {
        const float2 t = CG ? __ldcg(reinterpret_cast<const float2*>(p + j)) : __ldg(reinterpret_cast<const float2*>(p + j));
        v[j] = t.x;
        v[j + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NP; ++j) v[j] = CG ? __ldcg(p + j) : __ldg(p + j);
    }
  }
};
template <int NP, bool CG>
struct VecLoad<double, NP, CG> {
  static __device__ __forceinline__ void load(const double* p, double* v) {
    if constexpr (NP % 2 == 0) {
#pragma unroll
      for (int j = 0; j < NP; j += 2) {
        const double2 t =
            CG ? __ldcg(reinterpret_cast<const double2*>(p + j)) : __ldg(reinterpret_cast<const double2*>(p + j));
        v[j] = t.x;
        v[j + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NP; ++j) v[j] = CG ? __ldcg(p + j) : __ldg(p + j);
    }
  }
};

// Row i of (A x)_K for block row K: sum over the blocks of the row, block by
// block and column by column (the same order for every UNR).
// COHERENT: x is read through L2 only (x may have been written earlier in the same kernel).
template <typename T, int NP, bool VEC, int UNR, bool COHERENT = false>
__device__ __forceinline__ T row_acc(int K, int i, const int* __restrict__ rowptr, const int* __restrict__ col,
                                     const T* __restrict__ A, const T* __restrict__ x) {
  T acc = T(0);
  const int b0 = rowptr[K], b1 = rowptr[K + 1];
  if constexpr (VEC) {
    // even n_p: the row of the block and x_J are 8-byte (FP32) / 16-byte
    // (FP64) aligned runs, read as float2 / double2; UNR blocks per step
    // keep UNR times the loads in flight
    int bb = b0;
    for (; bb + UNR <= b1; bb += UNR) {
      T av[UNR][NP], xv[UNR][NP];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int J = ldg(col + bb + u);
        VecLoad<T, NP>::load(A + (size_t)(bb + u) * NP * NP + i * NP, av[u]);
        VecLoad<T, NP, COHERENT>::load(x + (size_t)J * NP, xv[u]);
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int j = 0; j < NP; ++j) acc = fma(av[u][j], xv[u][j], acc);
    }
    for (; bb < b1; ++bb) {
      T av[NP], xv[NP];
      VecLoad<T, NP>::load(A + (size_t)bb * NP * NP + i * NP, av);
      VecLoad<T, NP, COHERENT>::load(x + (size_t)ldg(col + bb) * NP, xv);
#pragma unroll
      for (int j = 0; j < NP; ++j) acc = fma(av[j], xv[j], acc);
    }
  } else {
    for (int bb = b0; bb < b1; ++bb) {
      const T* a = A + (size_t)bb * NP * NP + i * NP;
      const T* xj = x + (size_t)ldg(col + bb) * NP;
#pragma unroll
      for (int j = 0; j < NP; ++j) acc = fma(ldg(a + j), COHERENT ? __ldcg(xj + j) : ldg(xj + j), acc);
    }
  }
  return acc;
}

}  // namespace cdgk
