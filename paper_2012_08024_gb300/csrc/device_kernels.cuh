// Device helpers shared by the solve-phase kernels: read-only loads, aligned
// vector loads of n_p consecutive values, and row i of (A x)_K of a block-sparse
// operator (n_p x n_p row-major blocks, element-major vectors).
#pragma once

#include <cuda_runtime.h>

namespace cdgk {
template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

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
