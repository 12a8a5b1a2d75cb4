// The whole V-cycle (Section 4.3, Algorithm 3; reading R14) as ONE persistent
// kernel: a cooperative launch whose CTAs (all resident on the GPU) walk the
// phases of the cycle -- first smoothing step, smoothing sweeps, residual,
// restriction, the coarsest solve and its refinement, prolongation -- and meet
// at a grid barrier between phases.  It serves batched handles (many meshes of
// uneven size as one block-diagonal hierarchy), whose small levels would
// otherwise cost one launch each.  In every phase the work units (groups of
// 32 / n_p block rows, one warp each; one warp per coarsest row) are dealt to
// the warps of the grid in turn, so a phase needs no particular grid size.
//
// Each barrier counts arrivals on one global counter and releases the grid by
// bumping a generation word.  A CTA waits for the bump with an iteration
// limit; when the limit is reached it sets the error flag and returns, and so,
// one barrier later at most, does every other CTA: the kernel always ends.
// The host reads the flag (CDG_ETIMEOUT).  The counter and generation words
// are cleared before every launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_kernels.cuh"
#include "device_state.h"

namespace {

using cdgk::cvt;
using cdgk::ldg;
using cdgk::row_acc;

constexpr int kPThreads = 256;
constexpr int kBarrierLimit = 1 << 24;

struct PLevel {
  int n;
  const int *rowptr, *col, *hrowptr, *hcol, *parent, *childptr;
  const void *A, *Ahat, *Dinv, *L;
  void *x, *t, *r, *b, *bh;
};

struct PParams {
  int nlev, nu_pre, nu_post, nc, refine;
  double omega;
  PLevel lev[kMaxLev];
  const int *crow_seg, *crow_off;
  const long long* cinv_off;
  const double* coarse_inv;
  const void* b0;
  void* z0;
  unsigned* count;   // [0] arrivals, [1] generation
  int* err;
  int wait_limit;
};

// grid barrier with a bounded wait; false (and the error flag set) on expiry
__device__ bool grid_barrier(const PParams& P) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = P.count + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(P.count, 1u) == gridDim.x - 1) {
      atomicExch(P.count, 0u);
      __threadfence();
      atomicAdd(P.count + 1, 1u);
    } else {
      for (int it = 0; *gen == g; ++it) {
        if (it >= P.wait_limit) {
          ok = 0;
          atomicExch(P.err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// one warp per group of RPW block rows of level n: the group index g covers rows g * RPW + sub
template <typename F>
__device__ __forceinline__ void for_groups(int n, int np, F&& f) {
  const int rpw = 32 / np;
  const int warps = (int)(gridDim.x * (blockDim.x >> 5));
  const int lane = threadIdx.x & 31;
  const int sub = lane / np, i = lane - sub * np;
  for (int g = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); g * rpw < n; g += warps) {
    const int K = g * rpw + sub;
    if (sub < rpw && K < n) f(K, i);
  }
}

// Vectors written by earlier phases of this kernel are read through L2 only
// (__ldcg): the L1 and read-only caches of an SM are not kept coherent with
// other SMs' writes inside one kernel.  Operators are read-only (__ldg).

// MODE 1: y = b - A x; MODE 3: y = x + omega (bh - x - Ahat x)
template <typename T, int NP, bool VEC, int MODE>
__device__ void ph_bsr(int n, const int* rp, const int* cl, const T* A, const T* x, const T* b, T* y, T omega) {
  for_groups(n, NP, [&](int K, int i) {
    const T acc = row_acc<T, NP, VEC, 2, true>(K, i, rp, cl, A, x);
    const size_t row = (size_t)K * NP + i;
    if (MODE == 1) {
      y[row] = __ldcg(b + row) - acc;
    } else {
      const T xv = __ldcg(x + row);
      y[row] = xv + omega * (__ldcg(b + row) - xv - acc);
    }
  });
}

// bh = D^{-1} b and (write_x) x = omega bh
template <typename T, int NP>
__device__ void ph_first(int n, const T* Dinv, const T* b, T* bh, T* x, T omega, bool write_x) {
  for_groups(n, NP, [&](int K, int i) {
    const T* D = Dinv + (size_t)K * NP * NP + i * NP;
    const T* bk = b + (size_t)K * NP;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) s = fma(ldg(D + j), __ldcg(bk + j), s);
    bh[(size_t)K * NP + i] = s;
    if (write_x) x[(size_t)K * NP + i] = omega * s;
  });
}

// bc[A] = sum over the children K of A of L_K^T r_K
template <typename T, int NP>
__device__ void ph_restrict(int nc, const int* childptr, const T* L, const T* r, T* bc) {
  for_groups(nc, NP, [&](int Ag, int i) {
    T s = T(0);
    for (int K = childptr[Ag]; K < childptr[Ag + 1]; ++K) {
      const T* LK = L + (size_t)K * NP * NP + i;
      const T* rk = r + (size_t)K * NP;
#pragma unroll
      for (int j = 0; j < NP; ++j) s = fma(ldg(LK + j * NP), __ldcg(rk + j), s);
    }
    bc[(size_t)Ag * NP + i] = s;
  });
}

// x[K] (+)= L_K xc[parent K]
template <typename T, int NP>
__device__ void ph_prolong(int n, const int* parent, const T* L, const T* xc, T* x, bool add) {
  for_groups(n, NP, [&](int K, int i) {
    const T* LK = L + (size_t)K * NP * NP + i * NP;
    const T* xa = xc + (size_t)parent[K] * NP;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) s = fma(ldg(LK + j), __ldcg(xa + j), s);
    const size_t row = (size_t)K * NP + i;
    x[row] = add ? __ldcg(x + row) + s : s;
  });
}

// coarsest rows, one warp each: x (+)= Ainv_m b on the row's segment m, FP64 accumulation
template <typename T>
__device__ void ph_coarse(const PParams& P, const T* b, T* x, bool add) {
  const int warps = (int)(gridDim.x * (blockDim.x >> 5));
  const int lane = threadIdx.x & 31;
  for (int row = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); row < P.nc; row += warps) {
    const int m = P.crow_seg[row];
    const int r0 = P.crow_off[m], nm = P.crow_off[m + 1] - r0;
    const double* a = P.coarse_inv + P.cinv_off[m] + (size_t)(row - r0) * nm;
    const T* bm = b + r0;
    double s = 0.0;
    for (int j = lane; j < nm; j += 32) s = fma(ldg(a + j), cvt<double>(__ldcg(bm + j)), s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = add ? cvt<T>(cvt<double>(__ldcg(x + row)) + s) : cvt<T>(s);
  }
}

template <typename T, int NP>
__global__ void __launch_bounds__(kPThreads) vcycle_persistent_kernel(PParams P) {
  constexpr bool VEC = NP % 2 == 0;
  const T w = (T)P.omega;
  const int nlev = P.nlev;
  // where each level's iterate is at the end of its downward (x_down) and upward (x_fin) visit
  T* x_down[kMaxLev];
  T* x_fin[kMaxLev];
#define CDG_SYNC \
  if (!grid_barrier(P)) return
  // downward sweep: the buffers x and t of a level alternate per sweep
  for (int l = 0; l + 1 < nlev; ++l) {
    const PLevel& L = P.lev[l];
    const T* b = l == 0 ? (const T*)P.b0 : (const T*)L.b;
    T* xa = (T*)L.x;
    T* xb = (T*)L.t;
    if (P.nu_pre >= 1) {
      ph_first<T, NP>(L.n, (const T*)L.Dinv, b, (T*)L.bh, xa, w, true);
      CDG_SYNC;
      for (int k = 1; k < P.nu_pre; ++k) {
        ph_bsr<T, NP, VEC, 3>(L.n, L.hrowptr, L.hcol, (const T*)L.Ahat, xa, (const T*)L.bh, xb, w);
        CDG_SYNC;
        T* tmp = xa;
        xa = xb;
        xb = tmp;
      }
      ph_bsr<T, NP, VEC, 1>(L.n, L.rowptr, L.col, (const T*)L.A, xa, b, (T*)L.r, w);
      CDG_SYNC;
      ph_restrict<T, NP>(P.lev[l + 1].n, P.lev[l + 1].childptr, (const T*)L.L, (const T*)L.r, (T*)P.lev[l + 1].b);
    } else {
      ph_first<T, NP>(L.n, (const T*)L.Dinv, b, (T*)L.bh, xa, w, false);
      ph_restrict<T, NP>(P.lev[l + 1].n, P.lev[l + 1].childptr, (const T*)L.L, b, (T*)P.lev[l + 1].b);
    }
    x_down[l] = xa;
    CDG_SYNC;
  }
  // coarsest: dense inverse, then (FP64 operator present) one refinement step
  {
    const PLevel& C = P.lev[nlev - 1];
    T* xc = nlev == 1 ? (T*)P.z0 : (T*)C.x;
    const T* bc = nlev == 1 ? (const T*)P.b0 : (const T*)C.b;
    ph_coarse<T>(P, bc, xc, false);
    if (P.refine) {
      CDG_SYNC;
      ph_bsr<T, NP, VEC, 1>(C.n, C.rowptr, C.col, (const T*)C.A, xc, bc, (T*)C.r, w);
      CDG_SYNC;
      ph_coarse<T>(P, (const T*)C.r, xc, true);
    }
    x_fin[nlev - 1] = xc;
    if (nlev == 1) return;
    CDG_SYNC;
  }
  // upward sweep
  for (int l = nlev - 2; l >= 0; --l) {
    const PLevel& L = P.lev[l];
    T* xa = x_down[l];
    T* xb = xa == (T*)L.x ? (T*)L.t : (T*)L.x;
    ph_prolong<T, NP>(L.n, L.parent, (const T*)L.L, x_fin[l + 1], xa, P.nu_pre >= 1);
    for (int k = 0; k < P.nu_post; ++k) {
      CDG_SYNC;
      T* out = (l == 0 && k + 1 == P.nu_post) ? (T*)P.z0 : xb;
      ph_bsr<T, NP, VEC, 3>(L.n, L.hrowptr, L.hcol, (const T*)L.Ahat, xa, (const T*)L.bh, out, w);
      xb = xa;
      xa = out;
    }
    if (l == 0 && P.nu_post == 0) {
      CDG_SYNC;
      for_groups(L.n, NP, [&](int K, int i) { ((T*)P.z0)[(size_t)K * NP + i] = __ldcg(xa + (size_t)K * NP + i); });
    }
    x_fin[l] = xa;
    if (l > 0) CDG_SYNC;
  }
#undef CDG_SYNC
}

template <typename T, int NP>
int launch_one(const PParams& P, cudaStream_t s, int* grid_out) {
  auto kern = vcycle_persistent_kernel<T, NP>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, 0) != cudaSuccess || per_sm < 1)
    return -1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = per_sm * sms;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kern, P) != cudaSuccess) return -1;
  *grid_out = grid;
  return 0;
}

}  // namespace

// One V-cycle z0 = V(b0) of handle state D as one cooperative persistent launch.
// Needs every level at one n_p and agglomeration transfers (no degree steps).
// count: two device words, cleared here; err: the device error flag.
bool vcycle_persistent(DeviceState& D, const cdg_options& o, bool fp32, const void* b0, void* z0, unsigned* count,
                       int* err, cudaStream_t s) {
  PParams P = {};
  P.nlev = D.nlev;
  P.nu_pre = o.nu_pre;
  P.nu_post = o.nu_post;
  P.nc = D.nc;
  P.omega = o.omega;
  P.refine = (!fp32 && D.lev[D.nlev - 1].A != nullptr) ? 1 : 0;
  for (int l = 0; l < D.nlev; ++l) {
    const DevLevel& L = D.lev[l];
    if (L.np != D.np || L.ptrans) return false;
    PLevel& Q = P.lev[l];
    Q.n = L.n;
    Q.rowptr = L.rowptr;
    Q.col = L.col;
    Q.hrowptr = L.hrowptr;
    Q.hcol = L.hcol;
    Q.parent = L.parent;
    Q.childptr = L.childptr;
    Q.A = fp32 ? (const void*)L.A32 : (const void*)L.A;
    Q.Ahat = fp32 ? (const void*)L.Ahat32 : (const void*)L.Ahat;
    Q.Dinv = fp32 ? (const void*)L.Dinv32 : (const void*)L.Dinv;
    Q.L = fp32 ? (const void*)L.L32 : (const void*)L.L;
    Q.x = L.x;
    Q.t = L.t;
    Q.r = L.r;
    Q.b = L.b;
    Q.bh = L.bh;
  }
  if (P.refine) P.lev[D.nlev - 1].A = D.lev[D.nlev - 1].A;
  P.crow_seg = D.crow_seg;
  P.crow_off = D.crow_off;
  P.cinv_off = D.cinv_off;
  P.coarse_inv = D.coarse_inv;
  P.b0 = b0;
  P.z0 = z0;
  P.count = count;
  P.err = err;
  P.wait_limit = D.wait_limit < 0 ? kBarrierLimit : std::min(D.wait_limit, kBarrierLimit);
  cudaMemsetAsync(count, 0, 2 * sizeof(unsigned), s);
  int grid = 0, rc = -1;
  switch (D.np) {
    case 3: rc = fp32 ? launch_one<float, 3>(P, s, &grid) : launch_one<double, 3>(P, s, &grid); break;
    case 4: rc = fp32 ? launch_one<float, 4>(P, s, &grid) : launch_one<double, 4>(P, s, &grid); break;
    case 6: rc = fp32 ? launch_one<float, 6>(P, s, &grid) : launch_one<double, 6>(P, s, &grid); break;
    case 10: rc = fp32 ? launch_one<float, 10>(P, s, &grid) : launch_one<double, 10>(P, s, &grid); break;
    default: return false;
  }
  if (rc != 0) return false;
  count_launch();
  return true;
}
