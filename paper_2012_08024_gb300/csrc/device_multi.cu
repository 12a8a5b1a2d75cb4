// Many right-hand sides on one mesh (cdg_solve_multi): the same V-cycle
// preconditioned CG run for R columns at once.  Vectors are [n_l][n_p][R]
// (the R columns of one element's coefficient i are contiguous), so one block
// of an operator is read once per tile of columns: a CTA owns one to four
// block rows and a tile of columns, stages the rows' blocks in shared memory,
// and each thread applies them to one, two or four columns of the tile (the
// autotuner picks the shape).  The outer CG (residual, dots, updates, the
// level-0 operator) is FP64 with per-column scalars, its vector passes fused
// (the update also writes the FP32 copy of r for the V-cycle and the partial
// sums of r.r); the V-cycle runs on FP32 arithmetic on FP32 copies of the
// level operators, or (precision 2) on BF16 copies of the row-scaled smoother
// blocks D^-1(A - D) and of the transfer blocks (the residual operator and the
// block inverses stay FP32).  The level-0 operator can also run on the tensor
// cores by exact splitting (device_ozaki.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "device_kernels.cuh"
#include "device_state.h"

namespace {

using cdgk::cvt;
using cdgk::f32_to_f64;
using cdgk::f64_to_f32;

template <typename T>
struct Conv;
template <>
struct Conv<double> {
  static __device__ __forceinline__ double f(double v) { return v; }
};
template <>
struct Conv<float> {
  static __device__ __forceinline__ float f(float v) { return v; }
};
template <>
struct Conv<__nv_bfloat16> {
  static __device__ __forceinline__ float f(__nv_bfloat16 v) { return __bfloat162float(v); }
};

// the threads of one row group (threadIdx.y) copy ne values into shared memory
template <typename TA, typename TC>
__device__ __forceinline__ void stage_block(TC* s, const TA* a, int ne) {
  for (int t = threadIdx.x; t < ne; t += blockDim.x) s[t] = (TC)Conv<TA>::f(a[t]);
}

// y = A x (MODE 0), y = b - A x (1), y = x + omega (b - x - A x) (3; A = Ahat, b = D^-1 b).
// A CTA of blockDim (TX, BR) owns BR consecutive block rows and one tile of
// TX C right-hand sides: row group threadIdx.y stages its blocks in shared
// memory and thread x applies them to columns x + c TX (c < C) of the tile.
// Each block value read from shared memory feeds C fused multiply-adds, so
// with C = 1 the shared-memory reads, not the FMA pipe, set the pace.  TX, BR
// and C are the autotuned right-hand-side tile; every choice sums each column
// in the same order, so they change the timing only.
constexpr int kMrMaxBR = 4;

template <typename TA, typename TV, typename TC, int NP, int MODE, int C>
__device__ __forceinline__ void mr_bsr_body(int n, int R, const int* __restrict__ rowptr, const int* __restrict__ col,
                                            const TA* __restrict__ A, const TV* __restrict__ x,
                                            const TV* __restrict__ b, TV* __restrict__ y, TC omega) {
  __shared__ __align__(16) TC as[kMrMaxBR][NP * NP];
  const int BR = (int)blockDim.y, TX = (int)blockDim.x;
  const int K0 = blockIdx.x * BR;
  const int K = K0 + threadIdx.y;
  const int r0 = blockIdx.y * TX * C + threadIdx.x;
  int b0 = 0, nb = 0, nbmax = 0;
  for (int q = 0; q < BR; ++q) {
    if (K0 + q < n) {
      const int a0 = rowptr[K0 + q], cnt = rowptr[K0 + q + 1] - a0;
      nbmax = max(nbmax, cnt);
      if (q == (int)threadIdx.y) {
        b0 = a0;
        nb = cnt;
      }
    }
  }
  TC acc[C][NP];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[c][i] = TC(0);
  for (int t = 0; t < nbmax; ++t) {
    __syncthreads();
    if (t < nb) stage_block<TA, TC>(as[threadIdx.y], A + (size_t)(b0 + t) * NP * NP, NP * NP);
    __syncthreads();
    if (t < nb) {
      const TV* xj = x + (size_t)col[b0 + t] * NP * R;
      TC xv[C][NP];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int r = r0 + c * TX;
#pragma unroll
        for (int j = 0; j < NP; ++j) xv[c][j] = r < R ? (TC)xj[(size_t)j * R + r] : TC(0);
      }
#pragma unroll
      for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const TC a = as[threadIdx.y][i * NP + j];
#pragma unroll
          for (int c = 0; c < C; ++c) acc[c][i] = fma(a, xv[c][j], acc[c][i]);
        }
    }
  }
  if (K >= n) return;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int r = r0 + c * TX;
    if (r >= R) continue;
    const size_t base = (size_t)K * NP * R + r;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const size_t o = base + (size_t)i * R;
      if (MODE == 0) y[o] = (TV)acc[c][i];
      else if (MODE == 1) y[o] = (TV)((TC)b[o] - acc[c][i]);
      else y[o] = (TV)((TC)x[o] + omega * ((TC)b[o] - (TC)x[o] - acc[c][i]));
    }
  }
}

template <typename TA, typename TV, typename TC, int NP, int MODE, int C>
__global__ void mr_bsr_kernel(int n, int R, const int* __restrict__ rowptr, const int* __restrict__ col,
                              const TA* __restrict__ A, const TV* __restrict__ x, const TV* __restrict__ b,
                              TV* __restrict__ y, TC omega) {
  mr_bsr_body<TA, TV, TC, NP, MODE, C>(n, R, rowptr, col, A, x, b, y, omega);
}

// The same for CTAs of at most 128 threads, with the registers held so that
// eight such CTAs fit on an SM: the V-cycle sweeps wait on their x gathers,
// and more resident warps hide more of that latency (an autotuner choice).
template <typename TA, typename TV, typename TC, int NP, int MODE, int C>
__global__ void __launch_bounds__(128, 8) mr_bsr_kernel_lb(int n, int R, const int* __restrict__ rowptr,
                                                         const int* __restrict__ col, const TA* __restrict__ A,
                                                         const TV* __restrict__ x, const TV* __restrict__ b,
                                                         TV* __restrict__ y, TC omega) {
  mr_bsr_body<TA, TV, TC, NP, MODE, C>(n, R, rowptr, col, A, x, b, y, omega);
}

// per element K: out = B_K in (block-diagonal apply); with WRITE_X also x = omega out
template <typename TA, typename TV, int NP, bool WRITE_X>
__global__ void mr_diag_kernel(int R, const TA* __restrict__ B, const TV* __restrict__ in, TV* __restrict__ out,
                               TV* __restrict__ x, float omega) {
  __shared__ float as[NP * NP];
  const int K = blockIdx.x;
  const int r = threadIdx.x;
  stage_block<TA, float>(as, B + (size_t)K * NP * NP, NP * NP);
  __syncthreads();
  if (r >= R) return;
  const size_t base = (size_t)K * NP * R + r;
  float v[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) v[j] = (float)in[base + (size_t)j * R];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < NP; ++j) s = fmaf(as[i * NP + j], v[j], s);
    out[base + (size_t)i * R] = (TV)s;
    if (WRITE_X) x[base + (size_t)i * R] = (TV)(omega * s);
  }
}

// bc[A] = sum over children K of L_K^T r[K]
template <typename TA, typename TV, int NP>
__global__ void mr_restrict_kernel(int R, const int* __restrict__ childptr, const TA* __restrict__ L,
                                   const TV* __restrict__ rf, TV* __restrict__ bc) {
  __shared__ float ls[NP * NP];
  const int Ag = blockIdx.x;
  const int r = threadIdx.x;
  float acc[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) acc[i] = 0.f;
  for (int K = childptr[Ag]; K < childptr[Ag + 1]; ++K) {
    __syncthreads();
    stage_block<TA, float>(ls, L + (size_t)K * NP * NP, NP * NP);
    __syncthreads();
    if (r < R) {
      float v[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) v[j] = (float)rf[(size_t)K * NP * R + (size_t)j * R + r];
#pragma unroll
      for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[i] = fmaf(ls[j * NP + i], v[j], acc[i]);
    }
  }
  if (r >= R) return;
#pragma unroll
  for (int i = 0; i < NP; ++i) bc[(size_t)Ag * NP * R + (size_t)i * R + r] = (TV)acc[i];
}

// x[K] (+)= L_K xc[parent K]
template <typename TA, typename TV, int NP, bool ADD>
__global__ void mr_prolong_kernel(int R, const int* __restrict__ parent, const TA* __restrict__ L,
                                  const TV* __restrict__ xc, TV* __restrict__ x) {
  __shared__ float ls[NP * NP];
  const int K = blockIdx.x;
  const int r = threadIdx.x;
  stage_block<TA, float>(ls, L + (size_t)K * NP * NP, NP * NP);
  __syncthreads();
  if (r >= R) return;
  const TV* xa = xc + (size_t)parent[K] * NP * R + r;
  float v[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) v[j] = (float)xa[(size_t)j * R];
  const size_t base = (size_t)K * NP * R + r;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < NP; ++j) s = fmaf(ls[i * NP + j], v[j], s);
    x[base + (size_t)i * R] = ADD ? (TV)((float)x[base + (size_t)i * R] + s) : (TV)s;
  }
}

// coarsest (one mesh): x[row][r] = sum_j Ainv[row][j] b[j][r], FP64 accumulation
// in ascending j; a CTA owns CR consecutive rows and thread r one column, so
// each b value is widened once per CR rows
constexpr int kCoarseRows = 4;

template <typename TV, int CR>
__global__ void mr_coarse_kernel(int nc, int R, const double* __restrict__ Ainv, const TV* __restrict__ b,
                                 TV* __restrict__ x) {
  const int row0 = blockIdx.x * CR;
  const int r = threadIdx.x;
  if (r >= R) return;
  const int nr = min(CR, nc - row0);
  double s[CR];
#pragma unroll
  for (int q = 0; q < CR; ++q) s[q] = 0.0;
  for (int j = 0; j < nc; ++j) {
    const double bv = cvt<double>(b[(size_t)j * R + r]);
#pragma unroll
    for (int q = 0; q < CR; ++q)
      if (q < nr) s[q] = fma(Ainv[(size_t)(row0 + q) * nc + j], bv, s[q]);
  }
#pragma unroll
  for (int q = 0; q < CR; ++q)
    if (q < nr) x[(size_t)(row0 + q) * R + r] = cvt<TV>(s[q]);
}

template <typename TI, typename TO>
__global__ void mr_convert_kernel(size_t n, const TI* __restrict__ a, TO* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = cvt<TO>(a[i]);
}

// The per-column vector kernels of the outer CG share one partition: CTA g of
// G owns rows [nrows g / G, nrows (g + 1) / G) and thread r one column, so a
// column's partial sums run over its rows in ascending order whichever kernel
// forms them.  Rows go four at a time, all loads of a group before its
// arithmetic, to keep enough loads in flight per thread.
__device__ __forceinline__ void mr_rows(int nrows, int G, int g, int& lo, int& hi) {
  lo = (int)((long long)nrows * g / G);
  hi = (int)((long long)nrows * (g + 1) / G);
}

// per-column partial dots over a chunk of rows: partial[g][r] = sum x y (and
// partial[G + g][r] = sum x w); Y is FP64 or FP32 (a V-cycle output, widened exactly)
template <typename TY>
__global__ void mr_dot_kernel(int nrows, int R, int G, const double* __restrict__ x, const TY* __restrict__ y,
                              const TY* __restrict__ w, double* __restrict__ partial) {
  const int g = blockIdx.x, r = threadIdx.x;
  if (r >= R) return;
  int lo, hi;
  mr_rows(nrows, G, g, lo, hi);
  double s = 0.0, s2 = 0.0;
  int row = lo;
  for (; row + 4 <= hi; row += 4) {
    // all loads of the group first (raw words), conversions after: a
    // conversion's branch between two loads would keep them from overlapping
    double xv[4];
    TY yv[4], wv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t o = (size_t)(row + u) * R + r;
      xv[u] = x[o];
      yv[u] = y[o];
      wv[u] = w ? w[o] : TY(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      s = fma(xv[u], cvt<double>(yv[u]), s);
      if (w) s2 = fma(xv[u], cvt<double>(wv[u]), s2);
    }
  }
  for (; row < hi; ++row) {
    const size_t o = (size_t)row * R + r;
    s = fma(x[o], cvt<double>(y[o]), s);
    if (w) s2 = fma(x[o], cvt<double>(w[o]), s2);
  }
  partial[(size_t)g * R + r] = s;
  if (w) partial[(size_t)(G + g) * R + r] = s2;
}

// per column: sum the G partials in order and update that column's CG scalars
// (same rules as the single-column finalize: which 0 PQ, 1 RR, 2 RZ, 3 BB, 4 initial RR)
__global__ void mr_finalize_kernel(int R, int G, const double* __restrict__ partial, int which, int flexible,
                                   double tol, double* __restrict__ scal) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double tot = 0.0, tot2 = 0.0;
  for (int g = 0; g < G; ++g) tot += partial[(size_t)g * R + r];
  if (which == 2 && flexible)
    for (int g = 0; g < G; ++g) tot2 += partial[(size_t)(G + g) * R + r];
  double* sc = scal + (size_t)r * S_COUNT;
  const bool done = sc[S_DONE] != 0.0;
  if (which == 0) {
    sc[S_PQ] = tot;
    if (!done && !(tot > 0.0)) {
      sc[S_BREAK] = 1.0;
      sc[S_DONE] = 1.0;
    }
    sc[S_ALPHA] = sc[S_DONE] != 0.0 ? 0.0 : sc[S_RZ] / tot;
  } else if (which == 1 || which == 4) {
    if (!done) {
      sc[S_RR] = tot;
      if (which == 1) sc[S_IT] += 1.0;
      if (!isfinite(tot)) {
        sc[S_BREAK] = 1.0;
        sc[S_DONE] = 1.0;
      } else if (sqrt(tot) <= tol * sqrt(sc[S_BB])) {
        sc[S_DONE] = 1.0;
      }
    }
  } else if (which == 2) {
    const double rz_old = sc[S_RZ];
    sc[S_BETA] = done ? 0.0 : (flexible ? (tot - tot2) / rz_old : tot / rz_old);
    sc[S_RZ] = tot;
  } else {
    sc[S_BB] = tot;
    if (!(tot > 0.0)) sc[S_DONE] = 1.0;
  }
}

// x += alpha_r p; r -= alpha_r q per column, with the FP32 copy of r that the
// V-cycle reads and the partial r.r of the chunk (the sum mr_dot_kernel forms)
__global__ void mr_update_kernel(int nrows, int R, int G, const double* __restrict__ scal,
                                 const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                                 double* __restrict__ res, float* __restrict__ r32, double* __restrict__ partial) {
  const int g = blockIdx.x, r = threadIdx.x;
  if (r >= R) return;
  int lo, hi;
  mr_rows(nrows, G, g, lo, hi);
  const double a = scal[(size_t)r * S_COUNT + S_ALPHA];
  double s = 0.0;
  int row = lo;
  for (; row + 4 <= hi; row += 4) {
    double pv[4], qv[4], xv[4], rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t o = (size_t)(row + u) * R + r;
      pv[u] = p[o];
      qv[u] = q[o];
      xv[u] = x[o];
      rv[u] = res[o];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t o = (size_t)(row + u) * R + r;
      x[o] = fma(a, pv[u], xv[u]);
      const double v = fma(-a, qv[u], rv[u]);
      res[o] = v;
      r32[o] = f64_to_f32(v);
      s = fma(v, v, s);
    }
  }
  for (; row < hi; ++row) {
    const size_t o = (size_t)row * R + r;
    x[o] = fma(a, p[o], x[o]);
    const double v = fma(-a, q[o], res[o]);
    res[o] = v;
    r32[o] = f64_to_f32(v);
    s = fma(v, v, s);
  }
  partial[(size_t)g * R + r] = s;
}

// p = z + beta_r p per column (p = z on the first step); z is the V-cycle's FP32 output.
// With maxb, also the largest biased FP64 exponent of each column of the new p
// (atomicMax over the CTAs; maxb zeroed before), which the split apply needs
__device__ __forceinline__ int biased_exp(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF);
}

__global__ void mr_p_kernel(int nrows, int R, int G, const double* __restrict__ scal, int first,
                            const float* __restrict__ z, double* __restrict__ p, int* __restrict__ maxb) {
  const int g = blockIdx.x, r = threadIdx.x;
  if (r >= R) return;
  int lo, hi;
  mr_rows(nrows, G, g, lo, hi);
  const double beta = first ? 0.0 : scal[(size_t)r * S_COUNT + S_BETA];
  int em = 0;
  int row = lo;
  for (; row + 4 <= hi; row += 4) {
    float zv[4];   // raw words first, conversions after (see mr_dot_kernel)
    double pv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t o = (size_t)(row + u) * R + r;
      zv[u] = z[o];
      pv[u] = first ? 0.0 : p[o];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double zo = f32_to_f64(zv[u]);
      const double v = first ? zo : fma(beta, pv[u], zo);
      p[(size_t)(row + u) * R + r] = v;
      em = max(em, biased_exp(v));
    }
  }
  for (; row < hi; ++row) {
    const size_t o = (size_t)row * R + r;
    const double zo = f32_to_f64(z[o]);
    const double v = first ? zo : fma(beta, p[o], zo);
    p[o] = v;
    em = max(em, biased_exp(v));
  }
  if (maxb) atomicMax(maxb + r, em);
}

// b[k][i][r] = sum_q w_q phi_i(x_q) f[r][K][q], K = perm0[k]  (f only; zero boundary data)
template <int NP>
__global__ void mr_rhs_kernel(int R, int nq, int ne, const int* __restrict__ perm0, const double* __restrict__ V,
                              const double* __restrict__ f, double* __restrict__ b) {
  const int k = blockIdx.x, r = threadIdx.x;
  if (r >= R) return;
  const size_t K = perm0[k];
  const double* fk = f + ((size_t)r * ne + K) * nq;
  const double* Vk = V + (size_t)k * nq * NP;
  double s[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) s[i] = 0.0;
  for (int q = 0; q < nq; ++q) {
    const double fv = fk[q];
#pragma unroll
    for (int i = 0; i < NP; ++i) s[i] = fma(Vk[q * NP + i], fv, s[i]);
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) b[((size_t)k * NP + i) * R + r] = s[i];
}

// u[r][K][i] = x[k][i][r] (user layout: one contiguous solution per column)
__global__ void mr_out_kernel(int R, int np, const int* __restrict__ perm0, const double* __restrict__ x,
                              int ne, double* __restrict__ u) {
  const int k = blockIdx.x, r = threadIdx.x;
  if (r >= R) return;
  const size_t K = perm0[k];
  for (int i = 0; i < np; ++i) u[((size_t)r * ne + K) * np + i] = x[((size_t)k * np + i) * R + r];
}

}  // namespace

struct MRLevel {
  void* A = nullptr;      // V-cycle operator copies (FP32 or BF16)
  void* Ahat = nullptr;
  void* Dinv = nullptr;
  void* L = nullptr;
  float *x = nullptr, *t = nullptr, *r = nullptr, *b = nullptr, *bh = nullptr;
};

struct MR {
  int R = 0, G = 0;
  bool bf16 = false;
  MRLevel lev[kMaxLev];
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *bt = nullptr;
  // FP32 V-cycle input r32 and output z32; z32old holds the previous output
  // (flexible CG), the two swap roles every step
  float *r32 = nullptr, *z32 = nullptr, *z32old = nullptr;
  double* scal = nullptr;      // [R][S_COUNT]
  double* partial = nullptr;   // [2G][R]
  // autotuned (right-hand-side tile width, block rows per CTA) of mr_bsr_kernel per
  // level and mode (0 FP64 level-0 apply, 1 residual, 3 smoother sweep); 0 = not tuned
  int tile[kMaxLev][4] = {};
  int rows[kMaxLev][4] = {};
  int cols[kMaxLev][4] = {};   // right-hand sides per thread
  int lb[kMaxLev][4] = {};     // 1: the register-capped instance (CTAs of at most 128 threads)
  bool tuned = false;
  bool tc = false;             // smoother sweeps on tcgen05 (BF16 blocks)
  int* tc_err = nullptr;       // set by a tensor-core kernel whose wait timed out
  // FP64 level-0 apply on tcgen05 by exact splitting: B operand images of the
  // slices of A_0, row exponents, slices of x and column exponents (device_ozaki.cu)
  bool oz = false;
  void* oz_img = nullptr;
  int* oz_eA = nullptr;
  void* oz_xs = nullptr;
  int* oz_maxb = nullptr;
};

void mr_tuning(const MR& M, int level, int nlev, int32_t* out) {
  if (!M.tuned) return;
  if (level + 1 < nlev) {
    out[4] = M.tile[level][3];
    out[5] = M.rows[level][3];
    out[6] = M.tile[level][1];
    out[7] = M.rows[level][1];
    out[10] = M.cols[level][3];
    out[11] = M.cols[level][1];
  }
  if (level == 0) {
    out[8] = M.tile[0][0];
    out[9] = M.rows[0][0];
    out[12] = M.cols[0][0];
  }
}

namespace {

struct MRCarver {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

template <typename TA>
void upload_conv(void* dst, const std::vector<double>& src, cudaStream_t s) {
  if (src.empty()) return;
  std::vector<TA> h(src.size());
  for (size_t i = 0; i < src.size(); ++i) h[i] = (TA)src[i];
  cudaMemcpyAsync(dst, h.data(), sizeof(TA) * h.size(), cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
}

}  // namespace

MR* mr_new() { return new MR(); }
void mr_delete(MR* m) { delete m; }

// Carves the multi-column buffers after `off`; returns the new end offset.
size_t mr_layout(const cdg::Hierarchy& H, int R, int precision, int tc_fp64, MR* mr, char* base, size_t off) {
  MRCarver c{base, off};
  MR tmp;
  MR& M = mr ? *mr : tmp;
  M.R = R;
  M.G = 2 * 152;
  M.bf16 = precision == 2;
  const size_t ts = M.bf16 ? sizeof(__nv_bfloat16) : sizeof(float);
  const int np = H.np;
  const size_t nb2 = (size_t)np * np;
  const int nlev = (int)H.lev.size();
  for (int l = 0; l < nlev; ++l) {
    MRLevel& L = M.lev[l];
    const size_t n = (size_t)H.lev[l].n;
    // the residual operator stays FP32 in every mode: b - A x cancels, and BF16
    // blocks (8-bit significands) would leave only noise in a small residual
    L.A = c.take<char>(H.A_t[l].val.size() * sizeof(float));
    if (l + 1 < nlev) {
      L.Ahat = c.take<char>(std::max<size_t>(1, H.Ahat_t[l].val.size()) * ts);
      // block inverses stay FP32 too: with C_D = gamma/h_avg a diagonal block reaches
      // cond ~1e5, and an 8-bit rounding of its inverse is then no inverse at all
      L.Dinv = c.take<char>(n * nb2 * sizeof(float));
      L.L = c.take<char>(n * nb2 * ts);
    }
    L.x = c.take<float>(n * np * R);
    L.t = c.take<float>(n * np * R);
    L.r = c.take<float>(n * np * R);
    L.b = c.take<float>(n * np * R);
    L.bh = c.take<float>(n * np * R);
  }
  const size_t nv = (size_t)H.mesh.ne * np * R;
  M.x = c.take<double>(nv);
  M.r = c.take<double>(nv);
  M.p = c.take<double>(nv);
  M.q = c.take<double>(nv);
  M.bt = c.take<double>(nv);
  M.r32 = c.take<float>(nv);
  M.z32 = c.take<float>(nv);
  M.z32old = c.take<float>(nv);
  M.scal = c.take<double>((size_t)R * S_COUNT);
  M.partial = c.take<double>((size_t)2 * M.G * R);
  M.tc_err = c.take<int>(1);
  M.oz = tc_fp64 != 0 && oz_feasible(H.A_t[0], np);
  if (M.oz) {
    M.oz_img = c.take<char>(oz_image_bytes(H.A_t[0]));
    M.oz_eA = c.take<int>((size_t)H.lev[0].n * 16);
    M.oz_xs = c.take<char>(oz_xslice_bytes(H.lev[0].n, np, R));
    M.oz_maxb = c.take<int>(R);
  }
  return c.off;
}

void mr_upload(const cdg::Hierarchy& H, MR& M, cudaStream_t s) {
  const int nlev = (int)H.lev.size();
  for (int l = 0; l < nlev; ++l) {
    MRLevel& L = M.lev[l];
    auto up = [&](void* dst, const std::vector<double>& src) {
      if (!dst) return;
      if (M.bf16) upload_conv<__nv_bfloat16>(dst, src, s);
      else upload_conv<float>(dst, src, s);
    };
    upload_conv<float>(L.A, H.A_t[l].val, s);
    if (l + 1 < nlev) {
      up(L.Ahat, H.Ahat_t[l].val);
      upload_conv<float>(L.Dinv, H.Dinv_t[l], s);
      up(L.L, H.L_t[l]);
    }
  }
  if (M.oz) {
    std::vector<uint16_t> img;
    std::vector<int32_t> eA;
    if (oz_prepare(H.A_t[0], H.np, img, eA)) {
      cudaMemcpyAsync(M.oz_img, img.data(), sizeof(uint16_t) * img.size(), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(M.oz_eA, eA.data(), sizeof(int32_t) * eA.size(), cudaMemcpyHostToDevice, s);
      cudaStreamSynchronize(s);
    } else {
      M.oz = false;
    }
  }
}

namespace {

#define MR_NP_DISPATCH(NPV, ...)                            \
  switch (NPV) {                                            \
    case 3: { constexpr int NP = 3; __VA_ARGS__; break; }   \
    case 4: { constexpr int NP = 4; __VA_ARGS__; break; }   \
    case 6: { constexpr int NP = 6; __VA_ARGS__; break; }   \
    case 10: { constexpr int NP = 10; __VA_ARGS__; break; } \
    default: return false;                                  \
  }

// the same dispatch inside void lambdas (an unsupported n_p launches nothing)
#define MR_NP_DISPATCH_V(NPV, ...)                          \
  switch (NPV) {                                            \
    case 3: { constexpr int NP = 3; __VA_ARGS__; break; }   \
    case 4: { constexpr int NP = 4; __VA_ARGS__; break; }   \
    case 6: { constexpr int NP = 6; __VA_ARGS__; break; }   \
    case 10: { constexpr int NP = 10; __VA_ARGS__; break; } \
    default: break;                                         \
  }

inline unsigned threads_for(int R) { return (unsigned)(((R + 31) / 32) * 32); }

// threads per CTA that a kernel's register use allows (cached per instance)
template <typename Kern>
int max_threads_of(Kern k) {
  cudaFuncAttributes a{};
  return cudaFuncGetAttributes(&a, (const void*)k) == cudaSuccess ? a.maxThreadsPerBlock : 256;
}

template <typename TA, typename TV, typename TC, int NP, int MODE, int C>
void mr_bsr_launch_c(int tx, int br, bool lb, int n, int R, const int* rp, const int* cl, const TA* A, const TV* x,
                     const TV* b, TV* y, TC omega, cudaStream_t s) {
  if constexpr (C <= 2 && sizeof(TC) == 4) {   // the register-capped instance: FP32 arithmetic, <= 2 columns
    if (lb && tx * std::min(std::max(br, 1), kMrMaxBR) <= 128) {
      br = std::min(std::max(br, 1), kMrMaxBR);
      const dim3 grid((unsigned)((n + br - 1) / br), (unsigned)((R + tx * C - 1) / (tx * C))),
          block((unsigned)tx, (unsigned)br);
      mr_bsr_kernel_lb<TA, TV, TC, NP, MODE, C><<<grid, block, 0, s>>>(n, R, rp, cl, A, x, b, y, omega);
      count_launch();
      return;
    }
  }
  static const int mt = max_threads_of(mr_bsr_kernel<TA, TV, TC, NP, MODE, C>);
  br = std::min(std::max(br, 1), kMrMaxBR);
  // a CTA larger than the register file allows runs as fewer block rows, then
  // narrower tiles: the same columns in the same order, so the same results
  while (tx * br > mt && br > 1) br /= 2;
  while (tx * br > mt && tx > 32) tx /= 2;
  const dim3 grid((unsigned)((n + br - 1) / br), (unsigned)((R + tx * C - 1) / (tx * C))),
      block((unsigned)tx, (unsigned)br);
  mr_bsr_kernel<TA, TV, TC, NP, MODE, C><<<grid, block, 0, s>>>(n, R, rp, cl, A, x, b, y, omega);
  count_launch();
}

// mr_bsr_kernel with tx threads across the right-hand sides, rc columns per
// thread (a tile of tx rc columns) and br block rows per CTA
template <typename TA, typename TV, typename TC, int NP, int MODE>
void mr_bsr_launch(int tx, int br, int rc, bool lb, int n, int R, const int* rp, const int* cl, const TA* A,
                   const TV* x, const TV* b, TV* y, TC omega, cudaStream_t s) {
  if (rc >= 4) mr_bsr_launch_c<TA, TV, TC, NP, MODE, 4>(tx, br, lb, n, R, rp, cl, A, x, b, y, omega, s);
  else if (rc == 2) mr_bsr_launch_c<TA, TV, TC, NP, MODE, 2>(tx, br, lb, n, R, rp, cl, A, x, b, y, omega, s);
  else mr_bsr_launch_c<TA, TV, TC, NP, MODE, 1>(tx, br, lb, n, R, rp, cl, A, x, b, y, omega, s);
}

inline int tile_of(const MR& M, int l, int mode) { return M.tile[l][mode] ? M.tile[l][mode] : (int)threads_for(M.R); }
inline int rows_of(const MR& M, int l, int mode) { return M.rows[l][mode] ? M.rows[l][mode] : 1; }
inline int cols_of(const MR& M, int l, int mode) { return M.cols[l][mode] ? M.cols[l][mode] : 1; }
inline bool lb_of(const MR& M, int l, int mode) { return M.lb[l][mode] != 0; }

template <typename TA>
bool mr_vcycle(DeviceState& D, MR& M, const cdg_options& o, const float* b0, float* z0, cudaStream_t s) {
  const int np = D.np, nlev = D.nlev, R = M.R;
  const unsigned T = threads_for(R);
  const float w = (float)o.omega;
  auto bsr = [&](int mode, int l, const int* rp, const int* cl, const void* A, const float* x, const float* b,
                 float* y) -> bool {
    const int n = D.lev[l].n;
    if (mode == 3 && M.tc)
      return mr_tc_smooth(np, n, R, rp, cl, A, x, b, y, w, M.tc_err, D.wait_limit, s);
    const int tx = tile_of(M, l, mode), br = rows_of(M, l, mode), rc = cols_of(M, l, mode);
    const bool lb = lb_of(M, l, mode);
    MR_NP_DISPATCH(np, {
      if (mode == 1)
        mr_bsr_launch<float, float, float, NP, 1>(tx, br, rc, lb, n, R, rp, cl, (const float*)A, x, b, y, w, s);
      else
        mr_bsr_launch<TA, float, float, NP, 3>(tx, br, rc, lb, n, R, rp, cl, (const TA*)A, x, b, y, w, s);
    });
    return true;
  };
  if (nlev == 1) {
    mr_coarse_kernel<float, kCoarseRows><<<(D.nc + kCoarseRows - 1) / kCoarseRows, T, 0, s>>>(D.nc, R, D.coarse_inv,
                                                                                            b0, z0);
    count_launch();
    return true;
  }
  std::vector<const float*> bl(nlev);
  bl[0] = b0;
  for (int l = 1; l < nlev; ++l) bl[l] = M.lev[l].b;
  for (int l = 0; l + 1 < nlev; ++l) {
    MRLevel& L = M.lev[l];
    const DevLevel& DL = D.lev[l];
    float* x = L.x;
    float* t = L.t;
    const float* b = bl[l];
    if (o.nu_pre >= 1) {
      MR_NP_DISPATCH(np, mr_diag_kernel<float, float, NP, true><<<DL.n, T, 0, s>>>(R, (const float*)L.Dinv, b, L.bh, x, w));
      count_launch();
      for (int k = 1; k < o.nu_pre; ++k) {
        if (!bsr(3, l, DL.hrowptr, DL.hcol, L.Ahat, x, L.bh, t)) return false;
        std::swap(x, t);
      }
      if (!bsr(1, l, DL.rowptr, DL.col, L.A, x, b, L.r)) return false;
      MR_NP_DISPATCH(np, mr_restrict_kernel<TA, float, NP><<<D.lev[l + 1].n, T, 0, s>>>(
                             R, D.lev[l + 1].childptr, (const TA*)L.L, L.r, M.lev[l + 1].b));
      count_launch();
      L.x = x;
      L.t = t;
    } else {
      MR_NP_DISPATCH(np, mr_diag_kernel<float, float, NP, false><<<DL.n, T, 0, s>>>(R, (const float*)L.Dinv, b,
                                                                                    L.bh, (float*)nullptr, w));
      MR_NP_DISPATCH(np, mr_restrict_kernel<TA, float, NP><<<D.lev[l + 1].n, T, 0, s>>>(
                             R, D.lev[l + 1].childptr, (const TA*)L.L, b, M.lev[l + 1].b));
      count_launch(2);
    }
  }
  mr_coarse_kernel<float, kCoarseRows><<<(D.nc + kCoarseRows - 1) / kCoarseRows, T, 0, s>>>(
      D.nc, R, D.coarse_inv, M.lev[nlev - 1].b, M.lev[nlev - 1].x);
  count_launch();
  for (int l = nlev - 2; l >= 0; --l) {
    MRLevel& L = M.lev[l];
    const DevLevel& DL = D.lev[l];
    float* x = L.x;
    float* t = L.t;
    if (o.nu_pre >= 1) {
      MR_NP_DISPATCH(np, mr_prolong_kernel<TA, float, NP, true><<<DL.n, T, 0, s>>>(R, DL.parent, (const TA*)L.L,
                                                                                   M.lev[l + 1].x, x));
    } else {
      MR_NP_DISPATCH(np, mr_prolong_kernel<TA, float, NP, false><<<DL.n, T, 0, s>>>(R, DL.parent, (const TA*)L.L,
                                                                                    M.lev[l + 1].x, x));
    }
    count_launch();
    for (int k = 0; k < o.nu_post; ++k) {
      float* out = (l == 0 && k + 1 == o.nu_post) ? z0 : t;
      if (!bsr(3, l, DL.hrowptr, DL.hcol, L.Ahat, x, L.bh, out)) return false;
      if (out == t) std::swap(x, t);
      else x = out;
    }
    if (l == 0 && o.nu_post == 0)
      cudaMemcpyAsync(z0, x, sizeof(float) * (size_t)DL.n * np * R, cudaMemcpyDeviceToDevice, s);
    if (l > 0 && x != L.x) {
      L.t = L.x;
      L.x = x;
    }
  }
  return true;
}

// maxb_ready: the column exponents of x are already in M.oz_maxb (mr_p_kernel
// stores them for p); pq_groups (split apply only): the apply also leaves the
// partial sums of x . y in M.partial, *pq_groups of them per column
bool mr_apply64(DeviceState& D, MR& M, const double* x, double* y, cudaStream_t s, bool maxb_ready = false,
                int* pq_groups = nullptr) {
  const DevLevel& L0 = D.lev[0];
  if (M.oz)
    return oz_apply(D.np, L0.n, M.R, L0.rowptr, L0.col, M.oz_img, M.oz_eA, M.oz_xs, M.oz_maxb, maxb_ready, x, y,
                    pq_groups ? M.partial : nullptr, pq_groups, M.tc_err, D.wait_limit, s);
  const int tx = tile_of(M, 0, 0), br = rows_of(M, 0, 0), rc = cols_of(M, 0, 0);
  MR_NP_DISPATCH(D.np, (mr_bsr_launch<double, double, double, NP, 0>(tx, br, rc, false, L0.n, M.R, L0.rowptr, L0.col,
                                                                     L0.A,
                                                                     x, (const double*)nullptr, y, 0.0, s)));
  return true;
}

// Autotuner of the multi-right-hand-side block-sparse kernel: for every level
// and mode the solve launches, times the (tile width, block rows per CTA)
// pairs with tile width in {32, ..., 1024} up to the padded R and at most 1024
// threads per CTA, on the handle's operators and zero-filled work vectors, and
// keeps the fastest.
template <typename TA>
bool mr_autotune(DeviceState& D, MR& M, double omega, cudaStream_t s) {
  const int np = D.np, nlev = D.nlev, R = M.R;
  const int tmax = (int)threads_for(R);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return false;
  auto pick = [&](int l, int mode, auto&& launch_one) {
    float tbest = 3.0e38f;
    for (int rc : {1, 2, 4}) {
      for (int tx = 32; tx <= 1024; tx *= 2) {
        if (tx * rc > tmax && tx != 32) break;
        if (rc > 1 && tx * rc > tmax) break;   // a thread's extra columns would all be padding
        for (int br : {1, 2, 4}) {
          if (tx * br > 1024) continue;
          // the register-capped instance exists for FP32 arithmetic, CTAs of <= 128 threads, rc <= 2
          const bool lb_ok = mode != 0 && rc <= 2 && tx * br <= 128;
          for (int lb = 0; lb <= (lb_ok ? 1 : 0); ++lb) {
            const float t = time_calls(s, e0, e1, 2, [&] { launch_one(tx, br, rc, lb != 0); });
            if (t < tbest) {
              tbest = t;
              M.tile[l][mode] = tx;
              M.rows[l][mode] = br;
              M.cols[l][mode] = rc;
              M.lb[l][mode] = lb;
            }
          }
        }
      }
    }
  };
  bool ok = true;
  if (!M.oz) {   // the FP64 CUDA-core apply (the split apply has no variants)
    const DevLevel& L0 = D.lev[0];
    const size_t nv = (size_t)L0.n * np * R;
    cudaMemsetAsync(M.p, 0, nv * sizeof(double), s);
    pick(0, 0, [&](int tx, int br, int rc, bool) {
      MR_NP_DISPATCH_V(np, (mr_bsr_launch<double, double, double, NP, 0>(tx, br, rc, false, L0.n, R, L0.rowptr, L0.col,
                                                                         L0.A,
                                                                         (const double*)M.p, (const double*)nullptr,
                                                                         M.q, 0.0, s)));
    });
  }
  const float w = (float)omega;
  for (int l = 0; l + 1 < nlev; ++l) {
    const DevLevel& DL = D.lev[l];
    MRLevel& L = M.lev[l];
    const size_t nv = (size_t)DL.n * np * R;
    for (float* v : {L.x, L.b, L.bh, L.t}) cudaMemsetAsync(v, 0, nv * sizeof(float), s);
    pick(l, 1, [&](int tx, int br, int rc, bool lb) {
      MR_NP_DISPATCH_V(np, (mr_bsr_launch<float, float, float, NP, 1>(tx, br, rc, lb, DL.n, R, DL.rowptr, DL.col,
                                                                      (const float*)L.A, (const float*)L.x,
                                                                      (const float*)L.b, L.t, w, s)));
    });
    pick(l, 3, [&](int tx, int br, int rc, bool lb) {
      MR_NP_DISPATCH_V(np, (mr_bsr_launch<TA, float, float, NP, 3>(tx, br, rc, lb, DL.n, R, DL.hrowptr, DL.hcol,
                                                                   (const TA*)L.Ahat, (const float*)L.x,
                                                                   (const float*)L.bh, L.t, w, s)));
    });
  }
  ok = cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  M.tuned = ok;
  return ok;
}

// sums G partials per column (G = M.G unless given) into the CG scalars
void mr_finalize(MR& M, int which, bool flexible, double tol, cudaStream_t s, int G = 0) {
  mr_finalize_kernel<<<(M.R + 127) / 128, 128, 0, s>>>(M.R, G > 0 ? G : M.G, M.partial, which, flexible ? 1 : 0, tol,
                                                         M.scal);
  count_launch();
}

template <typename TY>
void mr_dot(DeviceState& D, MR& M, const double* x, const TY* y, const TY* w, int which, double tol, cudaStream_t s) {
  const int nrows = (int)(D.ne * D.np);
  const unsigned T = threads_for(M.R);
  mr_dot_kernel<TY><<<M.G, T, 0, s>>>(nrows, M.R, M.G, x, y, w, M.partial);
  mr_finalize(M, which, w != nullptr, tol, s);
}

}  // namespace

// Solves A_0 U = B for R columns: f_q [R][n_elements][nq] (device), u [R][n_elements][n_p]
// (device), res_hist [R][maxit+1] and iters [R] (host).
int dev_solve_multi(cdg_handle* h, const double* f_q, double* u, double* res_hist, int* iters, void* stream) {
  if (!h->dev || !h->dev->mr) {
    h->err = "cdg_solve_multi needs a handle created with nrhs > 0 and bound to a device buffer";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  MR& M = *D.mr;
  const cdg_options& o = h->opt;
  const int R = M.R;
  if (D.np != 3 && D.np != 4 && D.np != 6 && D.np != 10) {   // cdg_create rejects these already
    h->err = "unsupported n_p for cdg_solve_multi";
    return CDG_EINVAL;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  cudaStream_t s = D.stream;
  cudaEventRecord(D.ev_in, cs);
  cudaStreamWaitEvent(s, D.ev_in, 0);
  const size_t nv = (size_t)D.ne * D.np * R;
  const size_t nrows = (size_t)D.ne * D.np;
  const unsigned T = threads_for(R);
  const unsigned gv = 4 * 152;
  bool ok = true;
  if (o.autotune && !M.tuned) {
    ok = M.bf16 ? mr_autotune<__nv_bfloat16>(D, M, o.omega, s) : mr_autotune<float>(D, M, o.omega, s);
    if (!ok) {
      h->err = "cdg_solve_multi: autotuning failed (unsupported n_p or a CUDA error)";
      return CDG_ECUDA;
    }
  }
  cudaMemsetAsync(M.scal, 0, sizeof(double) * (size_t)R * S_COUNT, s);
  M.tc = M.bf16 && o.tensor_cores != 0 && D.np <= 16;
  if (M.tc || M.oz) cudaMemsetAsync(M.tc_err, 0, sizeof(int), s);
  MR_NP_DISPATCH(D.np, mr_rhs_kernel<NP><<<(unsigned)D.ne, T, 0, s>>>(R, D.nq, (int)D.ne, D.perm0, D.rhs_vol, f_q, M.bt));
  count_launch();
  cudaMemsetAsync(M.x, 0, sizeof(double) * nv, s);
  cudaMemcpyAsync(M.r, M.bt, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s);
  mr_dot<double>(D, M, M.bt, M.bt, nullptr, 3, o.tol, s);
  mr_dot<double>(D, M, M.r, M.r, nullptr, 4, o.tol, s);
  // the V-cycle maps r32 (FP32 copy of r, written by mr_update_kernel after the
  // first step) to z32; z = z32 widened exactly, so the FP64 steps read z32
  auto precond = [&]() -> bool {
    return M.bf16 ? mr_vcycle<__nv_bfloat16>(D, M, o, M.r32, M.z32, s) : mr_vcycle<float>(D, M, o, M.r32, M.z32, s);
  };
  std::vector<double> hs((size_t)R * S_COUNT);
  cudaMemcpyAsync(hs.data(), M.scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    h->err = std::string("solve_multi: ") + cudaGetErrorString(e);
    return CDG_ECUDA;
  }
  const int stride = o.maxit + 1;
  auto rel = [&](int r) {
    const double* sc = &hs[(size_t)r * S_COUNT];
    return sc[S_BB] > 0.0 ? std::sqrt(sc[S_RR] / sc[S_BB]) : 0.0;
  };
  std::vector<char> done(R, 0);
  int ndone = 0, status = CDG_OK, it = 0;
  for (int r = 0; r < R; ++r) {
    iters[r] = 0;
    if (res_hist) res_hist[(size_t)r * stride] = rel(r);
    if (hs[(size_t)r * S_COUNT + S_DONE] != 0.0) {
      done[r] = 1;
      ++ndone;
    }
  }
  if (ndone < R) {
    mr_convert_kernel<double, float><<<gv, 256, 0, s>>>(nv, M.r, M.r32);
    count_launch();
    ok = precond();
    mr_dot<float>(D, M, M.r, M.z32, nullptr, 2, o.tol, s);
    if (M.oz) cudaMemsetAsync(M.oz_maxb, 0, sizeof(int) * R, s);
    mr_p_kernel<<<M.G, T, 0, s>>>((int)nrows, R, M.G, M.scal, 1, M.z32, M.p, M.oz ? M.oz_maxb : nullptr);
    count_launch();
    while (ok) {
      if (it >= o.maxit) {
        status = CDG_ENOCONV;
        break;
      }
      if (M.oz) {   // p's column exponents come from mr_p_kernel, p . A p from the apply's epilogue
        int gq = 0;
        ok = mr_apply64(D, M, M.p, M.q, s, true, &gq);
        mr_finalize(M, 0, false, o.tol, s, gq);
      } else {
        ok = mr_apply64(D, M, M.p, M.q, s);
        mr_dot<double>(D, M, M.p, M.q, nullptr, 0, o.tol, s);
      }
      mr_update_kernel<<<M.G, T, 0, s>>>((int)nrows, R, M.G, M.scal, M.p, M.q, M.x, M.r, M.r32, M.partial);
      count_launch();
      mr_finalize(M, 1, false, o.tol, s);
      cudaMemcpyAsync(hs.data(), M.scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s);
      int tc_err_it = 0;
      if (M.tc || M.oz) cudaMemcpyAsync(&tc_err_it, M.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        h->err = std::string("solve_multi: ") + cudaGetErrorString(e);
        return CDG_ECUDA;
      }
      if (tc_err_it) break;   // a sweep gave up: its rows are not smoothed; reported below
      ++it;
      for (int r = 0; r < R; ++r) {
        if (done[r]) continue;
        iters[r] = it;
        if (res_hist) res_hist[(size_t)r * stride + it] = rel(r);
        const double* sc = &hs[(size_t)r * S_COUNT];
        if (sc[S_DONE] != 0.0) {
          done[r] = 1;
          ++ndone;
          if (sc[S_BREAK] != 0.0) {
            status = CDG_EBREAKDOWN;
            h->err = "CG breakdown in column " + std::to_string(r);
          }
        }
      }
      if (ndone == R) break;
      std::swap(M.z32, M.z32old);
      ok = precond();
      mr_dot<float>(D, M, M.r, M.z32, M.z32old, 2, o.tol, s);
      if (M.oz) cudaMemsetAsync(M.oz_maxb, 0, sizeof(int) * R, s);
      mr_p_kernel<<<M.G, T, 0, s>>>((int)nrows, R, M.G, M.scal, 0, M.z32, M.p, M.oz ? M.oz_maxb : nullptr);
      count_launch();
    }
  }
  if (!ok) {
    h->err = "unsupported n_p for cdg_solve_multi";
    return CDG_EINVAL;
  }
  mr_out_kernel<<<(unsigned)D.ne, T, 0, s>>>(R, D.np, D.perm0, M.x, (int)D.ne, u);
  count_launch();
  int tc_err = 0;
  if (M.tc || M.oz) cudaMemcpyAsync(&tc_err, M.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->err = std::string("solve_multi: ") + cudaGetErrorString(e);
    return CDG_ECUDA;
  }
  if (tc_err) {
    h->err = "solve_multi: a tensor-core wait reached its iteration limit";
    return CDG_ETIMEOUT;
  }
  if (status == CDG_ENOCONV) h->err = "maximum number of iterations reached";
  return status;
}

// y = A_0 x for the R columns of a multi-right-hand-side handle (tree order,
// [n][n_p][R] FP64, device), by the method its solves use; synchronous.
int dev_apply_multi(cdg_handle* h, const double* x, double* y, void* stream) {
  if (!h->dev || !h->dev->mr) {
    h->err = "cdg_apply_multi needs a handle created with nrhs > 0 and bound to a device buffer";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  MR& M = *D.mr;
  cudaStream_t s = (cudaStream_t)stream;
  if (M.oz) cudaMemsetAsync(M.tc_err, 0, sizeof(int), s);
  if (!mr_apply64(D, M, x, y, s)) {
    h->err = "unsupported n_p for cdg_apply_multi";
    return CDG_EINVAL;
  }
  int err = 0;
  if (M.oz) cudaMemcpyAsync(&err, M.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->err = std::string("cdg_apply_multi: ") + cudaGetErrorString(e);
    return CDG_ECUDA;
  }
  if (err) {
    h->err = "cdg_apply_multi: a tensor-core wait reached its iteration limit";
    return CDG_ETIMEOUT;
  }
  return CDG_OK;
}
