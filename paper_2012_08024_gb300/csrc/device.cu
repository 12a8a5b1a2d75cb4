// Device side of the solve phase: block-sparse CDG operator apply, damped
// block-Jacobi smoothing, restriction / prolongation between agglomerates and
// their children, the dense coarsest solve, the V-cycle (R14) and the outer CG
// (R15).  All device memory is carved from one caller-provided buffer.
//
// Layout in HBM (tree order: children of every agglomerate contiguous):
//   A_l      BSR, int32 rowptr/col, n_p x n_p row-major blocks, FP64 (+FP32 copy)
//   Dinv_l   [n_l][n_p][n_p] inverses of the diagonal blocks of A_l
//   L_l      [n_l][n_p][n_p] prolongation blocks to level l from its parent
//   vectors  [n_l][n_p] element-major
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device_kernels.cuh"
#include "device_state.h"

#include <atomic>
#include <mutex>

static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }

namespace {
using cdgk::cvt;
using cdgk::ldg;
using cdgk::row_acc;
using cdgk::VecLoad;

// ------------------------------------------------------------------ layout
struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Cuts the agglomerates of a level into consecutive chunks for the fused
// residual + restriction: chunks close at an agglomerate boundary once they
// hold about `target` fine rows (an agglomerate larger than that is a chunk of
// its own).  Returns the parent boundaries; rows / parents: largest chunk.
std::vector<int> agglomerate_chunks(const std::vector<cdg::i32>& cp, int target, int* rows, int* parents) {
  std::vector<int> out{0};
  *rows = *parents = 0;
  const int nc = (int)cp.size() - 1;
  int start = 0;
  for (int P = 0; P < nc; ++P) {
    const int before = cp[P] - cp[start];
    if (P > start && before + (cp[P + 1] - cp[P]) > target) {
      out.push_back(P);
      *rows = std::max(*rows, before);
      *parents = std::max(*parents, P - start);
      start = P;
    }
  }
  if (nc > start) {
    out.push_back(nc);
    *rows = std::max(*rows, (int)(cp[nc] - cp[start]));
    *parents = std::max(*parents, nc - start);
  }
  return out;
}

// fine rows per chunk of the fused restriction: four passes of a 256-thread CTA
inline int chunk_target(int np) { return 4 * (kThreads / 32) * (32 / np); }

size_t layout(const cdg::Hierarchy& H, int precision, int nrhs, DeviceState* S, char* base, int mr_precision,
              int gmres_m, int maxit, int tc_fp64) {
  Carver c{base};
  const int np = H.np;
  const int nlev = (int)H.lev.size();
  const int64_t ne = H.mesh.ne;
  const size_t vecbytes_elems = (size_t)ne * np;
  DeviceState tmp;
  DeviceState& D = S ? *S : tmp;
  D.nlev = nlev;
  D.np = np;
  D.d = H.mesh.d;
  D.nq = H.vrule.n();
  D.nfq = H.frule.n();
  D.ne = ne;
  D.ndofs = ne * np;
  D.nbf = (int64_t)H.mesh.bf_K.size();
  D.precision = precision;
  const size_t vsz = precision ? sizeof(float) : sizeof(double);
  D.nrhs = nrhs;
  for (int l = 0; l < nlev; ++l) {
    DevLevel& L = D.lev[l];
    const cdg::BSR& A = H.A_t[l];
    const int npl = H.np_l.empty() ? np : H.np_l[l];
    const size_t nb2l = (size_t)npl * npl;
    L.n = (int)A.nrows;
    L.np = npl;
    L.ptrans = l + 1 < nlev && H.L_t[l].empty();
    L.nnzb = A.nnzb();
    L.rowptr = c.take<int>(A.nrows + 1);
    L.col = c.take<int>(A.nnzb());
    const bool last = l + 1 == nlev;
    // FP64 operator: level 0 always (outer CG); all levels in FP64 mode
    if (l == 0 || precision == 0) L.A = c.take<double>(A.val.size());
    if (!last) {
      const cdg::BSR& Sh = H.Ahat_t[l];
      L.hnnzb = Sh.nnzb();
      L.hrowptr = c.take<int>(Sh.nrows + 1);
      L.hcol = c.take<int>(Sh.nnzb() + 1);
      // transfer blocks between agglomeration levels only (degree steps truncate)
      const size_t nL = H.L_t[l].size();
      if (precision == 0) {
        L.Dinv = c.take<double>((size_t)L.n * nb2l);
        if (nL) L.L = c.take<double>(nL);
        L.Ahat = c.take<double>(Sh.val.size() + 1);
      } else {
        L.A32 = c.take<float>(A.val.size());
        L.Dinv32 = c.take<float>((size_t)L.n * nb2l);
        if (nL) L.L32 = c.take<float>(nL);
        L.Ahat32 = c.take<float>(Sh.val.size() + 1);
      }
      L.parent = c.take<int>(L.n);
      if (!L.ptrans && l + 1 < nlev) {
        int rows = 0, parents = 0;
        const std::vector<int> ch = agglomerate_chunks(H.childptr_t[l + 1], chunk_target(npl), &rows, &parents);
        L.nchunk = (int)ch.size() - 1;
        L.chunk_rows = rows;
        L.chunk_parents = parents;
        L.chunk = c.take<int>(ch.size());
      }
    }
    if (l > 0) L.childptr = c.take<int>(L.n + 1);
    const size_t nv = (size_t)L.n * npl;
    L.x = c.take<char>(nv * vsz);
    L.t = c.take<char>(nv * vsz);
    L.r = c.take<char>(nv * vsz);
    L.b = c.take<char>(nv * vsz);
    L.bh = c.take<char>(nv * (l == 0 ? sizeof(double) : vsz));
  }
  D.nc = (int)(H.lev.back().n * D.lev[nlev - 1].np);
  D.nseg = (int)H.seg_rows[0].size() - 1;
  D.bps = D.nseg == 1 ? kDotBlocks1 : std::max(1, kDotBlocks / D.nseg);
  D.seg_dof = c.take<long long>(D.nseg + 1);
  D.crow_seg = c.take<int>(D.nc);
  D.crow_off = c.take<int>(D.nseg + 1);
  D.cinv_off = c.take<long long>(D.nseg + 1);
  D.coarse_inv = c.take<double>(H.coarse_inv.size());
  D.coarse_b = c.take<double>(D.nc);
  D.coarse_x = c.take<double>(D.nc);
  D.rhs_vol = c.take<double>(H.rhs_vol.size());
  D.rhs_bptr = c.take<int>(H.rhs_bptr.size());
  D.rhs_bface = c.take<int>(H.rhs_bface.size() + 1);
  D.rhs_bdata = c.take<double>(H.rhs_bD.size() + 1);
  D.btag = c.take<int>(D.nbf + 1);
  D.perm0 = c.take<int>(ne);
  D.dk_own = c.take<double>(H.dk_own.size() + 1);
  D.dk_ptr = c.take<int>(H.dk_ptr.size());
  D.dk_nbr = c.take<int>(H.dk_nbr.size() + 1);
  D.dk_blk = c.take<double>(H.dk_blk.size() + 1);
  D.kappa = c.take<double>(H.kappa_w.size());
  D.x = c.take<double>(vecbytes_elems);
  D.r = c.take<double>(vecbytes_elems);
  D.z = c.take<double>(vecbytes_elems);
  D.p = c.take<double>(vecbytes_elems);
  D.q = c.take<double>(vecbytes_elems);
  D.bt = c.take<double>(vecbytes_elems);
  D.zold = c.take<double>(vecbytes_elems);
  if (precision) {
    D.r32 = c.take<float>(vecbytes_elems);
    D.z32 = c.take<float>(vecbytes_elems);
  }
  D.f_stage = c.take<double>((size_t)ne * D.nq);
  D.gD_stage = c.take<double>((size_t)D.nbf * D.nfq + 1);
  D.gN_stage = c.take<double>((size_t)D.nbf * D.nfq + 1);
  D.u_stage = c.take<double>(vecbytes_elems);
  D.scal = c.take<double>((size_t)S_COUNT * D.nseg);
  D.pv_count = c.take<unsigned>(2);
  D.pv_err = c.take<int>(1);
  D.it_dev = c.take<int>(1);
  D.iters_dev = c.take<int>(D.nseg);
  D.hist_dev = c.take<double>((size_t)D.nseg * (maxit + 1));
  D.npartial = std::max<int>(std::max(kDotBlocks, D.nseg * D.bps), (int)((int64_t)ne * np / 64 + 2));
  D.partial = c.take<double>((size_t)D.npartial * 2);
  if (gmres_m > 0) {
    D.gm_m = gmres_m;
    D.gm_ld = (vecbytes_elems + 31) & ~size_t(31);   // every basis vector starts 256-byte aligned
    D.gm_V = c.take<double>((size_t)(gmres_m + 1) * D.gm_ld);
    D.gm_Z = c.take<double>((size_t)gmres_m * D.gm_ld);
    D.gm_part = c.take<double>((size_t)(gmres_m + 2) * kGmBlocks);
    D.gm_st = c.take<double>((size_t)GmLayout{gmres_m}.size());
  }
  if (nrhs > 0) {
    if (S && !S->mr) S->mr = mr_new();
    c.off = mr_layout(H, nrhs, mr_precision, tc_fp64, S ? S->mr : nullptr, base, c.off);
  }
  return (c.off + 255) & ~size_t(255);
}

// ------------------------------------------------------------------ kernels
// One thread per scalar row: lane = sub * NP + i handles row i of block row
// warp * (32 / NP) + sub.  MODE 0: y = A x, 1: y = b - A x,
// 3: y = x + omega (bh - x - Ahat x) with Ahat = D^{-1}(A - D) and bh = D^{-1} b,
// i.e. one damped block-Jacobi step.  With dot != nullptr, MODE 0 also writes
// the block partial of sum_i x_i y_i (for p^T A p).
// VEC kernels keep UNR blocks of the row in flight per step (UNR is chosen per
// level and mode by the autotuner at bind time; the summation order, block by
// block and column by column, is the same for every UNR).  The register budget
// grows with UNR (8 / UNR resident blocks of 256 threads per SM: 32, 64 or 128
// registers), so the variants trade occupancy for loads in flight.
template <typename T, int NP, int MODE, bool VEC, int UNR = 1>
__global__ void __launch_bounds__(kThreads, 8 / UNR) bsr_kernel(int n, const int* __restrict__ rowptr,
                                                       const int* __restrict__ col, const T* __restrict__ A,
                                                       const T* __restrict__ Dinv, const T* __restrict__ x,
                                                       const T* __restrict__ b, T* __restrict__ y, T omega,
                                                       double* __restrict__ dot) {
  constexpr int RPW = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int sub = lane / NP;
  const int i = lane - sub * NP;
  const int K = warp * RPW + sub;
  const bool active = (sub < RPW) && (K < n);
  const T acc = active ? row_acc<T, NP, VEC, UNR>(K, i, rowptr, col, A, x) : T(0);
  const size_t row = (size_t)K * NP + i;
  if (MODE == 0) {
    if (active) y[row] = acc;
    if (dot) {
      double v = active ? (double)x[row] * (double)acc : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      __shared__ double red[kThreads / 32];
      if (lane == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        dot[blockIdx.x] = s;
      }
    }
  } else if (active) {
    if (MODE == 1) y[row] = b[row] - acc;
    else y[row] = x[row] + omega * (b[row] - x[row] - acc);
  }
}


// Residual + restriction (Section 3.4), fused, with the first smoothing step of
// the coarse level.  The grid is cut into chunks of whole agglomerates: CTA c
// owns the parents [cpar[c], cpar[c+1]) of level l+1, whose children are the
// contiguous fine rows [ccp[cpar[c]], ccp[cpar[c+1]]).
//  1. every fine row of the chunk: r_K = b_K - A_K x (RESID; else r_K = b_K,
//     the residual of a zero guess), then its contribution L_K^T r_K, kept in
//     shared memory (the n_p lanes of a block row exchange r_K by shuffles);
//  2. every parent: b_{l+1}[A] = sum of its children's contributions, in child
//     order, written to bc;
//  3. SMOOTH >= 1: bh_{l+1}[A] = D_A^{-1} b_{l+1}[A], and SMOOTH = 2 also
//     x_{l+1}[A] = omega bh (the first damped block-Jacobi step from zero).
// The residual r is never written.  Dynamic shared memory: (rows + parents) of
// the largest chunk x NP values.
template <typename T, int NP, bool VEC, int UNR, bool RESID, int SMOOTH>
__global__ void __launch_bounds__(kThreads, 8 / (UNR < 2 ? 2 : UNR)) restrict_fused_kernel(
    const int* __restrict__ cpar, const int* __restrict__ ccp, const int* __restrict__ rowptr,
    const int* __restrict__ col, const T* __restrict__ A, const T* __restrict__ x, const T* __restrict__ b,
    const T* __restrict__ L, T* __restrict__ bc, const T* __restrict__ Dinv_c, T* __restrict__ bh_c,
    T* __restrict__ x_c, T omega, int max_rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_c = reinterpret_cast<T*>(smem_raw);
  T* s_b = s_c + (size_t)max_rows * NP;
  constexpr int RPW = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NP;
  const int i = lane - sub * NP;
  const int rpp = (blockDim.x >> 5) * RPW;   // fine rows per pass of the CTA
  const int P0 = cpar[blockIdx.x], P1 = cpar[blockIdx.x + 1];
  const int r0 = ccp[P0], r1 = ccp[P1];
  for (int base = 0; base < r1 - r0; base += rpp) {   // the same trip count in every thread
    const int lr = base + (int)(threadIdx.x >> 5) * RPW + sub;
    const int K = r0 + lr;
    const bool active = sub < RPW && K < r1;
    T r = T(0);
    if (active) {
      r = b[(size_t)K * NP + i];
      if constexpr (RESID) r -= row_acc<T, NP, VEC, UNR>(K, i, rowptr, col, A, x);
    }
    const T* LK = L + (size_t)(active ? K : r0) * NP * NP + i;
    T c = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const T rj = __shfl_sync(0xffffffffu, r, sub * NP + j);
      if (active) c = fma(ldg(LK + j * NP), rj, c);
    }
    if (active) s_c[(size_t)lr * NP + i] = c;
  }
  __syncthreads();
  const int np_ = (P1 - P0) * NP;
  for (int t = threadIdx.x; t < np_; t += blockDim.x) {
    const int Pl = t / NP, ii = t - Pl * NP;
    const int P = P0 + Pl;
    T sum = T(0);
    for (int k = ccp[P] - r0; k < ccp[P + 1] - r0; ++k) sum += s_c[(size_t)k * NP + ii];
    bc[(size_t)P * NP + ii] = sum;
    if constexpr (SMOOTH > 0) s_b[t] = sum;
  }
  if constexpr (SMOOTH > 0) {
    __syncthreads();
    for (int t = threadIdx.x; t < np_; t += blockDim.x) {
      const int Pl = t / NP, ii = t - Pl * NP;
      const int P = P0 + Pl;
      const T* D = Dinv_c + (size_t)P * NP * NP + ii * NP;
      T sum = T(0);
#pragma unroll
      for (int j = 0; j < NP; ++j) sum = fma(ldg(D + j), s_b[Pl * NP + j], sum);
      bh_c[(size_t)P * NP + ii] = sum;
      if constexpr (SMOOTH == 2) x_c[(size_t)P * NP + ii] = omega * sum;
    }
  }
}

// The last post-smoothing sweep of level l+1 fused with the prolongation to
// level l (Section 3.4): y_A = x_A + omega (bh_A - x_A - (Ahat x)_A), then for
// every child K of A: xf_K (+)= L_K y_A (ADD: the correction of a fine iterate;
// else the fine iterate itself, after a zero pre-smoothing).  The warp's y_A
// go to shared memory; the children of its coarse rows are one contiguous fine
// range, whose (child, row) outputs the 32 lanes share evenly (coalesced L_K
// rows and x_K, independent of how many children each agglomerate has).
template <typename T, int NP, bool VEC, int UNR, bool ADD>
__global__ void __launch_bounds__(kThreads, 8 / (UNR < 2 ? 2 : UNR)) smooth_prolong_kernel(
    int n, const int* __restrict__ rowptr, const int* __restrict__ col, const T* __restrict__ Ahat,
    const T* __restrict__ x, const T* __restrict__ bh, T* __restrict__ y, T omega, const int* __restrict__ childptr,
    const int* __restrict__ parent_f, const T* __restrict__ Lf, T* __restrict__ xf) {
  constexpr int RPW = 32 / NP;
  __shared__ T s_y[kThreads / 32][RPW * NP];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int sub = lane / NP;
  const int i = lane - sub * NP;
  const int A0 = warp * RPW;
  const int Ag = A0 + sub;
  const bool active = (sub < RPW) && (Ag < n);
  if (active) {
    const size_t row = (size_t)Ag * NP + i;
    const T acc = row_acc<T, NP, VEC, UNR>(Ag, i, rowptr, col, Ahat, x);
    const T xv = x[row];
    const T yv = xv + omega * (bh[row] - xv - acc);
    y[row] = yv;
    s_y[wib][sub * NP + i] = yv;
  }
  __syncwarp();
  if (A0 >= n) return;
  const int A1 = min(A0 + RPW, n);
  const int k0 = childptr[A0];
  const int tot = (childptr[A1] - k0) * NP;
#pragma unroll 2
  for (int o = lane; o < tot; o += 32) {
    const int K = k0 + o / NP;
    const int ii = o - (K - k0) * NP;
    const T* ya = &s_y[wib][(parent_f[K] - A0) * NP];
    const T* LK = Lf + (size_t)K * NP * NP + ii * NP;
    T sum = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) sum = fma(ldg(LK + j), ya[j], sum);
    const size_t row = (size_t)K * NP + ii;
    xf[row] = ADD ? xf[row] + sum : sum;
  }
}

// bh = Dinv b; with WRITE_X also x = omega bh (first smoothing step from a zero guess)
template <typename T, int NP, bool WRITE_X>
__global__ void __launch_bounds__(kThreads) smooth_first_kernel(int n, const T* __restrict__ Dinv,
                                                                const T* __restrict__ b, T* __restrict__ bh,
                                                                T* __restrict__ x, T omega) {
  constexpr int RPW = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int sub = lane / NP;
  const int i = lane - sub * NP;
  const int K = warp * RPW + sub;
  if (sub >= RPW || K >= n) return;
  const T* D = Dinv + (size_t)K * NP * NP + i * NP;
  const T* bk = b + (size_t)K * NP;
  T s = T(0);
#pragma unroll
  for (int j = 0; j < NP; ++j) s = fma(ldg(D + j), ldg(bk + j), s);
  bh[(size_t)K * NP + i] = s;
  if (WRITE_X) x[(size_t)K * NP + i] = omega * s;
}

// bc[A] = sum over children K of L_K^T r[K]
template <typename T, int NP>
__global__ void __launch_bounds__(kThreads) restrict_kernel(int nc, const int* __restrict__ childptr,
                                                            const T* __restrict__ L, const T* __restrict__ r,
                                                            T* __restrict__ bc) {
  constexpr int RPW = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int sub = lane / NP;
  const int i = lane - sub * NP;
  const int Ag = warp * RPW + sub;
  if (sub >= RPW || Ag >= nc) return;
  T s = T(0);
  for (int K = childptr[Ag]; K < childptr[Ag + 1]; ++K) {
    const T* LK = L + (size_t)K * NP * NP + i;
    const T* rk = r + (size_t)K * NP;
#pragma unroll
    for (int j = 0; j < NP; ++j) s = fma(ldg(LK + j * NP), ldg(rk + j), s);
  }
  bc[(size_t)Ag * NP + i] = s;
}

// x[K] (+)= L_K xc[parent K]
template <typename T, int NP, bool ADD>
__global__ void __launch_bounds__(kThreads) prolong_kernel(int n, const int* __restrict__ parent,
                                                           const T* __restrict__ L, const T* __restrict__ xc,
                                                           T* __restrict__ x) {
  constexpr int RPW = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int sub = lane / NP;
  const int i = lane - sub * NP;
  const int K = warp * RPW + sub;
  if (sub >= RPW || K >= n) return;
  const T* LK = L + (size_t)K * NP * NP + i * NP;
  const T* xa = xc + (size_t)parent[K] * NP;
  T s = T(0);
#pragma unroll
  for (int j = 0; j < NP; ++j) s = fma(ldg(LK + j), ldg(xa + j), s);
  const size_t row = (size_t)K * NP + i;
  x[row] = ADD ? x[row] + s : s;
}

// coarsest solve: x = Ainv_m b (ADD: x += Ainv_m b) on every segment m, one
// warp per row; each segment has its own dense inverse (row-major, n_m x n_m),
// FP64 accumulation
template <typename TI, typename TO, bool ADD = false>
__global__ void coarse_kernel(int nc, const int* __restrict__ crow_seg, const int* __restrict__ crow_off,
                              const long long* __restrict__ cinv_off, const double* __restrict__ Ainv,
                              const TI* __restrict__ b, TO* __restrict__ x) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nc) return;
  const int m = crow_seg[row];
  const int r0 = crow_off[m], nm = crow_off[m + 1] - r0;
  const double* a = Ainv + cinv_off[m] + (size_t)(row - r0) * nm;
  const TI* bm = b + r0;
  double s = 0.0;
  for (int j = lane; j < nm; j += 32) s = fma(a[j], cvt<double>(bm[j]), s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = ADD ? cvt<TO>(cvt<double>(x[row]) + s) : cvt<TO>(s);
}

// Between two degrees of the p-multigrid levels (Section 4.4) the orthonormal
// bases are nested: the degree q-1 basis is the first npc functions of the
// degree q basis on the same element, so restriction keeps the first npc
// coefficients of every element and prolongation adds them back (ADD) or
// writes them with zero higher coefficients.
template <typename T>
__global__ void __launch_bounds__(kThreads) ptrunc_restrict_kernel(int n, int npf, int npc,
                                                                   const T* __restrict__ r, T* __restrict__ bc) {
  const size_t tot = (size_t)n * npc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const size_t K = t / npc;
    bc[t] = r[K * npf + (t - K * npc)];
  }
}

template <typename T, bool ADD>
__global__ void __launch_bounds__(kThreads) ptrunc_prolong_kernel(int n, int npf, int npc,
                                                                  const T* __restrict__ xc, T* __restrict__ x) {
  const size_t tot = (size_t)n * npf;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const size_t K = t / npf;
    const int i = (int)(t - K * npf);
    const T v = i < npc ? xc[K * npc + i] : T(0);
    x[t] = ADD ? x[t] + v : v;
  }
}

template <typename TI, typename TO>
__global__ void convert_kernel(size_t n, const TI* __restrict__ a, TO* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = cvt<TO>(a[i]);
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

// Segmented vector kernels: block seg * bps + c handles chunk c of segment
// seg (the level-0 dofs of one mesh), so every block has one set of scalars.
__device__ __forceinline__ void seg_range(const long long* __restrict__ seg_dof, int bps, int& seg, size_t& lo,
                                          size_t& hi) {
  seg = blockIdx.x / bps;
  const int c = blockIdx.x - seg * bps;
  const size_t a = (size_t)seg_dof[seg], len = (size_t)seg_dof[seg + 1] - a;
  lo = a + len * c / bps;
  hi = a + len * (c + 1) / bps;
}

// partial[blk] = sum x.y over the block's chunk (and partial[npart + blk] = sum x.w)
__global__ void __launch_bounds__(kThreads) dot_kernel(const long long* __restrict__ seg_dof, int bps,
                                                       const double* __restrict__ x, const double* __restrict__ y,
                                                       const double* __restrict__ w, double* __restrict__ partial,
                                                       int npart) {
  int seg;
  size_t lo, hi;
  seg_range(seg_dof, bps, seg, lo, hi);
  // four elements' loads in flight per step; the sums run over the thread's
  // elements in ascending order (the rounding does not depend on the unrolling)
  double s = 0.0, s2 = 0.0;
  const size_t bd = blockDim.x;
  size_t i = lo + threadIdx.x;
  for (; i + 3 * bd < hi; i += 4 * bd) {
    double xv[4], yv[4], wv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      xv[u] = x[i + u * bd];
      yv[u] = y[i + u * bd];
      wv[u] = w ? w[i + u * bd] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      s = fma(xv[u], yv[u], s);
      if (w) s2 = fma(xv[u], wv[u], s2);
    }
  }
  for (; i < hi; i += bd) {
    s = fma(x[i], y[i], s);
    if (w) s2 = fma(x[i], w[i], s2);
  }
  s = block_sum(s);
  if (w) s2 = block_sum(s2);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    if (w) partial[npart + blockIdx.x] = s2;
  }
}

// One block per segment: sums its cnt partials in a fixed order and updates the
// segment's CG scalars.  which: 0 PQ (alpha; breakdown if p.Ap <= 0), 1 RR
// (iteration count, convergence ||r|| <= tol ||b||), 2 RZ (beta: Fletcher-Reeves,
// or Polak-Ribiere with the second partial (r_new, z_old) when flexible),
// 3 BB, 4 initial RR.  A segment marked done gets alpha = beta = 0.
__global__ void finalize_kernel(const double* __restrict__ partial, int cnt, int npart, int which, int flexible,
                                double tol, double* __restrict__ scal) {
  __shared__ double red[kThreads / 32];
  const int m = blockIdx.x;
  const double* pm = partial + (size_t)m * cnt;
  double s = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    s += pm[i];
    if (which == 2 && flexible) s2 += partial[npart + (size_t)m * cnt + i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) tot += red[w];
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot2 = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) tot2 += red[w];
    double* sc = scal + (size_t)m * S_COUNT;
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
}

// x += alpha p; r -= alpha q; partial of r.r (per segment chunk)
__global__ void __launch_bounds__(kThreads) cg_update_kernel(const long long* __restrict__ seg_dof, int bps,
                                                             const double* __restrict__ scal,
                                                             const double* __restrict__ p,
                                                             const double* __restrict__ q, double* __restrict__ x,
                                                             double* __restrict__ r, double* __restrict__ partial) {
  int seg;
  size_t lo, hi;
  seg_range(seg_dof, bps, seg, lo, hi);
  const double alpha = scal[(size_t)seg * S_COUNT + S_ALPHA];
  double s = 0.0;
  const size_t bd = blockDim.x;
  size_t i = lo + threadIdx.x;
  for (; i + 3 * bd < hi; i += 4 * bd) {   // four elements' loads in flight, ascending sum
    double pv[4], qv[4], xv[4], rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pv[u] = p[i + u * bd];
      qv[u] = q[i + u * bd];
      xv[u] = x[i + u * bd];
      rv[u] = r[i + u * bd];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[i + u * bd] = fma(alpha, pv[u], xv[u]);
      const double ri = fma(-alpha, qv[u], rv[u]);
      r[i + u * bd] = ri;
      s = fma(ri, ri, s);
    }
  }
  for (; i < hi; i += bd) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Single-graph solve: mark the segments converged before the loop as closed
__global__ void hist_init_kernel(int nseg, double* __restrict__ scal) {
  for (int m = threadIdx.x; m < nseg; m += blockDim.x) scal[(size_t)m * S_COUNT + S_HDONE] = scal[(size_t)m * S_COUNT + S_DONE];
}

// Single-graph solve, after G1 of iteration it: record ||r||/||b|| and the iteration count of every
// segment still open (a segment closes in the iteration it converges or breaks down), and keep the
// loop running while a segment is open and it < maxit.
__global__ void cg_check_kernel(cudaGraphConditionalHandle cond, int nseg, int maxit, double* __restrict__ scal,
                                int* __restrict__ it_dev, double* __restrict__ hist, int* __restrict__ iters,
                                const int* __restrict__ wait_err) {
  __shared__ int open;
  if (threadIdx.x == 0) open = 0;
  __syncthreads();
  const int it = *it_dev + 1;
  for (int m = threadIdx.x; m < nseg; m += blockDim.x) {
    double* sc = scal + (size_t)m * S_COUNT;
    if (sc[S_HDONE] != 0.0) continue;
    hist[(size_t)m * (maxit + 1) + it] = sc[S_BB] > 0.0 ? sqrt(sc[S_RR] / sc[S_BB]) : 0.0;
    iters[m] = it;
    if (sc[S_DONE] != 0.0) sc[S_HDONE] = 1.0;
    else atomicOr(&open, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *it_dev = it;
    // a device wait that expired (persistent V-cycle) ends the loop: its output is not a V-cycle
    cudaGraphSetConditional(cond, (open != 0 && it < maxit && *wait_err == 0) ? 1u : 0u);
  }
}

// p = z + beta p (first: p = z)
__global__ void __launch_bounds__(kThreads) cg_p_kernel(const long long* __restrict__ seg_dof, int bps,
                                                        const double* __restrict__ scal, int first,
                                                        const double* __restrict__ z, double* __restrict__ p) {
  int seg;
  size_t lo, hi;
  seg_range(seg_dof, bps, seg, lo, hi);
  const double beta = first ? 0.0 : scal[(size_t)seg * S_COUNT + S_BETA];
  const size_t bd = blockDim.x;
  size_t i = lo + threadIdx.x;
  for (; i + 3 * bd < hi; i += 4 * bd) {
    double zv[4], pv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      zv[u] = z[i + u * bd];
      pv[u] = first ? 0.0 : p[i + u * bd];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) p[i + u * bd] = first ? zv[u] : fma(beta, pv[u], zv[u]);
  }
  for (; i < hi; i += bd) p[i] = first ? z[i] : fma(beta, p[i], z[i]);
}

// b (tree order, or user order) from f at volume points and g_D / g_N at boundary points
template <int NP>
__global__ void __launch_bounds__(kThreads) rhs_kernel(int ne, int nq, int nfq, const int* __restrict__ perm0,
                                                       const double* __restrict__ V, const double* __restrict__ f,
                                                       const int* __restrict__ bptr, const int* __restrict__ bface,
                                                       const double* __restrict__ bdata, const int* __restrict__ btag,
                                                       const double* __restrict__ gD, const double* __restrict__ gN,
                                                       double* __restrict__ b, int user_out) {
  constexpr int RPW = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int sub = lane / NP;
  const int i = lane - sub * NP;
  const int k = warp * RPW + sub;
  if (sub >= RPW || k >= ne) return;
  const int K = perm0[k];
  double s = 0.0;
  const double* Vk = V + (size_t)k * nq * NP + i;
  const double* fk = f + (size_t)K * nq;
  for (int q = 0; q < nq; ++q) s = fma(Vk[(size_t)q * NP], fk[q], s);
  for (int t = bptr[k]; t < bptr[k + 1]; ++t) {
    const int bf = bface[t];
    const double* g = btag[bf] == 0 ? gD : gN;
    if (!g) continue;
    const double* Bd = bdata + (size_t)bf * nfq * NP + i;
    for (int q = 0; q < nfq; ++q) s = fma(Bd[(size_t)q * NP], g[(size_t)bf * nfq + q], s);
  }
  b[(size_t)(user_out ? K : k) * NP + i] = s;
}

__global__ void permute_kernel(int ne, int np, const int* __restrict__ perm0, const double* __restrict__ in,
                               double* __restrict__ out, int to_tree) {
  const size_t n = (size_t)ne * np;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t / np, i = t - k * np;
    const size_t K = perm0[k];
    if (to_tree) out[k * np + i] = in[K * np + i];
    else out[K * np + i] = in[k * np + i];
  }
}


// dL/dkappa_K = lambda^T (db/dkappa_K - dA/dkappa_K u): A_0 and b are linear in
// kappa (every term is owned by one element, R7), so dA/dkappa_K is the
// unit-kappa sum of K's own pieces.  Thread (sub, i) of the usual row mapping
// accumulates row i of every piece; the NP lanes of an element then reduce.
template <int NP>
__global__ void __launch_bounds__(kThreads) kappa_grad_kernel(
    int ne, int nfq, const int* __restrict__ perm0, const double* __restrict__ own, const int* __restrict__ ptr,
    const int* __restrict__ nbr, const double* __restrict__ blk, const double* __restrict__ kappa,
    const double* __restrict__ lam, const double* __restrict__ u, const int* __restrict__ bptr,
    const int* __restrict__ bface, const double* __restrict__ bdata, const int* __restrict__ btag,
    const double* __restrict__ gD, double* __restrict__ out) {
  constexpr int RPW = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int sub = lane / NP;
  const int i = lane - sub * NP;
  const int k = warp * RPW + sub;
  const bool active = (sub < RPW) && (k < ne);
  double t = 0.0;
  if (active) {
    const double* uk = u + (size_t)k * NP;
    const double lk = lam[(size_t)k * NP + i];
    const double* O = own + (size_t)k * NP * NP + i * NP;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) s = fma(O[j], uk[j], s);
    t = -lk * s;
    for (int f = ptr[k]; f < ptr[k + 1]; ++f) {
      const int J = nbr[f];
      const double* uJ = u + (size_t)J * NP;
      const double lJ = lam[(size_t)J * NP + i];
      const double* B = blk + (size_t)f * 3 * NP * NP + i * NP;
      double s_kj = 0.0, s_jk = 0.0, s_jj = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        s_kj = fma(B[j], uJ[j], s_kj);
        s_jk = fma(B[NP * NP + j], uk[j], s_jk);
        s_jj = fma(B[2 * NP * NP + j], uJ[j], s_jj);
      }
      t -= lk * s_kj + lJ * (s_jk + s_jj);
    }
    if (gD) {
      const double ik = 1.0 / kappa[k];
      for (int b = bptr[k]; b < bptr[k + 1]; ++b) {
        const int bf = bface[b];
        if (btag[bf] != 0) continue;
        const double* Bd = bdata + (size_t)bf * nfq * NP + i;
        double s2 = 0.0;
        for (int q = 0; q < nfq; ++q) s2 = fma(Bd[(size_t)q * NP], gD[(size_t)bf * nfq + q], s2);
        t += lk * s2 * ik;
      }
    }
  }
  double g = 0.0;
#pragma unroll
  for (int j = 0; j < NP; ++j) g += __shfl_sync(0xffffffffu, t, sub * NP + j);
  if (active && i == 0) out[perm0[k]] = g;
}

// dL/df_q = (db/df)^T lambda: out[K][q] = sum_i w_q phi_i(x_q) lambda_K[i] (user order)
template <int NP>
__global__ void rhs_adjoint_kernel(int ne, int nq, const int* __restrict__ perm0, const double* __restrict__ V,
                                   const double* __restrict__ lam, double* __restrict__ out) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)ne * nq) return;
  const size_t k = t / nq, q = t - k * nq;
  const double* Vq = V + (k * nq + q) * NP;
  const double* lk = lam + k * NP;
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < NP; ++i) s = fma(Vq[i], lk[i], s);
  out[(size_t)perm0[k] * nq + q] = s;
}

// FP64 FMA throughput probe: CHAINS independent dependency chains per thread,
// all operands in registers (m and c arrive as arguments), so the FP64 pipe,
// not the FMA latency, limits the rate.  The values depend on the runtime
// arguments (nothing folds at compile time); sink is written only if the
// chains end exactly at a value they cannot reach.
template <int CHAINS>
__global__ void __launch_bounds__(kThreads) fma64_probe_kernel(long long iters, double seed, double m, double c,
                                                             double* sink) {
  double a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = seed + 1e-3 * k + 1e-9 * threadIdx.x;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  if (s == -1.0) *sink = s;
}

// ------------------------------------------------------------------ launch helpers
// Every kernel launch of the library goes through here (counted for the
// benchmark's launch accounting).
template <typename... KArgs, typename... Args>
inline void launch(void (*k)(KArgs...), dim3 g, dim3 b, cudaStream_t s, Args... args) {
  k<<<g, b, 0, s>>>(args...);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

inline unsigned rows_grid(int64_t nrows, int np) {
  const int64_t rpw = 32 / np;
  const int64_t warps = (nrows + rpw - 1) / rpw;
  return (unsigned)std::max<int64_t>(1, (warps * 32 + kThreads - 1) / kThreads);
}

#define CDG_NP_DISPATCH(NPV, ...)                          \
  switch (NPV) {                                           \
    case 3: { constexpr int NP = 3; __VA_ARGS__; break; }  \
    case 4: { constexpr int NP = 4; __VA_ARGS__; break; }  \
    case 6: { constexpr int NP = 6; __VA_ARGS__; break; }  \
    case 10: { constexpr int NP = 10; __VA_ARGS__; break; } \
    case 15: { constexpr int NP = 15; __VA_ARGS__; break; } \
    case 20: { constexpr int NP = 20; __VA_ARGS__; break; } \
    case 21: { constexpr int NP = 21; __VA_ARGS__; break; } \
    case 28: { constexpr int NP = 28; __VA_ARGS__; break; } \
    default: return false;                                 \
  }

template <typename T, int NP, int MODE, int UNR>
void launch_vec(unsigned g, cudaStream_t s, int n, const int* rowptr, const int* col, const T* A, const T* x,
                const T* b, T* y, double omega, double* dot) {
  launch(bsr_kernel<T, NP, MODE, true, UNR>, g, kThreads, s, n, rowptr, col, A, (const T*)nullptr, x, b, y,
         (T)omega, MODE == 0 ? dot : (double*)nullptr);
}

template <typename T, int NP, int MODE>
void launch_vec_unr(int unr, unsigned g, cudaStream_t s, int n, const int* rowptr, const int* col, const T* A,
                    const T* x, const T* b, T* y, double omega, double* dot) {
  if (unr >= 4) launch_vec<T, NP, MODE, 4>(g, s, n, rowptr, col, A, x, b, y, omega, dot);
  else if (unr == 1) launch_vec<T, NP, MODE, 1>(g, s, n, rowptr, col, A, x, b, y, omega, dot);
  else launch_vec<T, NP, MODE, 2>(g, s, n, rowptr, col, A, x, b, y, omega, dot);
}

// mode 0: y = A x (+ dot partials), 1: y = b - A x, 3: y = x + omega (bh - x - Ahat x).
// unr: blocks in flight per step of the vector-load kernel (autotuned per level and mode).
template <typename T>
bool launch_bsr(int mode, int np, int n, const int* rowptr, const int* col, const T* A, const T* x, const T* b,
                T* y, double omega, double* dot, cudaStream_t s, double* flag = nullptr, int unr = 2) {
  const unsigned g = rows_grid(n, np);
  // flag != nullptr marks vectors known to be 16-byte aligned: even n_p then
  // takes the vector-load kernel
  if (flag && np % 2 == 0) {
    CDG_NP_DISPATCH(np, {
      if constexpr (NP % 2 == 0) {
        if (mode == 0) launch_vec_unr<T, NP, 0>(unr, g, s, n, rowptr, col, A, x, b, y, omega, dot);
        else if (mode == 1) launch_vec_unr<T, NP, 1>(unr, g, s, n, rowptr, col, A, x, b, y, omega, dot);
        else launch_vec_unr<T, NP, 3>(unr, g, s, n, rowptr, col, A, x, b, y, omega, dot);
      }
    });
    return true;
  }
  CDG_NP_DISPATCH(np, {
    if (mode == 0)
      launch(bsr_kernel<T, NP, 0, false>, g, kThreads, s, n, rowptr, col, A, (const T*)nullptr, x, b, y, (T)omega,
             dot);
    else if (mode == 1)
      launch(bsr_kernel<T, NP, 1, false>, g, kThreads, s, n, rowptr, col, A, (const T*)nullptr, x, b, y, (T)omega,
             (double*)nullptr);
    else
      launch(bsr_kernel<T, NP, 3, false>, g, kThreads, s, n, rowptr, col, A, (const T*)nullptr, x, b, y, (T)omega,
             (double*)nullptr);
  });
  return true;
}

template <typename T>
bool launch_smooth_first(int np, int n, const T* Dinv, const T* b, T* bh, T* x, double omega, cudaStream_t s) {
  CDG_NP_DISPATCH(np, {
    if (x) launch(smooth_first_kernel<T, NP, true>, rows_grid(n, np), kThreads, s, n, Dinv, b, bh, x, (T)omega);
    else launch(smooth_first_kernel<T, NP, false>, rows_grid(n, np), kThreads, s, n, Dinv, b, bh, x, (T)omega);
  });
  return true;
}

// 64-thread CTAs: a warp's loop runs to the largest child count among its
// agglomerates, and small CTAs spread that uneven work over the SMs more evenly
template <typename T>
bool launch_restrict(int np, int nc, const int* cp, const T* L, const T* r, T* bc, cudaStream_t s) {
  constexpr int kRT = 64;
  const int64_t warps = ((int64_t)nc + 32 / np - 1) / (32 / np);
  const unsigned g = (unsigned)std::max<int64_t>(1, (warps * 32 + kRT - 1) / kRT);
  CDG_NP_DISPATCH(np, launch(restrict_kernel<T, NP>, g, kRT, s, nc, cp, L, r, bc));
  return true;
}

template <typename T>
bool launch_prolong(int np, int n, const int* parent, const T* L, const T* xc, T* x, bool add, cudaStream_t s) {
  CDG_NP_DISPATCH(np, {
    if (add) launch(prolong_kernel<T, NP, true>, rows_grid(n, np), kThreads, s, n, parent, L, xc, x);
    else launch(prolong_kernel<T, NP, false>, rows_grid(n, np), kThreads, s, n, parent, L, xc, x);
  });
  return true;
}

unsigned vec_grid(size_t n) { return (unsigned)std::min<size_t>(kDotBlocks, (n + kThreads - 1) / kThreads + 1); }

// restriction / prolongation between levels l and l+1: transfer blocks between
// agglomeration levels, truncation between two degrees on the same elements
template <typename T>
bool transfer_restrict(const DeviceState& D, int l, const T* Lb, const T* r, T* bc, cudaStream_t s) {
  const DevLevel& F = D.lev[l];
  const DevLevel& C = D.lev[l + 1];
  if (F.ptrans) {
    launch(ptrunc_restrict_kernel<T>, vec_grid((size_t)C.n * C.np), kThreads, s, C.n, F.np, C.np, r, bc);
    return true;
  }
  return launch_restrict<T>(F.np, C.n, C.childptr, Lb, r, bc, s);
}

template <typename T>
bool transfer_prolong(const DeviceState& D, int l, const T* Lb, const T* xc, T* x, bool add, cudaStream_t s) {
  const DevLevel& F = D.lev[l];
  const DevLevel& C = D.lev[l + 1];
  if (F.ptrans) {
    if (add) launch(ptrunc_prolong_kernel<T, true>, vec_grid((size_t)F.n * F.np), kThreads, s, F.n, F.np, C.np, xc, x);
    else launch(ptrunc_prolong_kernel<T, false>, vec_grid((size_t)F.n * F.np), kThreads, s, F.n, F.np, C.np, xc, x);
    return true;
  }
  return launch_prolong<T>(F.np, F.n, F.parent, Lb, xc, x, add, s);
}

int cuda_fail(cdg_handle* h, cudaError_t e, const char* where) {
  h->err = std::string(where) + ": " + cudaGetErrorString(e);
  return CDG_ECUDA;
}

#define CDG_CHECK_LAUNCH(h, where)                        \
  do {                                                    \
    cudaError_t e_ = cudaGetLastError();                  \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

template <typename T>
const T* opA(const DevLevel& L);
template <>
const double* opA<double>(const DevLevel& L) { return L.A; }
template <>
const float* opA<float>(const DevLevel& L) { return L.A32; }
template <typename T>
const T* opD(const DevLevel& L);
template <>
const double* opD<double>(const DevLevel& L) { return L.Dinv; }
template <>
const float* opD<float>(const DevLevel& L) { return L.Dinv32; }
template <typename T>
const T* opH(const DevLevel& L);
template <>
const double* opH<double>(const DevLevel& L) { return L.Ahat; }
template <>
const float* opH<float>(const DevLevel& L) { return L.Ahat32; }
template <typename T>
const T* opL(const DevLevel& L);
template <>
const double* opL<double>(const DevLevel& L) { return L.L; }
template <>
const float* opL<float>(const DevLevel& L) { return L.L32; }

template <typename T>
int unr_of(const DevLevel& L, int mode) { return L.unr[sizeof(T) == 8 ? 0 : 1][mode]; }

// Fused residual + restriction from level l to l+1 (+ the coarse level's first
// smoothing step, smooth: 0 none, 1 bh only, 2 bh and x = omega bh); false when
// the level has no chunk table or needs more shared memory than a CTA has by
// default (then the caller takes the separate kernels).
template <typename T>
bool launch_restrict_fused(const DeviceState& D, int l, bool resid, int smooth, const T* x, const T* b, T* bc,
                           double omega, cudaStream_t s, double* flag) {
  const DevLevel& F = D.lev[l];
  const DevLevel& C = D.lev[l + 1];
  if (!F.chunk || F.nchunk < 1) return false;
  const size_t smem = (size_t)(F.chunk_rows + F.chunk_parents) * F.np * sizeof(T);
  if (smem > 48 * 1024) return false;
  const int unr = std::max(1, std::min(4, unr_of<T>(F, 1)));
  const T* A = opA<T>(F);
  const T* Lb = opL<T>(F);
  const T* Dc = smooth ? opD<T>(C) : nullptr;
  const bool vec = flag && F.np % 2 == 0;
  bool ok = true;
  auto go = [&](auto kern) {
    kern<<<(unsigned)F.nchunk, kThreads, smem, s>>>(F.chunk, C.childptr, F.rowptr, F.col, A, x, b, Lb, bc, Dc,
                                                   (T*)C.bh, (T*)C.x, (T)omega, F.chunk_rows);
    count_launch();
  };
  // RESID x SMOOTH variants; VEC with 1, 2 or 4 blocks in flight for even n_p
#define CDG_RF(NPV, VEC, UNR)                                                                                \
  {                                                                                                          \
    if (resid) {                                                                                             \
      if (smooth == 2) go(restrict_fused_kernel<T, NPV, VEC, UNR, true, 2>);                                 \
      else if (smooth == 1) go(restrict_fused_kernel<T, NPV, VEC, UNR, true, 1>);                            \
      else go(restrict_fused_kernel<T, NPV, VEC, UNR, true, 0>);                                             \
    } else {                                                                                                 \
      if (smooth == 2) go(restrict_fused_kernel<T, NPV, VEC, UNR, false, 2>);                                \
      else if (smooth == 1) go(restrict_fused_kernel<T, NPV, VEC, UNR, false, 1>);                           \
      else go(restrict_fused_kernel<T, NPV, VEC, UNR, false, 0>);                                            \
    }                                                                                                        \
  }
  auto dispatch = [&]() -> bool {
    CDG_NP_DISPATCH(F.np, {
      if constexpr (NP % 2 == 0) {
        if (vec) {
          if (unr >= 4) CDG_RF(NP, true, 4) else if (unr == 1) CDG_RF(NP, true, 1) else CDG_RF(NP, true, 2)
        } else CDG_RF(NP, false, 1)
      } else CDG_RF(NP, false, 1)
    });
    return true;
  };
#undef CDG_RF
  ok = dispatch();
  return ok;
}

// The last post-smoothing sweep of level c = l+1 fused with the prolongation to level l.
template <typename T>
bool launch_smooth_prolong(const DeviceState& D, int l, const T* x, const T* bh, T* y, double omega, bool add,
                           cudaStream_t s, double* flag) {
  const DevLevel& F = D.lev[l];
  const DevLevel& C = D.lev[l + 1];
  const unsigned g = rows_grid(C.n, C.np);
  const int unr = std::max(1, std::min(4, unr_of<T>(C, 3)));
  const bool vec = flag && C.np % 2 == 0;
  auto go = [&](auto kern) {
    kern<<<g, kThreads, 0, s>>>(C.n, C.hrowptr, C.hcol, opH<T>(C), x, bh, y, (T)omega, C.childptr, F.parent,
                                opL<T>(F), (T*)F.x);
    count_launch();
  };
#define CDG_SP(NPV, VEC, UNR)                                       \
  {                                                                 \
    if (add) go(smooth_prolong_kernel<T, NPV, VEC, UNR, true>);     \
    else go(smooth_prolong_kernel<T, NPV, VEC, UNR, false>);        \
  }
  auto dispatch = [&]() -> bool {
    CDG_NP_DISPATCH(C.np, {
      if constexpr (NP % 2 == 0) {
        if (vec) {
          if (unr >= 4) CDG_SP(NP, true, 4) else if (unr == 1) CDG_SP(NP, true, 1) else CDG_SP(NP, true, 2)
        } else CDG_SP(NP, false, 1)
      } else CDG_SP(NP, false, 1)
    });
    return true;
  };
#undef CDG_SP
  return dispatch();
}

// Direct solve on the coarsest level (Algorithm 3): x = A_n^{-1} b through the
// dense inverse.  With the FP64 operator on the device (FP64 V-cycle) one step
// of iterative refinement follows, x += A_n^{-1} (b - A_n x) with the residual
// from the block-sparse A_n: an explicit inverse times b is not backward
// stable, the refined solution is (Skeel 1980), so it agrees with a
// factorisation-based solve to cond(A_n) eps.  r is a coarsest-level work
// vector that aliases neither b nor x.
template <typename T>
void coarse_solve(DeviceState& D, const T* b, T* x, cudaStream_t s) {
  const unsigned g = (unsigned)((D.nc * 32 + 255) / 256);
  launch(coarse_kernel<T, T, false>, g, 256, s, D.nc, D.crow_seg, D.crow_off, D.cinv_off, D.coarse_inv, b, x);
  if constexpr (sizeof(T) == sizeof(double)) {
    const DevLevel& C = D.lev[D.nlev - 1];
    if (!C.A || D.precision != 0) return;   // the work vectors of an FP32 V-cycle hold floats
    double* r = (double*)C.r;
    const bool aligned = (((uintptr_t)b | (uintptr_t)x) & 15) == 0;
    launch_bsr<double>(1, C.np, C.n, C.rowptr, C.col, C.A, x, b, r, 0.0, nullptr, s,
                       aligned ? D.scal + S_FLAG : nullptr, unr_of<double>(C, 1));
    launch(coarse_kernel<double, double, true>, g, 256, s, D.nc, D.crow_seg, D.crow_off, D.cinv_off, D.coarse_inv,
           (const double*)r, x);
  }
}

// One V(nu_pre, nu_post) cycle from a zero guess (R14) on levels 0..n, with
// b0 / z0 the level-0 right-hand side and result (precision T).  With
// fuse_transfers, between two agglomeration levels the residual, its
// restriction and the coarse level's first smoothing step are one kernel, and
// the coarse level's last post-smoothing sweep carries the prolongation; the
// separate kernels remain for degree steps of the p-multigrid front end, for
// the coarsest level and for V(nu, 0).
template <typename T>
bool vcycle(DeviceState& D, const cdg_options& o, const T* b0, T* z0, cudaStream_t s) {
  const int nlev = D.nlev;
  const double w = o.omega;
  double* flag = D.scal + S_FLAG;
  if (nlev == 1) {
    coarse_solve<T>(D, b0, z0, s);
    return true;
  }
  const bool fuse = (o.fuse_transfers & 1) != 0;        // residual + restriction + first coarse step
  const bool fuse_up = (o.fuse_transfers & 2) != 0;     // prolongation in the coarse level's last sweep
  std::vector<const T*> bl(nlev);
  bl[0] = b0;
  for (int l = 1; l < nlev; ++l) bl[l] = (const T*)D.lev[l].b;
  std::vector<char> first_done(nlev, 0);   // the level's first smoothing step came with its right-hand side
  // downward sweep
  for (int l = 0; l + 1 < nlev; ++l) {
    DevLevel& L = D.lev[l];
    const int np = L.np;
    T* x = (T*)L.x;
    T* t = (T*)L.t;
    const T* b = bl[l];
    T* bh = (T*)L.bh;
    const bool coarse_is_last = l + 2 == nlev;
    if (o.nu_pre >= 1) {
      if (!first_done[l] && !launch_smooth_first<T>(np, L.n, opD<T>(L), b, bh, x, w, s)) return false;
      for (int k = 1; k < o.nu_pre; ++k) {
        if (!launch_bsr<T>(3, np, L.n, L.hrowptr, L.hcol, opH<T>(L), x, bh, t, w, nullptr, s, flag,
                           unr_of<T>(L, 3)))
          return false;
        std::swap(x, t);
      }
      const int smooth = coarse_is_last ? 0 : 2;
      if (fuse && !L.ptrans &&
          launch_restrict_fused<T>(D, l, true, smooth, x, b, (T*)D.lev[l + 1].b, w, s, flag)) {
        first_done[l + 1] = smooth != 0;
      } else {
        if (!launch_bsr<T>(1, np, L.n, L.rowptr, L.col, opA<T>(L), x, b, (T*)L.r, w, nullptr, s, flag,
                           unr_of<T>(L, 1)))
          return false;
        if (!transfer_restrict<T>(D, l, opL<T>(L), (const T*)L.r, (T*)D.lev[l + 1].b, s)) return false;
      }
      // remember which buffer holds x
      L.x = x;
      L.t = t;
    } else {
      if (!first_done[l] && !launch_smooth_first<T>(np, L.n, opD<T>(L), b, bh, (T*)nullptr, w, s)) return false;
      const int smooth = coarse_is_last ? 0 : 1;
      if (fuse && !L.ptrans &&
          launch_restrict_fused<T>(D, l, false, smooth, (const T*)nullptr, b, (T*)D.lev[l + 1].b, w, s, flag)) {
        first_done[l + 1] = smooth != 0;
      } else if (!transfer_restrict<T>(D, l, opL<T>(L), b, (T*)D.lev[l + 1].b, s)) {
        return false;
      }
    }
  }
  // coarsest
  {
    const DevLevel& C = D.lev[nlev - 1];
    coarse_solve<T>(D, (const T*)C.b, (T*)C.x, s);
  }
  // upward sweep
  std::vector<char> prolonged(nlev, 0);   // the level's correction came with the coarser level's last sweep
  for (int l = nlev - 2; l >= 0; --l) {
    DevLevel& L = D.lev[l];
    const int np = L.np;
    T* x = (T*)L.x;
    T* t = (T*)L.t;
    if (!prolonged[l] &&
        !transfer_prolong<T>(D, l, opL<T>(L), (const T*)D.lev[l + 1].x, x, o.nu_pre >= 1, s))
      return false;
    // the last sweep of this level also prolongs into level l-1 (agglomeration step)
    const bool carry = fuse_up && l >= 1 && !D.lev[l - 1].ptrans && opL<T>(D.lev[l - 1]) != nullptr;
    for (int k = 0; k < o.nu_post; ++k) {
      T* out = (l == 0 && k + 1 == o.nu_post) ? z0 : t;
      if (carry && k + 1 == o.nu_post) {
        if (!launch_smooth_prolong<T>(D, l - 1, x, (const T*)L.bh, out, w, o.nu_pre >= 1, s, flag)) return false;
        prolonged[l - 1] = 1;
      } else if (!launch_bsr<T>(3, np, L.n, L.hrowptr, L.hcol, opH<T>(L), x, (const T*)L.bh, out, w, nullptr, s,
                                flag, unr_of<T>(L, 3))) {
        return false;
      }
      if (out == t) std::swap(x, t);
      else x = out;
    }
    if (l == 0 && o.nu_post == 0)
      cudaMemcpyAsync(z0, x, sizeof(T) * (size_t)L.n * np, cudaMemcpyDeviceToDevice, s);
    if (l > 0) {
      // the coarse solution of this level must sit in L.x for the next prolongation
      if (x != (T*)L.x) {
        L.t = L.x;
        L.x = x;
      }
    }
  }
  return true;
}

int precond(cdg_handle* h, const double* r, double* z, cudaStream_t s) {
  DeviceState& D = *h->dev;
  const size_t n = (size_t)D.ndofs;
  bool ok;
  const bool pv = h->opt.persistent_vcycle != 0 && !D.pv_failed;
  if (D.precision == 0) {
    ok = pv && vcycle_persistent(D, h->opt, false, r, z, D.pv_count, D.pv_err, s);
    if (!ok) {
      if (pv) cudaGetLastError();   // a refused cooperative launch: take the per-phase kernels
      D.pv_failed = D.pv_failed || pv;
      ok = vcycle<double>(D, h->opt, r, z, s);
    }
  } else {
    launch(convert_kernel<double, float>, vec_grid(n), kThreads, s, n, r, D.r32);
    ok = pv && vcycle_persistent(D, h->opt, true, D.r32, D.z32, D.pv_count, D.pv_err, s);
    if (!ok) {
      if (pv) cudaGetLastError();
      D.pv_failed = D.pv_failed || pv;
      ok = vcycle<float>(D, h->opt, D.r32, D.z32, s);
    }
    launch(convert_kernel<float, double>, vec_grid(n), kThreads, s, n, D.z32, z);
  }
  if (!ok) {
    h->err = "unsupported number of basis functions per element";
    return CDG_EINVAL;
  }
  CDG_CHECK_LAUNCH(h, "vcycle");
  return CDG_OK;
}

int dot_to(cdg_handle* h, const double* x, const double* y, const double* w, int which, cudaStream_t s) {
  DeviceState& D = *h->dev;
  const unsigned g = (unsigned)(D.nseg * D.bps);
  launch(dot_kernel, g, kThreads, s, (const long long*)D.seg_dof, D.bps, x, y, w, D.partial, D.npartial);
  launch(finalize_kernel, (unsigned)D.nseg, kThreads, s, (const double*)D.partial, D.bps, D.npartial, which,
         w != nullptr ? 1 : 0, h->opt.tol, D.scal);
  CDG_CHECK_LAUNCH(h, "dot");
  return CDG_OK;
}

template <typename T>
void upload(T* dst, const std::vector<T>& src, cudaStream_t s) {
  if (!src.empty()) cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s);
}

std::vector<float> to_f32(const std::vector<double>& v) {
  std::vector<float> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
  return o;
}

std::vector<int> to_i32(const std::vector<int64_t>& v) {
  std::vector<int> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (int)v[i];
  return o;
}

}  // namespace

// ------------------------------------------------------------------ entry points
long long dev_launch_count() { return g_launches.load(); }

int dev_precond(cdg_handle* h, const double* r, double* z, cudaStream_t s) { return precond(h, r, z, s); }

int dev_apply0(cdg_handle* h, int mode, const double* x, const double* b, double* y, cudaStream_t s) {
  DeviceState& D = *h->dev;
  const DevLevel& L0 = D.lev[0];
  if (!launch_bsr<double>(mode, D.np, L0.n, L0.rowptr, L0.col, L0.A, x, b, y, h->opt.omega, nullptr, s,
                          D.scal + S_FLAG, unr_of<double>(L0, mode))) {
    h->err = "unsupported number of basis functions per element";
    return CDG_EINVAL;
  }
  CDG_CHECK_LAUNCH(h, "level-0 operator");
  return CDG_OK;
}

int dev_dot(cdg_handle* h, const double* x, const double* y, int which, cudaStream_t s) {
  return dot_to(h, x, y, nullptr, which, s);
}

int dev_cuda_fail(cdg_handle* h, cudaError_t e, const char* where) { return cuda_fail(h, e, where); }

// ------------------------------------------------------------------ allocation-free smoother
// Fixed scratch for cdg_smooth_static: holds D^{-1} b of one level.  Every call
// in the process shares it; nothing has to start at zero (the first kernel
// overwrites all entries it later reads).
static __device__ __align__(256) double g_static_scratch[CDG_STATIC_SCRATCH];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {};
// the context each cached address belongs to: after cudaDeviceReset, or with
// another context current, the address is looked up again
void* g_static_ctx[kMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry-point query (no link
// dependency on the driver library); nullptr if the query fails
void* current_context() {
  using Fn = int (*)(void**);
  static Fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return (Fn)f;
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}
}  // namespace

int dev_smooth_static(cdg_handle* h, int level, const double* x, const double* b, double* y, void* stream) {
  if (!h) return CDG_EINVAL;
  if (!h->dev) {
    h->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  if (level < 0 || level + 1 >= D.nlev || !x || !b || !y || !D.lev[level].Ahat) {
    h->err = "cdg_smooth_static: bad level, NULL vector, or handle not in FP64 precision";
    return CDG_EINVAL;
  }
  const DevLevel& L = D.lev[level];
  if ((int64_t)L.n * L.np > (int64_t)CDG_STATIC_SCRATCH) {
    h->err = "cdg_smooth_static: level has " + std::to_string((int64_t)L.n * L.np) +
             " unknowns, more than the fixed scratch of " + std::to_string((int64_t)CDG_STATIC_SCRATCH);
    return CDG_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "cdg_smooth_static");
  if (dev < 0 || dev >= kMaxDevices) {
    h->err = "cdg_smooth_static: device index out of range";
    return CDG_EINVAL;
  }
  double* scratch = nullptr;
  {
    // once per device and context, with that device current: the symbol's device address
    std::lock_guard<std::mutex> lock(g_static_mutex);
    void* ctx = current_context();
    if (!g_static_ptr[dev] || ctx != g_static_ctx[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress");
      g_static_ptr[dev] = (double*)p;
      g_static_ctx[dev] = ctx;
    }
    scratch = g_static_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const bool ok = launch_smooth_first<double>(L.np, L.n, L.Dinv, b, scratch, (double*)nullptr, h->opt.omega, s) &&
                  launch_bsr<double>(3, L.np, L.n, L.hrowptr, L.hcol, L.Ahat, x, (const double*)scratch, y,
                                     h->opt.omega, nullptr, s,
                                     (((uintptr_t)x | (uintptr_t)y) & 15) == 0 ? D.scal + S_FLAG : nullptr,
                                     unr_of<double>(L, 3));
  if (!ok) {
    h->err = "unsupported n_p";
    return CDG_EINVAL;
  }
  CDG_CHECK_LAUNCH(h, "cdg_smooth_static");
  return CDG_OK;
}

static int gmres_len(const cdg_options& o) { return o.krylov == 1 ? o.restart : 0; }

int dev_bytes(const cdg_handle* h, int64_t* bytes) {
  *bytes = (int64_t)layout(h->H, h->opt.precision == 2 ? 1 : h->opt.precision, h->opt.nrhs, nullptr, nullptr,
                          h->opt.precision, gmres_len(h->opt), h->opt.maxit, h->opt.tc_fp64_apply);
  return CDG_OK;
}

void dev_release(cdg_handle* h) {
  if (h->dev) {
    DeviceState& D = *h->dev;
    if (D.g1) cudaGraphExecDestroy(D.g1);
    if (D.g2) cudaGraphExecDestroy(D.g2);
    if (D.gsolve) cudaGraphExecDestroy(D.gsolve);
    gmres_release(D);
    if (D.stream) {
      cudaStreamSynchronize(D.stream);
      cudaStreamDestroy(D.stream);
    }
    if (D.ev_in) cudaEventDestroy(D.ev_in);
    mr_delete(D.mr);
  }
  delete h->dev;
  h->dev = nullptr;
}

// Autotuner of the block-row tiling: times the vector-load block-sparse kernel
// with 1, 2 and 4 blocks in flight per step for every (level, operator
// precision, mode) that a solve launches, on the handle's own operators and
// zero-filled work vectors, and keeps the fastest.  Every variant sums in the
// same order, so the choice changes the timing only, never a result.
static int autotune_bsr(cdg_handle* h, cudaStream_t s) {
  DeviceState& D = *h->dev;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  const double w = h->opt.omega;
  double* flag = D.scal + S_FLAG;
  auto pick = [&](auto&& launch_one) -> int {
    int best = 2;
    float tbest = 3.0e38f;
    for (int u : {1, 2, 4}) {
      const float t = time_calls(s, e0, e1, 3, [&] { launch_one(u); });
      if (t < tbest) {
        tbest = t;
        best = u;
      }
    }
    return best;
  };
  // odd n_p: the scalar-load kernel has no variants (levels keep the default)
  // level 0, FP64: the outer apply and residual
  if (D.lev[0].np % 2 == 0) {
    DevLevel& L = D.lev[0];
    const int np = L.np;
    const size_t nb = sizeof(double) * (size_t)D.ndofs;
    cudaMemsetAsync(D.p, 0, nb, s);
    cudaMemsetAsync(D.q, 0, nb, s);
    cudaMemsetAsync(D.r, 0, nb, s);
    L.unr[0][0] = pick([&](int u) {
      launch_bsr<double>(0, np, L.n, L.rowptr, L.col, L.A, D.p, (const double*)nullptr, D.q, w, nullptr, s, flag, u);
    });
    L.unr[0][1] = pick([&](int u) {
      launch_bsr<double>(1, np, L.n, L.rowptr, L.col, L.A, D.p, D.r, D.q, w, nullptr, s, flag, u);
    });
  }
  // V-cycle levels in the V-cycle precision: residual and smoother sweep
  auto tune_level = [&](auto zero, DevLevel& L, int l) {
    using T = decltype(zero);
    const int np = L.np;
    if (np % 2 != 0) return;
    const int ti = sizeof(T) == 8 ? 0 : 1;
    const size_t nb = sizeof(T) * (size_t)L.n * np;
    T *x = (T*)L.x, *b = (T*)L.b, *bh = (T*)L.bh, *y = (T*)L.t;
    cudaMemsetAsync(x, 0, nb, s);
    cudaMemsetAsync(b, 0, nb, s);
    cudaMemsetAsync(bh, 0, nb, s);
    cudaMemsetAsync(y, 0, nb, s);
    if (l > 0 || ti == 1)
      L.unr[ti][1] = pick([&](int u) {
        launch_bsr<T>(1, np, L.n, L.rowptr, L.col, opA<T>(L), x, b, y, w, nullptr, s, flag, u);
      });
    L.unr[ti][3] = pick([&](int u) {
      launch_bsr<T>(3, np, L.n, L.hrowptr, L.hcol, opH<T>(L), x, bh, y, w, nullptr, s, flag, u);
    });
    if (ti == 1)   // the FP32 apply (cdg_apply_f32)
      L.unr[1][0] = pick([&](int u) {
        launch_bsr<T>(0, np, L.n, L.rowptr, L.col, opA<T>(L), x, (const T*)nullptr, y, w, nullptr, s, flag, u);
      });
  };
  for (int l = 0; l + 1 < D.nlev; ++l) {
    if (D.precision == 0) tune_level(0.0, D.lev[l], l);
    else tune_level(0.0f, D.lev[l], l);
  }
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  return CDG_OK;
}

int dev_tuning(const cdg_handle* h, int level, int32_t* out) {
  for (int k = 0; k < 13; ++k) out[k] = 0;
  const DeviceState& D = *h->dev;
  const DevLevel& L = D.lev[level];
  const bool vec = L.np % 2 == 0;
  if (vec && level == 0) {
    out[0] = L.unr[0][0];
    out[1] = L.unr[0][1];
  }
  if (vec && level + 1 < D.nlev) {
    const int ti = D.precision == 0 ? 0 : 1;
    out[2] = L.unr[ti][1];
    out[3] = L.unr[ti][3];
  }
  if (D.mr) mr_tuning(*D.mr, level, D.nlev, out);
  return CDG_OK;
}

int dev_bind(cdg_handle* h, void* buf, int64_t bytes, void* stream) {
  const cdg::Hierarchy& H = h->H;
  const int prec = h->opt.precision == 2 ? 1 : h->opt.precision;
  const int64_t need =
      (int64_t)layout(H, prec, h->opt.nrhs, nullptr, nullptr, h->opt.precision, gmres_len(h->opt), h->opt.maxit,
                      h->opt.tc_fp64_apply);
  if (bytes < need) {
    h->err = "device buffer too small: need " + std::to_string(need) + " bytes";
    return CDG_ENOMEM;
  }
  if (((uintptr_t)buf & 255) != 0) {
    h->err = "device buffer must be 256-byte aligned";
    return CDG_EINVAL;
  }
  dev_release(h);
  h->dev = new DeviceState();
  DeviceState& D = *h->dev;
  D.base = (char*)buf;
  D.bytes = bytes;
  layout(H, prec, h->opt.nrhs, &D, (char*)buf, h->opt.precision, gmres_len(h->opt), h->opt.maxit,
         h->opt.tc_fp64_apply);
  D.precision = h->opt.precision == 2 ? 1 : h->opt.precision;
  cudaStream_t s = (cudaStream_t)stream;
  const int nlev = D.nlev;
  for (int l = 0; l < nlev; ++l) {
    DevLevel& L = D.lev[l];
    const cdg::BSR& A = H.A_t[l];
    upload(L.rowptr, to_i32(A.rowptr), s);
    upload(L.col, A.col, s);
    if (L.A) upload(L.A, A.val, s);
    if (L.A32) upload(L.A32, to_f32(A.val), s);
    if (l + 1 < nlev) {
      if (L.Dinv) upload(L.Dinv, H.Dinv_t[l], s);
      if (L.L) upload(L.L, H.L_t[l], s);
      if (L.Dinv32) upload(L.Dinv32, to_f32(H.Dinv_t[l]), s);
      if (L.L32) upload(L.L32, to_f32(H.L_t[l]), s);
      upload(L.parent, H.parent_t[l], s);
      const cdg::BSR& Sh = H.Ahat_t[l];
      upload(L.hrowptr, to_i32(Sh.rowptr), s);
      upload(L.hcol, Sh.col, s);
      if (L.Ahat) upload(L.Ahat, Sh.val, s);
      if (L.Ahat32) upload(L.Ahat32, to_f32(Sh.val), s);
    }
    if (l > 0) upload(L.childptr, H.childptr_t[l], s);
    if (L.chunk) {
      int rows = 0, parents = 0;
      upload(L.chunk, agglomerate_chunks(H.childptr_t[l + 1], chunk_target(L.np), &rows, &parents), s);
    }
    // every synchronous upload above finishes before the host vectors die
    cudaStreamSynchronize(s);
  }
  upload(D.coarse_inv, H.coarse_inv, s);
  {
    std::vector<long long> sd(D.nseg + 1), co(D.nseg + 1);
    std::vector<int> cro(D.nseg + 1), crs(D.nc);
    const std::vector<cdg::i64>& r0 = H.seg_rows[0];
    const std::vector<cdg::i64>& rc = H.seg_rows[D.nlev - 1];
    for (int m = 0; m <= D.nseg; ++m) {
      sd[m] = (long long)r0[m] * D.np;
      cro[m] = (int)(rc[m] * D.lev[D.nlev - 1].np);
      co[m] = (long long)H.seg_coarse[m];
    }
    for (int m = 0; m < D.nseg; ++m)
      for (int r = cro[m]; r < cro[m + 1]; ++r) crs[r] = m;
    D.h_seg_dof = sd;
    upload(D.seg_dof, sd, s);
    upload(D.crow_off, cro, s);
    upload(D.cinv_off, co, s);
    upload(D.crow_seg, crs, s);
    cudaStreamSynchronize(s);
  }
  upload(D.rhs_vol, H.rhs_vol, s);
  upload(D.rhs_bptr, to_i32(H.rhs_bptr), s);
  upload(D.rhs_bface, to_i32(H.rhs_bface), s);
  upload(D.rhs_bdata, H.rhs_bD, s);
  upload(D.btag, std::vector<int>(H.mesh.bf_tag.begin(), H.mesh.bf_tag.end()), s);
  upload(D.perm0, to_i32(H.order[0]), s);
  upload(D.dk_own, H.dk_own, s);
  upload(D.dk_ptr, to_i32(H.dk_ptr), s);
  upload(D.dk_nbr, to_i32(H.dk_nbr), s);
  upload(D.dk_blk, H.dk_blk, s);
  upload(D.kappa, H.kappa_w, s);
  cudaMemsetAsync(D.scal, 0, sizeof(double) * S_COUNT * D.nseg, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&D.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&D.ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess && D.mr) {
    mr_upload(H, *D.mr, s);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "bind");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "bind");
  if (h->opt.autotune) return autotune_bsr(h, s);
  return CDG_OK;
}

int dev_rhs(cdg_handle* h, const double* f_q, const double* gD, const double* gN, double* b, bool user_out,
            void* stream) {
  if (!h->dev) {
    h->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  cudaStream_t s = (cudaStream_t)stream;
  CDG_NP_DISPATCH(D.np, launch(rhs_kernel<NP>, rows_grid(D.ne, D.np), kThreads, s, 
                            (int)D.ne, D.nq, D.nfq, D.perm0, D.rhs_vol, f_q, D.rhs_bptr, D.rhs_bface, D.rhs_bdata,
                            D.btag, gD, gN, b, user_out ? 1 : 0));
  CDG_CHECK_LAUNCH(h, "rhs");
  return CDG_OK;
}

int dev_permute(cdg_handle* h, const double* in, double* out, bool to_tree, void* stream) {
  if (!h || !h->dev) return h ? (h->err = "not bound", CDG_ESTATE) : CDG_EINVAL;
  DeviceState& D = *h->dev;
  cudaStream_t s = (cudaStream_t)stream;
  launch(permute_kernel, vec_grid((size_t)D.ndofs), kThreads, s, (int)D.ne, D.np, D.perm0, in, out, to_tree);
  CDG_CHECK_LAUNCH(h, "permute");
  return CDG_OK;
}

int dev_level_op(cdg_handle* h, int op, int level, const double* x, const double* b, double* y, void* stream) {
  if (!h) return CDG_EINVAL;
  if (!h->dev) {
    h->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  cudaStream_t s = (cudaStream_t)stream;
  if (op == 5) {
    if (!x || !y) {
      h->err = "NULL vector";
      return CDG_EINVAL;
    }
    coarse_solve<double>(D, x, y, s);
    CDG_CHECK_LAUNCH(h, "coarse");
    return CDG_OK;
  }
  if (level < 0 || level >= D.nlev || !x || !y) {
    h->err = "bad level or NULL vector";
    return CDG_EINVAL;
  }
  const DevLevel& L = D.lev[level];
  const bool last = level + 1 == D.nlev;
  const bool fp64 = L.A != nullptr;
  if (((op == 2 || op == 3 || op == 4) && (last || !L.Dinv)) || (op <= 1 && !fp64) || ((op == 1 || op == 2) && !b)) {
    h->err = "operation not available on this level in this precision";
    return CDG_EINVAL;
  }
  bool ok = true;
  // caller vectors that are not 16-byte aligned take the kernel without vector loads
  const bool aligned = (((uintptr_t)x | (uintptr_t)y | (uintptr_t)b) & 15) == 0;
  double* flag = aligned ? D.scal + S_FLAG : nullptr;
  if (op <= 1) {
    ok = launch_bsr<double>(op, L.np, L.n, L.rowptr, L.col, L.A, x, b, y, h->opt.omega, nullptr, s, flag,
                            unr_of<double>(L, op));
  } else if (op == 2) {
    ok = launch_smooth_first<double>(L.np, L.n, L.Dinv, b, (double*)L.bh, (double*)nullptr, h->opt.omega, s) &&
         launch_bsr<double>(3, L.np, L.n, L.hrowptr, L.hcol, L.Ahat, x, (const double*)L.bh, y, h->opt.omega,
                            nullptr, s, flag, unr_of<double>(L, 3));
  }
  else if (op == 3) ok = transfer_restrict<double>(D, level, L.L, x, y, s);
  else ok = transfer_prolong<double>(D, level, L.L, x, y, true, s);
  if (!ok) {
    h->err = "unsupported n_p";
    return CDG_EINVAL;
  }
  CDG_CHECK_LAUNCH(h, "level op");
  return CDG_OK;
}

int dev_set_wait_limit(cdg_handle* h, int limit) {
  if (!h->dev) {
    h->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  const int v = limit < 0 ? -1 : limit;
  if (v != D.wait_limit) {
    // captured graphs hold the limit as a kernel argument: capture again at the next solve
    cudaStreamSynchronize(D.stream);
    if (D.g1) cudaGraphExecDestroy(D.g1);
    if (D.g2) cudaGraphExecDestroy(D.g2);
    if (D.gsolve) cudaGraphExecDestroy(D.gsolve);
    D.g1 = D.g2 = D.gsolve = nullptr;
    gmres_release(D);
  }
  D.wait_limit = v;
  return CDG_OK;
}

int dev_fma_probe(int blocks, long long iters, double* sink, void* stream) {
  // 16 chains of iters / 2 steps: the same FMA count as 8 chains of iters steps
  launch(fma64_probe_kernel<16>, (unsigned)blocks, kThreads, (cudaStream_t)stream, (iters + 1) / 2, 0.5,
         0.9999999, 1e-7, sink);
  return cudaGetLastError() == cudaSuccess ? CDG_OK : CDG_ECUDA;
}

int dev_convert(const void* in, void* out, long long n, int to_fp32, void* stream) {
  if (n == 0) return CDG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (to_fp32)
    launch(convert_kernel<double, float>, vec_grid((size_t)n), kThreads, s, (size_t)n, (const double*)in, (float*)out);
  else
    launch(convert_kernel<float, double>, vec_grid((size_t)n), kThreads, s, (size_t)n, (const float*)in, (double*)out);
  return cudaGetLastError() == cudaSuccess ? CDG_OK : CDG_ECUDA;
}

int dev_solve_graph(const cdg_handle* h) { return h && h->dev && (h->dev->gsolve || h->dev->gm_cycle) ? 1 : 0; }

int dev_apply_f32(cdg_handle* h, int level, const float* x, float* y, void* stream) {
  if (!h || !x || !y) return CDG_EINVAL;
  if (!h->dev) {
    h->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  if (level < 0 || level >= D.nlev || !D.lev[level].A32) {
    h->err = "no FP32 operator on this level (precision 1 or 2 handles, levels below the coarsest)";
    return CDG_EINVAL;
  }
  const DevLevel& L = D.lev[level];
  const bool aligned = (((uintptr_t)x | (uintptr_t)y) & 15) == 0;
  if (!launch_bsr<float>(0, L.np, L.n, L.rowptr, L.col, L.A32, x, (const float*)nullptr, y, h->opt.omega, nullptr,
                         (cudaStream_t)stream, aligned ? D.scal + S_FLAG : nullptr, unr_of<float>(L, 0))) {
    h->err = "unsupported n_p";
    return CDG_EINVAL;
  }
  CDG_CHECK_LAUNCH(h, "cdg_apply_f32");
  return CDG_OK;
}

int dev_vcycle(cdg_handle* h, const double* r, double* z, void* stream) {
  if (!h) return CDG_EINVAL;
  if (!h->dev) {
    h->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  return precond(h, r, z, (cudaStream_t)stream);
}

// One CG iteration is split in two captured graphs: G1 = [q = A p, p.q, x and r
// updates, r.r] and G2 = [z = V(r), r.z, p = z + beta p].  The host reads the
// per-segment scalars between them (convergence of every mesh is decided on the
// device; converged meshes get alpha = beta = 0).
static int cg_part1(cdg_handle* h, cudaStream_t s) {
  DeviceState& D = *h->dev;
  const DevLevel& L0 = D.lev[0];
  const unsigned gseg = (unsigned)(D.nseg * D.bps);
  if (D.nseg == 1) {
    const unsigned g = rows_grid(L0.n, D.np);
    launch_bsr<double>(0, D.np, L0.n, L0.rowptr, L0.col, L0.A, D.p, (const double*)nullptr, D.q, h->opt.omega,
                       D.partial, s, D.scal + S_FLAG, unr_of<double>(L0, 0));
    launch(finalize_kernel, 1u, kThreads, s, (const double*)D.partial, (int)g, D.npartial, 0, 0, h->opt.tol,
           D.scal);
  } else {
    launch_bsr<double>(0, D.np, L0.n, L0.rowptr, L0.col, L0.A, D.p, (const double*)nullptr, D.q, h->opt.omega,
                       (double*)nullptr, s, D.scal + S_FLAG, unr_of<double>(L0, 0));
    int rc = dot_to(h, D.p, D.q, nullptr, 0, s);
    if (rc != CDG_OK) return rc;
  }
  launch(cg_update_kernel, gseg, kThreads, s, (const long long*)D.seg_dof, D.bps, (const double*)D.scal,
         (const double*)D.p, (const double*)D.q, D.x, D.r, D.partial);
  launch(finalize_kernel, (unsigned)D.nseg, kThreads, s, (const double*)D.partial, D.bps, D.npartial, 1, 0,
         h->opt.tol, D.scal);
  CDG_CHECK_LAUNCH(h, "cg");
  return CDG_OK;
}

static int cg_part2(cdg_handle* h, cudaStream_t s) {
  DeviceState& D = *h->dev;
  const bool flexible = D.precision != 0;
  const size_t n = (size_t)D.ndofs;
  if (flexible) cudaMemcpyAsync(D.zold, D.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  int rc = precond(h, D.r, D.z, s);
  if (rc != CDG_OK) return rc;
  if ((rc = dot_to(h, D.r, D.z, flexible ? D.zold : nullptr, 2, s)) != CDG_OK) return rc;
  launch(cg_p_kernel, (unsigned)(D.nseg * D.bps), kThreads, s, (const long long*)D.seg_dof, D.bps,
         (const double*)D.scal, 0, (const double*)D.z, D.p);
  CDG_CHECK_LAUNCH(h, "cg");
  return CDG_OK;
}

// Captures one part into an executable graph on the private stream.
static int capture(cdg_handle* h, int (*part)(cdg_handle*, cudaStream_t), cudaGraphExec_t* exec,
                   long long* kernels) {
  DeviceState& D = *h->dev;
  cudaGraph_t g = nullptr;
  const long long before = g_launches.load();
  cudaError_t e = cudaStreamBeginCapture(D.stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
  const int rc = part(h, D.stream);
  e = cudaStreamEndCapture(D.stream, &g);
  // captured launches run when the graph is launched: count them there
  *kernels = g_launches.load() - before;
  g_launches.fetch_sub(*kernels, std::memory_order_relaxed);
  if (rc != CDG_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
  return CDG_OK;
}

// The whole CG loop as one executable graph: WHILE (cond) { G1; check; G2 }.  The condition
// starts at 1 on every launch; the check kernel clears it when every segment has converged or
// maxit iterations are done, so the loop always ends.  G2 of the last iteration is not needed
// (it changes z and p only).
static int capture_solve(cdg_handle* h) {
  DeviceState& D = *h->dev;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "solve graph");
  cudaGraphConditionalHandle cond;
  e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = cond;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(h, e, "solve graph");
  }
  cudaGraph_t body = p.conditional.phGraph_out[0];
  const long long before = g_launches.load();
  e = cudaStreamBeginCaptureToGraph(D.stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(h, e, "solve graph capture");
  }
  int rc = cg_part1(h, D.stream);
  if (rc == CDG_OK) {
    launch(cg_check_kernel, 1u, 64u, D.stream, cond, D.nseg, h->opt.maxit, D.scal, D.it_dev, D.hist_dev,
           D.iters_dev, (const int*)D.pv_err);
    rc = cg_part2(h, D.stream);
  }
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(D.stream, &captured);
  D.gsolve_kernels = g_launches.load() - before;
  g_launches.fetch_sub(D.gsolve_kernels, std::memory_order_relaxed);
  if (rc != CDG_OK || e2 != cudaSuccess) {
    cudaGraphDestroy(g);
    return rc != CDG_OK ? rc : cuda_fail(h, e2, "solve graph capture");
  }
  e = cudaGraphInstantiate(&D.gsolve, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    D.gsolve = nullptr;
    return cuda_fail(h, e, "solve graph instantiate");
  }
  return CDG_OK;
}

int dev_solve(cdg_handle* h, const double* f_q, const double* gD, const double* gN, const double* b_user, double* u,
              int use_u0, double* res_hist, int* iters, int host_ptrs, void* stream) {
  if (!h->dev) {
    h->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  const int nseg = D.nseg;
  for (int m = 0; m < nseg; ++m) iters[m] = 0;
  // all work on the private stream, ordered after the caller's stream
  cudaStream_t cs = (cudaStream_t)stream;
  cudaStream_t s = D.stream;
  cudaEventRecord(D.ev_in, cs);
  cudaStreamWaitEvent(s, D.ev_in, 0);
  const cdg_options& o = h->opt;
  const size_t n = (size_t)D.ndofs;
  double* u_dev = u;
  int rc;
  if (host_ptrs) {
    cudaMemcpyAsync(D.f_stage, f_q, sizeof(double) * D.ne * D.nq, cudaMemcpyHostToDevice, s);
    if (gD) cudaMemcpyAsync(D.gD_stage, gD, sizeof(double) * D.nbf * D.nfq, cudaMemcpyHostToDevice, s);
    if (gN) cudaMemcpyAsync(D.gN_stage, gN, sizeof(double) * D.nbf * D.nfq, cudaMemcpyHostToDevice, s);
    if (use_u0) cudaMemcpyAsync(D.u_stage, u, sizeof(double) * n, cudaMemcpyHostToDevice, s);
    f_q = D.f_stage;
    gD = gD ? D.gD_stage : nullptr;
    gN = gN ? D.gN_stage : nullptr;
    u_dev = D.u_stage;
  }
  cudaMemsetAsync(D.scal, 0, sizeof(double) * S_COUNT * nseg, s);   // scalars and the wait-timeout flag
  cudaMemsetAsync(D.pv_err, 0, sizeof(int), s);
  // right-hand side in tree order
  if (b_user) {
    launch(permute_kernel, vec_grid(n), kThreads, s, (int)D.ne, D.np, D.perm0, b_user, D.bt, 1);
  } else if ((rc = dev_rhs(h, f_q, gD, gN, D.bt, false, s)) != CDG_OK) {
    return rc;
  }
  // initial guess and residual
  const DevLevel& L0 = D.lev[0];
  if (use_u0) {
    launch(permute_kernel, vec_grid(n), kThreads, s, (int)D.ne, D.np, D.perm0, u_dev, D.x, 1);
    launch_bsr<double>(1, D.np, L0.n, L0.rowptr, L0.col, L0.A, D.x, D.bt, D.r, o.omega, nullptr, s, D.scal + S_FLAG,
                       unr_of<double>(L0, 1));
  } else {
    cudaMemsetAsync(D.x, 0, sizeof(double) * n, s);
    cudaMemcpyAsync(D.r, D.bt, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  }
  if ((rc = dot_to(h, D.bt, D.bt, nullptr, 3, s)) != CDG_OK) return rc;
  if ((rc = dot_to(h, D.r, D.r, nullptr, 4, s)) != CDG_OK) return rc;
  std::vector<double> hs((size_t)S_COUNT * nseg);
  cudaMemcpyAsync(hs.data(), D.scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "solve init");
  const int stride = o.maxit + 1;
  auto rel = [&](int m) {
    const double* sc = &hs[(size_t)m * S_COUNT];
    return sc[S_BB] > 0.0 ? std::sqrt(sc[S_RR] / sc[S_BB]) : 0.0;
  };
  std::vector<char> done(nseg, 0);
  int ndone = 0;
  for (int m = 0; m < nseg; ++m) {
    if (res_hist) res_hist[(size_t)m * stride] = rel(m);
    if (hs[(size_t)m * S_COUNT + S_DONE] != 0.0) {
      done[m] = 1;
      ++ndone;
    }
  }
  int status = CDG_OK;
  int it = 0;
  if (o.krylov == 1) {
    if (ndone < nseg) {
      status = gmres_run(h, s, res_hist, iters);
      if (status != CDG_OK && status != CDG_ENOCONV && status != CDG_EBREAKDOWN) return status;
      it = iters[0];
      done[0] = status != CDG_ENOCONV;
    }
  } else if (ndone < nseg) {
    if ((rc = precond(h, D.r, D.z, s)) != CDG_OK) return rc;
    if ((rc = dot_to(h, D.r, D.z, nullptr, 2, s)) != CDG_OK) return rc;
    launch(cg_p_kernel, (unsigned)(nseg * D.bps), kThreads, s, (const long long*)D.seg_dof, D.bps,
           (const double*)D.scal, 1, (const double*)D.z, D.p);
    if (o.solve_graph && o.maxit > 0 && !D.gsolve && !D.gsolve_failed && capture_solve(h) != CDG_OK) {
      D.gsolve_failed = true;   // refused by this driver: keep the host-driven loop
      h->err.clear();
      cudaGetLastError();
    }
    bool in_graph = false;
    if (o.solve_graph && o.maxit > 0 && D.gsolve) {
      launch(hist_init_kernel, 1u, 64u, s, nseg, D.scal);
      cudaMemsetAsync(D.it_dev, 0, sizeof(int), s);
      cudaMemsetAsync(D.iters_dev, 0, sizeof(int) * nseg, s);
      e = cudaGraphLaunch(D.gsolve, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
      std::vector<double> hh((size_t)nseg * stride);
      std::vector<int> ih(nseg);
      int itd = 0;
      cudaMemcpyAsync(hh.data(), D.hist_dev, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(ih.data(), D.iters_dev, sizeof(int) * nseg, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(&itd, D.it_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(hs.data(), D.scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(h, e, "cg");
      g_launches.fetch_add(D.gsolve_kernels * itd, std::memory_order_relaxed);
      it = itd;
      for (int m = 0; m < nseg; ++m) {
        if (done[m]) continue;
        iters[m] = ih[m];
        if (res_hist)
          for (int k = 1; k <= ih[m]; ++k) res_hist[(size_t)m * stride + k] = hh[(size_t)m * stride + k];
        const double* sc = &hs[(size_t)m * S_COUNT];
        if (sc[S_DONE] != 0.0) {
          done[m] = 1;
          ++ndone;
          if (sc[S_BREAK] != 0.0) {
            status = CDG_EBREAKDOWN;
            h->err = "CG breakdown on mesh " + std::to_string(m) + " at iteration " + std::to_string(ih[m]) +
                     ": p^T A p = " + std::to_string(sc[S_PQ]) + ", ||r||^2 = " + std::to_string(sc[S_RR]);
          }
        }
      }
      if (ndone < nseg) status = CDG_ENOCONV;
      in_graph = true;
    }
    if (!in_graph && !D.g1 && (rc = capture(h, cg_part1, &D.g1, &D.g1_kernels)) != CDG_OK) return rc;
    if (!in_graph && !D.g2 && (rc = capture(h, cg_part2, &D.g2, &D.g2_kernels)) != CDG_OK) return rc;
    while (!in_graph) {
      if (it >= o.maxit) {
        status = CDG_ENOCONV;
        break;
      }
      e = cudaGraphLaunch(D.g1, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
      cudaMemcpyAsync(hs.data(), D.scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(h, e, "cg");
      g_launches.fetch_add(D.g1_kernels, std::memory_order_relaxed);
      ++it;
      for (int m = 0; m < nseg; ++m) {
        if (done[m]) continue;
        const double* sc = &hs[(size_t)m * S_COUNT];
        iters[m] = it;
        if (res_hist) res_hist[(size_t)m * stride + it] = rel(m);
        if (sc[S_DONE] != 0.0) {
          done[m] = 1;
          ++ndone;
          if (sc[S_BREAK] != 0.0) {
            status = CDG_EBREAKDOWN;
            h->err = "CG breakdown on mesh " + std::to_string(m) + " at iteration " + std::to_string(it) +
                     ": p^T A p = " + std::to_string(sc[S_PQ]) + ", ||r||^2 = " + std::to_string(sc[S_RR]);
          }
        }
      }
      if (ndone == nseg) break;
      e = cudaGraphLaunch(D.g2, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
      g_launches.fetch_add(D.g2_kernels, std::memory_order_relaxed);
    }
  }
  launch(permute_kernel, vec_grid(n), kThreads, s, (int)D.ne, D.np, D.perm0, D.x, u_dev, 0);
  if (host_ptrs) cudaMemcpyAsync(u, D.u_stage, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
  int pv_err = 0;
  cudaMemcpyAsync(&pv_err, D.pv_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "solve end");
  CDG_CHECK_LAUNCH(h, "solve end");
  if (pv_err) {
    h->err = "a grid barrier of the persistent V-cycle reached its iteration limit";
    return CDG_ETIMEOUT;
  }
  if (status == CDG_ENOCONV) {
    for (int m = 0; m < nseg; ++m)
      if (!done[m]) iters[m] = it;
    h->err = "maximum number of iterations reached";
  }
  return status;
}

int dev_adjoint(cdg_handle* h, int what, const double* lam_user, const double* u_user, const double* gD,
                double* out, void* stream) {
  if (!h) return CDG_EINVAL;
  if (!h->dev) {
    h->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  DeviceState& D = *h->dev;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)D.ndofs;
  // lambda (and u) to tree order in the CG work vectors (free outside a solve)
  launch(permute_kernel, vec_grid(n), kThreads, s, (int)D.ne, D.np, D.perm0, lam_user, D.r, 1);
  if (what == 0) {
    const size_t tot = (size_t)D.ne * D.nq;
    CDG_NP_DISPATCH(D.np, launch(rhs_adjoint_kernel<NP>, (unsigned)((tot + 255) / 256), 256, s, (int)D.ne, D.nq,
                                 D.perm0, D.rhs_vol, D.r, out));
  } else {
    launch(permute_kernel, vec_grid(n), kThreads, s, (int)D.ne, D.np, D.perm0, u_user, D.z, 1);
    CDG_NP_DISPATCH(D.np, launch(kappa_grad_kernel<NP>, rows_grid(D.ne, D.np), kThreads, s, (int)D.ne, D.nfq,
                                 D.perm0, D.dk_own, D.dk_ptr, D.dk_nbr, D.dk_blk, D.kappa, D.r, D.z, D.rhs_bptr,
                                 D.rhs_bface, D.rhs_bdata, D.btag, gD, out));
  }
  CDG_CHECK_LAUNCH(h, "adjoint");
  return CDG_OK;
}
