// Restarted GMRES(m) with one V-cycle as right preconditioner: the outer Krylov
// method of the paper (Section 4; GMRES(50) with V(0,3) and a relative
// residual of 1e-8 in Section 5).  The flexible form (Saad 1993) keeps the
// preconditioned vectors z_j = M^{-1} v_j, so x = x0 + Z_k y_k needs no extra
// V-cycle and an FP32 V-cycle (not an exactly fixed linear operator) is still
// handled exactly by the minimisation.  With a fixed preconditioner it equals
// right-preconditioned GMRES.
//
// One Arnoldi step is one captured CUDA graph; the step index j lives in device
// memory, so the same graph serves every step:
//   r <- v_j;  z <- V-cycle(r);  z_j <- z;  w <- A_0 z
//   classical Gram-Schmidt:  h = V_j^T w,  w -= V_j h,  and a second pass when
//   ||w|| dropped below ||w_before||/sqrt(2) (re-orthogonalisation, "twice is
//   enough"); h_{j+1,j} = ||w||;  v_{j+1} = w / h_{j+1,j}
//   plane rotations on the new Hessenberg column, g_{j+1} = -s_j g_j,
//   convergence |g_{j+1}| <= tol ||b||, j <- j + 1.
// The host reads the scalars after each step (as the CG driver does).  At the
// end of a cycle y solves the k x k triangular system, x += Z_k y, and the
// true residual b - A_0 x starts the next cycle.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "device_state.h"

namespace {

template <typename... KArgs, typename... Args>
inline void launch(void (*k)(KArgs...), dim3 g, dim3 b, cudaStream_t s, Args... args) {
  k<<<g, b, 0, s>>>(args...);
  count_launch();
}

// rows [a, b) of n owned by this block
__device__ __forceinline__ void block_rows(size_t n, size_t& a, size_t& b) {
  a = n * blockIdx.x / gridDim.x;
  b = n * (blockIdx.x + 1) / gridDim.x;
}

__device__ __forceinline__ int step_index(const GmLayout& L, const double* st) {
  return (int)st[L.misc() + GM_J];
}

__device__ __forceinline__ bool reorth_skipped(const GmLayout& L, int pass, const double* st) {
  return pass == 2 && st[L.misc() + GM_REORTH] == 0.0;
}

// sum of one row of kGmBlocks partials in a fixed order (one block)
__device__ __forceinline__ double sum_row(const double* __restrict__ row, int G) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int t = threadIdx.x; t < G; t += blockDim.x) s += row[t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) tot += red[w];
  return tot;
}

// V_0 = r / ||r||, g = ||r|| e_1, j = 0 (||r||^2 is S_RR of the CG scalars)
__global__ void __launch_bounds__(kThreads) gm_init_kernel(size_t n, GmLayout L, const double* __restrict__ scal,
                                                           const double* __restrict__ r, double* __restrict__ V0,
                                                           double* __restrict__ st) {
  const double beta = sqrt(scal[S_RR]);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    V0[i] = r[i] / beta;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st[L.g()] = beta;
    st[L.misc() + GM_J] = 0.0;
  }
}

// out = V_j (load) or V_j = in (store, into the Z basis), j from the device
template <bool STORE>
__global__ void __launch_bounds__(kThreads) gm_copy_kernel(size_t n, size_t ld, GmLayout L,
                                                           const double* __restrict__ st, double* __restrict__ basis,
                                                           double* __restrict__ vec) {
  double* v = basis + (size_t)step_index(L, st) * ld;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (STORE) v[i] = vec[i];
    else vec[i] = v[i];
  }
}

// Partial dots over the block's rows: part[i][blk] = (v_i, w) for i <= j and,
// in pass 1, part[m][blk] = (w, w).  Eight basis vectors per sweep over the
// rows, so w is read once per eight dots (from L2 after the first sweep).
__global__ void __launch_bounds__(kThreads) gm_dot_kernel(size_t n, size_t ld, GmLayout L, int pass,
                                                          const double* __restrict__ st,
                                                          const double* __restrict__ V,
                                                          const double* __restrict__ w, double* __restrict__ part) {
  if (reorth_skipped(L, pass, st)) return;
  __shared__ double red[9][kThreads / 32];
  const int nd = step_index(L, st) + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  size_t a, b;
  block_rows(n, a, b);
  for (int i0 = 0; i0 < nd; i0 += 8) {
    const int cnt = min(8, nd - i0);
    const double* v = V + (size_t)i0 * ld;
    double acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0;
    for (size_t r = a + threadIdx.x; r < b; r += blockDim.x) {
      const double wr = w[r];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < cnt) acc[k] = fma(v[(size_t)k * ld + r], wr, acc[k]);
      acc[8] = fma(wr, wr, acc[8]);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double x = acc[k];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
      const int k = threadIdx.x;
      double s = 0.0;
      for (int q = 0; q < kThreads / 32; ++q) s += red[k][q];
      if (k < cnt) part[(size_t)(i0 + k) * gridDim.x + blockIdx.x] = s;
      else if (k == 8 && pass == 1 && i0 == 0) part[(size_t)L.m * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// Block i sums partial row i.  Pass 1: h[i] for i <= j, and ||w||^2 before the
// projection from row m (block m).  Pass 2: h2[i], and h[i] += h2[i].
__global__ void __launch_bounds__(kThreads) gm_hsum_kernel(GmLayout L, int pass, int G,
                                                           const double* __restrict__ part, double* __restrict__ st) {
  if (reorth_skipped(L, pass, st)) return;
  const int j = step_index(L, st);
  const int i = blockIdx.x;
  int row;
  if (i <= j) row = i;
  else if (pass == 1 && i == L.m) row = L.m;
  else return;
  const double s = sum_row(part + (size_t)row * G, G);
  if (threadIdx.x != 0) return;
  if (i > j) st[L.misc() + GM_WN0] = s;
  else if (pass == 1) st[L.h() + i] = s;
  else {
    st[L.h2() + i] = s;
    st[L.h() + i] += s;
  }
}

// w -= sum_{i <= j} c_i v_i (c = h in pass 1, h2 in pass 2) and
// part[m+1][blk] = (w, w) over the block's rows
__global__ void __launch_bounds__(kThreads) gm_axpy_kernel(size_t n, size_t ld, GmLayout L, int pass,
                                                           const double* __restrict__ st,
                                                           const double* __restrict__ V, double* __restrict__ w,
                                                           double* __restrict__ part) {
  if (reorth_skipped(L, pass, st)) return;
  extern __shared__ double c[];
  const int nd = step_index(L, st) + 1;
  const double* coef = st + (pass == 1 ? L.h() : L.h2());
  for (int t = threadIdx.x; t < nd; t += blockDim.x) c[t] = coef[t];
  __syncthreads();
  size_t a, b;
  block_rows(n, a, b);
  double s = 0.0;
  for (size_t r = a + threadIdx.x; r < b; r += blockDim.x) {
    double acc = w[r];
    int i = 0;
    for (; i + 4 <= nd; i += 4) {
      const double v0 = V[(size_t)i * ld + r], v1 = V[(size_t)(i + 1) * ld + r];
      const double v2 = V[(size_t)(i + 2) * ld + r], v3 = V[(size_t)(i + 3) * ld + r];
      acc = fma(-c[i], v0, acc);
      acc = fma(-c[i + 1], v1, acc);
      acc = fma(-c[i + 2], v2, acc);
      acc = fma(-c[i + 3], v3, acc);
    }
    for (; i < nd; ++i) acc = fma(-c[i], V[(size_t)i * ld + r], acc);
    w[r] = acc;
    s = fma(acc, acc, s);
  }
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) tot += red[q];
    part[(size_t)(L.m + 1) * gridDim.x + blockIdx.x] = tot;
  }
}

// h_{j+1,j} = ||w||.  Pass 1 also decides the second pass: ||w|| < ||w_before||/sqrt(2).
__global__ void __launch_bounds__(kThreads) gm_norm_kernel(GmLayout L, int pass, int G,
                                                           const double* __restrict__ part, double* __restrict__ st) {
  if (reorth_skipped(L, pass, st)) return;
  const double s = sum_row(part + (size_t)(L.m + 1) * G, G);
  if (threadIdx.x != 0) return;
  st[L.misc() + GM_HNEXT] = sqrt(s);
  if (pass == 1) {
    st[L.misc() + GM_WN1] = s;
    st[L.misc() + GM_REORTH] = (s < 0.5 * st[L.misc() + GM_WN0]) ? 1.0 : 0.0;
  }
}

// v_{j+1} = w / h_{j+1,j} (skipped on a happy or a non-finite breakdown)
__global__ void __launch_bounds__(kThreads) gm_scale_kernel(size_t n, size_t ld, GmLayout L,
                                                            const double* __restrict__ st,
                                                            const double* __restrict__ w, double* __restrict__ V) {
  const double hn = st[L.misc() + GM_HNEXT];
  if (!(hn > 0.0) || !isfinite(hn)) return;
  double* v = V + (size_t)(step_index(L, st) + 1) * ld;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = w[i] / hn;
}

// One thread: the earlier rotations on column j of the Hessenberg, a new
// rotation that zeroes h_{j+1,j}, the rotated right-hand side g, the
// residual estimate |g_{j+1}| (into S_RR as its square) and the stop test.
__global__ void gm_givens_kernel(GmLayout L, double tol, double* __restrict__ st, double* __restrict__ scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = L.m;
  const int j = step_index(L, st);
  double* col = st + L.h();
  const double hn = st[L.misc() + GM_HNEXT];
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double c = st[L.cs() + i], s = st[L.sn() + i];
    const double a = col[i], b = col[i + 1];
    col[i] = c * a + s * b;
    col[i + 1] = -s * a + c * b;
  }
  const double a = col[j], b = col[j + 1];
  double c = 1.0, s = 0.0, r = a;
  if (b != 0.0) {
    r = hypot(a, b);
    c = a / r;
    s = b / r;
  }
  st[L.cs() + j] = c;
  st[L.sn() + j] = s;
  for (int i = 0; i < j; ++i) st[L.R() + i + (size_t)j * m] = col[i];
  st[L.R() + j + (size_t)j * m] = r;
  const double gj = st[L.g() + j];
  st[L.g() + j + 1] = -s * gj;
  st[L.g() + j] = c * gj;
  const double res = fabs(st[L.g() + j + 1]);
  scal[S_RR] = res * res;
  scal[S_IT] += 1.0;
  if (!isfinite(res) || !isfinite(r) || r == 0.0) {
    scal[S_BREAK] = 1.0;
    scal[S_DONE] = 1.0;
  } else if (res <= tol * sqrt(scal[S_BB]) || hn == 0.0) {
    scal[S_DONE] = 1.0;
  }
  st[L.misc() + GM_J] = (double)(j + 1);
}

// y = R_k^{-1} g_k (k x k upper triangular, one thread)
__global__ void gm_backsolve_kernel(GmLayout L, int k, double* __restrict__ st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = L.m;
  for (int i = k - 1; i >= 0; --i) {
    double s = st[L.g() + i];
    for (int l = i + 1; l < k; ++l) s -= st[L.R() + i + (size_t)l * m] * st[L.y() + l];
    st[L.y() + i] = s / st[L.R() + i + (size_t)i * m];
  }
}

// x += Z_k y
__global__ void __launch_bounds__(kThreads) gm_update_kernel(size_t n, size_t ld, GmLayout L, int k,
                                                             const double* __restrict__ st,
                                                             const double* __restrict__ Z, double* __restrict__ x) {
  extern __shared__ double y[];
  for (int t = threadIdx.x; t < k; t += blockDim.x) y[t] = st[L.y() + t];
  __syncthreads();
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < n; r += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc = fma(y[i], Z[(size_t)i * ld + r], acc);
    x[r] += acc;
  }
}

// After an Arnoldi step of the single-graph cycle (one thread): count the step,
// record |g_{j+1}|/||b||, and keep looping while the cycle has room (j < m), the
// solve is not done and fewer than maxit steps have run.
__global__ void gm_check_kernel(cudaGraphConditionalHandle cond, GmLayout L, int maxit,
                                const double* __restrict__ st, const double* __restrict__ scal,
                                int* __restrict__ it_dev, double* __restrict__ hist) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int it = *it_dev + 1;
  *it_dev = it;
  hist[it] = scal[S_BB] > 0.0 ? sqrt(scal[S_RR] / scal[S_BB]) : 0.0;
  const int j = step_index(L, st);
  cudaGraphSetConditional(cond, (scal[S_DONE] == 0.0 && j < L.m && it < maxit) ? 1u : 0u);
}

// One Arnoldi step (captured once per handle into D.gm_step).
int arnoldi_step(cdg_handle* h, cudaStream_t s) {
  DeviceState& D = *h->dev;
  const GmLayout L{D.gm_m};
  const size_t n = (size_t)D.ndofs, ld = D.gm_ld;
  const unsigned G = kGmBlocks;
  const size_t coef_bytes = sizeof(double) * (size_t)(D.gm_m + 1);
  int rc;
  launch(gm_copy_kernel<false>, G, kThreads, s, n, ld, L, (const double*)D.gm_st, D.gm_V, D.r);
  if ((rc = dev_precond(h, D.r, D.z, s)) != CDG_OK) return rc;
  launch(gm_copy_kernel<true>, G, kThreads, s, n, ld, L, (const double*)D.gm_st, D.gm_Z, D.z);
  if ((rc = dev_apply0(h, 0, D.z, nullptr, D.q, s)) != CDG_OK) return rc;
  for (int pass = 1; pass <= 2; ++pass) {
    launch(gm_dot_kernel, G, kThreads, s, n, ld, L, pass, (const double*)D.gm_st, (const double*)D.gm_V,
           (const double*)D.q, D.gm_part);
    launch(gm_hsum_kernel, (unsigned)(D.gm_m + 1), kThreads, s, L, pass, (int)G, (const double*)D.gm_part,
           D.gm_st);
    gm_axpy_kernel<<<G, kThreads, coef_bytes, s>>>(n, ld, L, pass, D.gm_st, D.gm_V, D.q, D.gm_part);
    count_launch();
    launch(gm_norm_kernel, 1u, kThreads, s, L, pass, (int)G, (const double*)D.gm_part, D.gm_st);
  }
  launch(gm_scale_kernel, G, kThreads, s, n, ld, L, (const double*)D.gm_st, (const double*)D.q, D.gm_V);
  launch(gm_givens_kernel, 1u, 32u, s, L, h->opt.tol, D.gm_st, D.scal);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dev_cuda_fail(h, e, "GMRES step");
  return CDG_OK;
}

int capture_step(cdg_handle* h) {
  DeviceState& D = *h->dev;
  cudaGraph_t g = nullptr;
  const long long before = launch_count();
  cudaError_t e = cudaStreamBeginCapture(D.stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return dev_cuda_fail(h, e, "GMRES graph capture");
  const int rc = arnoldi_step(h, D.stream);
  e = cudaStreamEndCapture(D.stream, &g);
  // captured launches run when the graph is launched: count them there
  D.gm_step_kernels = launch_count() - before;
  count_launch(-D.gm_step_kernels);
  if (rc != CDG_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return dev_cuda_fail(h, e, "GMRES graph capture");
  e = cudaGraphInstantiate(&D.gm_step, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return dev_cuda_fail(h, e, "GMRES graph instantiate");
  return CDG_OK;
}

// A restart cycle as one executable graph: WHILE (cond) { Arnoldi step; check }.  The
// condition is 1 at every launch; the check clears it at convergence, breakdown, a full
// cycle or maxit, and the step counter bounds the loop.
int capture_cycle(cdg_handle* h) {
  DeviceState& D = *h->dev;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return dev_cuda_fail(h, e, "GMRES cycle graph");
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
    return dev_cuda_fail(h, e, "GMRES cycle graph");
  }
  const long long before = launch_count();
  e = cudaStreamBeginCaptureToGraph(D.stream, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return dev_cuda_fail(h, e, "GMRES cycle capture");
  }
  int rc = arnoldi_step(h, D.stream);
  if (rc == CDG_OK)
    launch(gm_check_kernel, 1u, 32u, D.stream, cond, GmLayout{D.gm_m}, h->opt.maxit, (const double*)D.gm_st,
           (const double*)D.scal, D.it_dev, D.hist_dev);
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(D.stream, &captured);
  // captured launches are counted per executed step
  count_launch(-(launch_count() - before));
  if (rc != CDG_OK || e2 != cudaSuccess) {
    cudaGraphDestroy(g);
    return rc != CDG_OK ? rc : dev_cuda_fail(h, e2, "GMRES cycle capture");
  }
  e = cudaGraphInstantiate(&D.gm_cycle, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    D.gm_cycle = nullptr;
    return dev_cuda_fail(h, e, "GMRES cycle instantiate");
  }
  return CDG_OK;
}

}  // namespace

void gmres_release(DeviceState& D) {
  if (D.gm_step) cudaGraphExecDestroy(D.gm_step);
  if (D.gm_cycle) cudaGraphExecDestroy(D.gm_cycle);
  D.gm_step = nullptr;
  D.gm_cycle = nullptr;
}

int gmres_run(cdg_handle* h, cudaStream_t s, double* res_hist, int* iters) {
  DeviceState& D = *h->dev;
  const cdg_options& o = h->opt;
  iters[0] = 0;
  if (D.nseg != 1 || D.gm_m < 1 || !D.gm_V) {
    h->err = "GMRES needs a single-mesh handle created with krylov = 1";
    return CDG_EINVAL;
  }
  const GmLayout L{D.gm_m};
  const size_t n = (size_t)D.ndofs, ld = D.gm_ld;
  const unsigned G = kGmBlocks;
  int rc;
  if (!D.gm_step && (rc = capture_step(h)) != CDG_OK) return rc;
  if (o.solve_graph && !D.gm_cycle && !D.gm_cycle_failed && capture_cycle(h) != CDG_OK) {
    D.gm_cycle_failed = true;   // refused by this driver: one graph launch and host read per step
    h->err.clear();
    cudaGetLastError();
  }
  cudaMemsetAsync(D.it_dev, 0, sizeof(int), s);
  const long long gk = D.gm_step_kernels + 1;   // kernels per step of the cycle graph
  std::vector<double> hs(S_COUNT);
  auto read = [&](const char* where) -> int {
    cudaMemcpyAsync(hs.data(), D.scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? CDG_OK : dev_cuda_fail(h, e, where);
  };
  auto rel = [&]() { return hs[S_BB] > 0.0 ? std::sqrt(hs[S_RR] / hs[S_BB]) : 0.0; };
  int it = 0, status = CDG_OK;
  while (true) {
    launch(gm_init_kernel, G, kThreads, s, n, L, (const double*)D.scal, (const double*)D.r, D.gm_V, D.gm_st);
    int k = 0;
    bool stop = false, broke = false;
    if (D.gm_cycle && it < o.maxit) {
      const cudaError_t e = cudaGraphLaunch(D.gm_cycle, s);
      if (e != cudaSuccess) return dev_cuda_fail(h, e, "GMRES graph launch");
      int itd = it;
      std::vector<double> hh((size_t)o.maxit + 1);
      cudaMemcpyAsync(&itd, D.it_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(hh.data(), D.hist_dev, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, s);
      if ((rc = read("GMRES cycle")) != CDG_OK) return rc;
      k = itd - it;
      count_launch(gk * k);
      if (res_hist)
        for (int t = it + 1; t <= itd; ++t) res_hist[t] = hh[t];
      it = itd;
      broke = hs[S_BREAK] != 0.0;
      stop = broke || hs[S_DONE] != 0.0;
    }
    while (!D.gm_cycle && k < D.gm_m && it < o.maxit) {
      const cudaError_t e = cudaGraphLaunch(D.gm_step, s);
      if (e != cudaSuccess) return dev_cuda_fail(h, e, "GMRES graph launch");
      count_launch(D.gm_step_kernels);
      if ((rc = read("GMRES step")) != CDG_OK) return rc;
      ++k;
      ++it;
      if (res_hist) res_hist[it] = rel();
      if (hs[S_BREAK] != 0.0) {
        broke = stop = true;
        break;
      }
      if (hs[S_DONE] != 0.0) {
        stop = true;
        break;
      }
    }
    // a breakdown column (singular or non-finite) is left out of the update
    const int kk = broke ? k - 1 : k;
    if (kk > 0) {
      launch(gm_backsolve_kernel, 1u, 32u, s, L, kk, D.gm_st);
      gm_update_kernel<<<G, kThreads, sizeof(double) * (size_t)kk, s>>>(n, ld, L, kk, D.gm_st, D.gm_Z, D.x);
      count_launch();
    }
    // true residual of the updated x (starts the next cycle)
    if ((rc = dev_apply0(h, 1, D.x, D.bt, D.r, s)) != CDG_OK) return rc;
    cudaMemsetAsync(D.scal + S_DONE, 0, sizeof(double), s);
    if ((rc = dev_dot(h, D.r, D.r, 4, s)) != CDG_OK) return rc;
    if ((rc = read("GMRES restart")) != CDG_OK) return rc;
    if (res_hist) res_hist[it] = rel();
    if (broke) {
      status = CDG_EBREAKDOWN;
      h->err = "GMRES breakdown at iteration " + std::to_string(it) + " (singular or non-finite Hessenberg column)";
      break;
    }
    if (stop || hs[S_DONE] != 0.0) break;
    if (it >= o.maxit) {
      status = CDG_ENOCONV;
      break;
    }
  }
  iters[0] = it;
  return status;
}
