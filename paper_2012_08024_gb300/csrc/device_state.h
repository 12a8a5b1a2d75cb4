// Device-side state of a bound handle, shared by the solve-phase translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <vector>

#include "handle.h"

constexpr int kMaxLev = CDG_MAX_LEVELS;
constexpr int kThreads = 256;
constexpr int kDotBlocks = 8 * 152;   // fixed grid of the vector kernels of batched handles (8 CTAs per SM)
constexpr int kDotBlocks1 = 2 * 152;  // the same for single-mesh handles (their dot partials: 2 CTAs per SM)

// per-segment CG scalars (one row of S_COUNT doubles per mesh of the handle)
// S_HDONE: the segment's residual history is closed (single-graph solve)
enum Scal { S_RZ = 0, S_PQ, S_RR, S_BB, S_ALPHA, S_BETA, S_DONE, S_BREAK, S_IT, S_HDONE, S_FLAG = 15, S_COUNT = 16 };

struct DevLevel {
  int n = 0;
  int np = 0;                // basis functions per element on this level
  bool ptrans = false;       // level l -> l+1 lowers the degree on the same elements (truncation)
  int64_t nnzb = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* A = nullptr;
  double* Dinv = nullptr;
  double* L = nullptr;
  int* parent = nullptr;
  int* childptr = nullptr;   // children range of each element of this level (l >= 1)
  // chunks of whole agglomerates of level l+1 for the fused residual + restriction
  // (one CTA each): parent boundaries [nchunk+1]; rows / parents of the largest chunk
  int* chunk = nullptr;
  int nchunk = 0, chunk_rows = 0, chunk_parents = 0;
  float* A32 = nullptr;
  float* Dinv32 = nullptr;
  float* L32 = nullptr;
  int* hrowptr = nullptr;    // Ahat = D^{-1}(A - D): row-scaled off-diagonal blocks (smoother)
  int* hcol = nullptr;
  double* Ahat = nullptr;
  float* Ahat32 = nullptr;
  int64_t hnnzb = 0;
  // autotuned blocks in flight per step of the vector-load block-sparse kernel,
  // [0] FP64 / [1] FP32 operator, by mode (0 apply, 1 residual, 3 smoother)
  int unr[2][4] = {{2, 2, 2, 2}, {2, 2, 2, 2}};
  void* bh = nullptr;        // D^{-1} b of the current V-cycle visit
  void* x = nullptr;         // V-cycle work vectors in the V-cycle precision
  void* t = nullptr;
  void* r = nullptr;
  void* b = nullptr;
};

struct DeviceState {
  char* base = nullptr;
  int64_t bytes = 0;
  int nlev = 0, np = 0, d = 0, nq = 0, nfq = 0, precision = 0;
  int64_t ne = 0, ndofs = 0, nbf = 0;
  DevLevel lev[kMaxLev];
  double* coarse_inv = nullptr;
  int nc = 0;
  double* coarse_b = nullptr;   // FP64 staging of the coarsest right-hand side / solution
  double* coarse_x = nullptr;
  // rhs data
  double* rhs_vol = nullptr;
  int* rhs_bptr = nullptr;
  int* rhs_bface = nullptr;
  double* rhs_bdata = nullptr;
  int* btag = nullptr;
  int* perm0 = nullptr;         // tree row -> user element
  // d A_0 / d kappa pieces (tree order)
  double* dk_own = nullptr;
  int* dk_ptr = nullptr;
  int* dk_nbr = nullptr;
  double* dk_blk = nullptr;
  double* kappa = nullptr;
  // CG vectors (FP64, tree order)
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *bt = nullptr,
         *zold = nullptr;
  float *r32 = nullptr, *z32 = nullptr;
  // staging for host-pointer solves
  double *f_stage = nullptr, *gD_stage = nullptr, *gN_stage = nullptr, *u_stage = nullptr;
  double* scal = nullptr;       // [nseg][S_COUNT]
  double* partial = nullptr;
  int npartial = 0;
  // segments (meshes of a batched handle)
  int nseg = 1, bps = 1;        // blocks per segment of the segmented vector kernels
  long long* seg_dof = nullptr; // [nseg+1] level-0 dof offsets
  int* crow_seg = nullptr;      // [nc] segment of each coarsest row
  int* crow_off = nullptr;      // [nseg+1] coarsest row offsets
  long long* cinv_off = nullptr;// [nseg+1] offsets of the dense inverses
  std::vector<long long> h_seg_dof;
  // private stream and the two captured graphs of a CG iteration
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr;
  cudaGraphExec_t g1 = nullptr, g2 = nullptr;
  long long g1_kernels = 0, g2_kernels = 0;
  // iteration limit of the bounded device waits inside kernel loops (< 0: each kernel's
  // default); set by cdg_set_wait_limit to exercise the timeout path
  int wait_limit = -1;
  // persistent V-cycle (device_persist.cu): grid-barrier words, its error flag, and
  // whether it was refused (e.g. a cooperative launch inside a graph capture)
  unsigned* pv_count = nullptr;
  int* pv_err = nullptr;
  bool pv_failed = false;
  // the whole CG solve as one graph: a conditional WHILE node around [G1, check, G2];
  // the check kernel records the residual histories and ends the loop on the device
  cudaGraphExec_t gsolve = nullptr;
  long long gsolve_kernels = 0;   // kernels per loop iteration
  bool gsolve_failed = false;     // capture or instantiation refused: two graphs per iteration
  int* it_dev = nullptr;          // iterations done
  int* iters_dev = nullptr;       // [nseg]
  double* hist_dev = nullptr;     // [nseg][maxit+1]
  // multi-right-hand-side solve (cdg_solve_multi): R columns per vector
  int nrhs = 0;
  struct MR* mr = nullptr;   // device_multi.cu
  // restarted flexible GMRES (device_gmres.cu): Krylov basis V, preconditioned
  // vectors Z (row stride gm_ld), dot partials and the small Arnoldi state
  int gm_m = 0;
  size_t gm_ld = 0;
  double* gm_V = nullptr;    // [m+1][gm_ld]
  double* gm_Z = nullptr;    // [m][gm_ld]
  double* gm_part = nullptr; // [m+2][kGmBlocks]
  double* gm_st = nullptr;   // GmLayout(m).size() doubles
  cudaGraphExec_t gm_step = nullptr;
  long long gm_step_kernels = 0;
  // one restart cycle as one graph: WHILE (cond) { Arnoldi step; check }
  cudaGraphExec_t gm_cycle = nullptr;
  bool gm_cycle_failed = false;
};

// blocks of the GMRES vector kernels (fixed: the dot partials are summed in a fixed order)
constexpr int kGmBlocks = 4 * 152;

// Offsets of the Arnoldi state of GMRES(m) in DeviceState::gm_st.
struct GmLayout {
  int m;
  __host__ __device__ int h() const { return 0; }                // [m+1] projection coefficients of step j
  __host__ __device__ int h2() const { return m + 1; }           // [m+1] second (re-orthogonalisation) pass
  __host__ __device__ int R() const { return 2 * (m + 1); }      // [m][m] rotated Hessenberg, column-major
  __host__ __device__ int cs() const { return R() + m * m; }     // [m] plane rotations
  __host__ __device__ int sn() const { return cs() + m; }
  __host__ __device__ int g() const { return sn() + m; }         // [m+1] rotated ||r0|| e1
  __host__ __device__ int y() const { return g() + m + 1; }      // [m] least-squares solution
  __host__ __device__ int misc() const { return y() + m; }       // see GmMisc
  __host__ __device__ int size() const { return misc() + 8; }
};
enum GmMisc { GM_WN0 = 0, GM_WN1, GM_HNEXT, GM_REORTH, GM_J };

// Autotuning helper: average time in ms of `reps` calls of fn on stream s,
// after one untimed call.
template <typename F>
float time_calls(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps, F&& fn) {
  fn();
  cudaEventRecord(e0, s);
  for (int k = 0; k < reps; ++k) fn();
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / reps;
}

// launch counter shared by all translation units
void count_launch(long long n = 1);
long long launch_count();

// device.cu, for the GMRES driver: one V-cycle z = M^{-1} r on level-0 vectors;
// y = A_0 x (mode 0) or y = b - A_0 x (mode 1) on 256-byte aligned tree-order
// vectors; a level-0 dot into the CG scalars (dot_to's `which`); CUDA error text
int dev_precond(cdg_handle* h, const double* r, double* z, cudaStream_t s);
int dev_apply0(cdg_handle* h, int mode, const double* x, const double* b, double* y, cudaStream_t s);
int dev_dot(cdg_handle* h, const double* x, const double* y, int which, cudaStream_t s);
int dev_cuda_fail(cdg_handle* h, cudaError_t e, const char* where);

// device_gmres.cu: the GMRES iteration of cdg_solve from x, r = b - A x and the
// scalars S_BB, S_RR, S_DONE already on the device (single segment)
int gmres_run(cdg_handle* h, cudaStream_t s, double* res_hist, int* iters);
void gmres_release(DeviceState& D);


// device_multi.cu
namespace cdg { struct Hierarchy; }
MR* mr_new();
void mr_delete(MR* m);
// tc_fp64: the FP64 level-0 apply of the outer CG on tcgen05 by exact splitting (device_ozaki.cu)
size_t mr_layout(const cdg::Hierarchy& H, int R, int precision, int tc_fp64, MR* mr, char* base, size_t off);
void mr_upload(const cdg::Hierarchy& H, MR& M, cudaStream_t s);
int dev_apply_multi(cdg_handle* h, const double* x, double* y, void* stream);

// device_persist.cu: one V-cycle as one cooperative persistent launch (false: not applicable
// to this hierarchy, or the launch was refused)
bool vcycle_persistent(DeviceState& D, const cdg_options& o, bool fp32, const void* b0, void* z0, unsigned* count,
                       int* err, cudaStream_t s);

// device_ozaki.cu
namespace cdg { struct BSR; }
size_t oz_image_bytes(const cdg::BSR& A);
size_t oz_xslice_bytes(int64_t n, int np, int R);
bool oz_feasible(const cdg::BSR& A, int np);
bool oz_prepare(const cdg::BSR& A, int np, std::vector<uint16_t>& img, std::vector<int32_t>& eA);
// y = A_0 x by exact splitting; maxb [R] receives the largest biased FP64
// exponent of every column of x, unless maxb_ready says the caller already
// stored it there (the CG's p update does).  pq_partial (nullable): per-CTA
// partial sums of x . y per column, [*pq_groups][R], for the CG's p . A p.
bool oz_apply(int np, int n, int R, const int* rowptr, const int* col, const void* img, const int* eA, void* xs,
              int* maxb, bool maxb_ready, const double* x, double* y, double* pq_partial, int* pq_groups, int* err,
              int wait_limit, cudaStream_t s);
void mr_tuning(const MR& M, int level, int nlev, int32_t* out);

// device_tc.cu: multi-right-hand-side smoother sweep y = x + omega (bh - x - Ahat x) on
// tcgen05 tensor cores, Ahat BF16 [nnzb][np][np], vectors [n][np][R]; err set on a wait timeout
// wait_limit: iteration limit of the waits inside the loop (< 0: the default)
bool mr_tc_smooth(int np, int n, int R, const int* rowptr, const int* col, const void* Ahat_bf16, const float* x,
                  const float* bh, float* y, float omega, int* err, int wait_limit, cudaStream_t s);
