/*
 * cdg.h -- C ABI of the GB300 agglomeration h-multigrid solver for Compact
 * Discontinuous Galerkin (CDG) discretisations of Poisson's equation
 * (Pan & Persson, "Agglomeration-Based Geometric Multigrid Solvers for Compact
 * Discontinuous Galerkin Discretizations on Unstructured Meshes").
 *
 * Problem (Section 2.1, eq. poisson, sign as in the symmetric positive definite
 * form): -div(kappa grad u) = f in Omega, u = g_D on Gamma_D, kappa du/dn = g_N
 * on Gamma_N, |Gamma_D| > 0, kappa = 1 unless given.  Discretisation: CDG with
 * switch function S (Section 2.2) and penalty C_D = gamma / h_avg, primal form
 * A u = b (Section 2.3, eq. primal_form).  Solver: CG preconditioned by one
 * V(nu_pre, nu_post) cycle of damped block Jacobi (alpha = omega, Section 4.3)
 * over the greedy agglomeration hierarchy (Section 3.2, Algorithm 2) with
 * flux-coarsened operators (Section 4.1).
 *
 * Conventions
 *  - Every function returns CDG_OK (0) or one of the error codes below; the
 *    message of the last failure of a handle is cdg_last_error(handle), that of
 *    a failed cdg_create is cdg_last_error(NULL) (per thread).  No C++
 *    exception leaves an entry point: a failed host allocation returns
 *    CDG_ENOMEM (a cdg_bind_device that fails that way leaves the handle
 *    unbound).
 *  - The caller owns every array it passes; the library copies what it keeps.
 *    A handle owns its host-side hierarchy; its device data lives inside ONE
 *    caller-allocated device buffer given to cdg_bind_device (the library
 *    performs no device allocation of its own), which the caller keeps alive
 *    until cdg_destroy.
 *  - DG coefficient vectors are element-major [element][n_p], coefficients of
 *    the orthonormalised scaled-monomial basis of each element (R2: monomials
 *    of degree <= p in (x - c)/h, graded order, orthonormalised by Cholesky).
 *    In this basis the coefficient 2-norm is the L2 norm.
 *  - "User order" is the caller's element order; "tree order" numbers every
 *    level so that the children of each agglomerate are contiguous
 *    (cdg_export_level gives the permutation).  Per-level entry points use
 *    tree order; cdg_solve / cdg_rhs use user order.
 *  - Device entry points take device pointers and a cudaStream_t passed as
 *    void* (NULL = legacy default stream) and are asynchronous unless stated.
 */
#ifndef CDG_H_
#define CDG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CDG_OK 0
#define CDG_EINVAL 1      /* null pointer, bad size or option */
#define CDG_EMESH 2       /* degenerate element, non-manifold face, no Dirichlet boundary */
#define CDG_ENOCONV 3     /* maxit reached; outputs are still written */
#define CDG_EBREAKDOWN 4  /* p^T A p <= 0 in CG, a singular GMRES Hessenberg, or a non-finite residual */
#define CDG_ECUDA 5       /* a CUDA runtime call failed */
#define CDG_ETIMEOUT 6    /* a bounded device wait expired */
#define CDG_ENOMEM 7      /* host allocation failed or device buffer too small */
#define CDG_ESTATE 8      /* call out of order (e.g. solve before cdg_bind_device) */

typedef struct cdg_handle cdg_handle;

/* Mesh of simplices (Section 2.2: meshes T_h = {K}).  Boundary faces missing
 * from bface are Dirichlet.  Element orientation is free.  cdg_create returns
 * CDG_EINVAL for a vertex id out of range, a btag other than 0 or 1, and a
 * bface entry that is not a boundary face of the mesh or is listed twice. */
typedef struct {
  int32_t dim;              /* 2 (triangles) or 3 (tetrahedra) */
  int64_t n_vertices;
  const double* xyz;        /* [n_vertices][dim] */
  int64_t n_elements;
  const int64_t* elem;      /* [n_elements][dim+1] vertex ids */
  int64_t n_bfaces;         /* may be 0 */
  const int64_t* bface;     /* [n_bfaces][dim] vertex ids */
  const int32_t* btag;      /* [n_bfaces] 0 = Dirichlet, 1 = Neumann */
} cdg_mesh;

typedef struct {
  int32_t p;                /* polynomial degree: 1..6 on triangles, 1..3 on tetrahedra
                               (n_p = C(p+d, d)) */
  double gamma;             /* C_D = gamma / h_avg (Section 2.2), default 1e4 */
  int32_t nu_pre, nu_post;  /* smoothing steps; equal values give a symmetric V-cycle */
  double omega;             /* block-Jacobi damping, default 2/3 (Section 4.3) */
  int32_t max_levels;       /* levels including level 0 (Algorithm 1 stops earlier at 1 element) */
  uint64_t seed;            /* tie-break seed of Algorithm 2 */
  int32_t precision;        /* 0: FP64 V-cycle; 1: FP32 V-cycle inside FP64 CG;
                               2: for cdg_solve_multi, BF16 row-scaled smoother blocks and
                                  transfer blocks (FP32 residual operator, block inverses
                                  and arithmetic) */
  int32_t switch_kind;      /* 0: directional consistent switch, 1: natural switch (Section 2.2) */
  const int8_t* face_switch;   /* nullable: S_{K1}^{K2} = +1 or -1 per interior face (library face order) */
  const int64_t* enumeration;  /* nullable: element enumeration N(K) of the natural switch, distinct values */
  const double* kappa;         /* nullable: per-element diffusion coefficient (user order) */
  int32_t coarsen;          /* 0: flux coarsening (Section 4.1), 1: primal A_{l+1} = R A_l L */
  double tol;               /* relative residual ||r||/||b|| to stop CG, default 1e-10 */
  int32_t maxit;            /* CG iteration limit, default 500 */
  int32_t nrhs;             /* columns of cdg_solve_multi (0 = none), at most 1024; needs
                               n_p = 3, 4, 6 or 10 (2D p <= 3, 3D p <= 2) */
  int32_t krylov;           /* outer Krylov method of cdg_solve: 0 CG (A_0 is SPD; needs a
                               symmetric V-cycle, nu_pre = nu_post), 1 restarted GMRES with
                               the V-cycle as right preconditioner (Section 4; flexible form,
                               single-mesh handles only) */
  int32_t restart;          /* GMRES restart length m in [1, 512], default 50 (Section 5) */
  int32_t pmg;              /* 1: p-multigrid front end (Section 4.4): the levels of degree p,
                               p-1, ..., 2 on the fine mesh (CDG rediscretised at each degree,
                               truncation transfers) come before the agglomeration hierarchy,
                               built at p = 1 with max_levels levels; not with nrhs or batched
                               handles.  Default 0. */
  int32_t autotune;         /* 1 (default): cdg_bind_device times the block-sparse kernel's
                               variants (blocks in flight per step) on every level and keeps
                               the fastest, and the first cdg_solve_multi does the same for the
                               right-hand-side tile width and block rows per CTA; 0: fixed
                               defaults.  Results are bit-identical either way. */
  double beta;              /* convection-diffusion (Section 5): solve -div(kappa grad u) +
                               beta v . grad u = f, convection in upwind DG form, constant v;
                               A_0 is then non-symmetric: needs krylov = 1, nrhs = 0, no
                               batched handle, no adjoint.  Default 0 (Poisson). */
  double velocity[3];       /* v (first dim entries used) */
  int32_t solve_graph;      /* 1 (default): cdg_solve runs the whole CG loop (GMRES: each restart
                               cycle) as one CUDA graph launch with a conditional WHILE node;
                               0: host-driven loop, graphs per iteration half (per Arnoldi step),
                               one host read each.  Same kernels, same order, bit-identical
                               results; 0 is the form that kernel profilers list launch by launch */
  int32_t tensor_cores;     /* 1 (default): with precision 2, cdg_solve_multi runs the V-cycle's
                               smoother sweeps on the tcgen05 tensor cores (BF16 blocks exact in
                               TF32, x split into two TF32 parts: FP32 accuracy); 0: CUDA cores.
                               A wait that reaches its limit returns CDG_ETIMEOUT. */
  int32_t fuse_transfers;   /* bit 0: between two agglomeration levels the V-cycle computes the
                               residual, its restriction (Section 3.4) and the coarse level's
                               first smoothing step in one kernel; bit 1: the coarse level's
                               last post-smoothing sweep carries the prolongation.  0 (default):
                               separate kernels, measured faster on GB300.  The same arithmetic
                               up to summation order. */
  int32_t tc_fp64_apply;    /* 1: with nrhs, the FP64 level-0 apply of the outer CG runs on the
                               tcgen05 tensor cores by exact splitting (rows of A_0 and columns
                               of x scaled by powers of two and cut into eight 7-bit slices,
                               BF16 slice products summed exactly in FP32 per diagonal,
                               combined in integers and rounded once to FP64; Ozaki et al.
                               2012); relative truncation below 2^-56 of the row and column
                               scales.  Used where the FP32 sums provably stay exact (blocks per
                               row x n_p x 8 x 127^2 < 2^23), else the FP64 CUDA-core apply.
                               0 (default): the FP64 CUDA-core apply. */
  int32_t persistent_vcycle; /* 1: each V-cycle is ONE cooperative persistent kernel whose CTAs
                               walk the cycle's phases with grid barriers (bounded waits; an
                               expired wait ends the solve with CDG_ETIMEOUT); used when every
                               level has the same n_p (no p-multigrid degree steps), else the
                               per-phase kernels.  0 (default): one kernel per phase. */
} cdg_options;

#define CDG_MAX_LEVELS 16

typedef struct {
  int32_t dim, p, n_p, n_levels;
  int32_t nq;               /* volume quadrature points per element */
  int32_t nfq;              /* quadrature points per face */
  int64_t n_elements, n_interior_faces, n_bfaces, n_dofs;
  int64_t n_l[CDG_MAX_LEVELS];      /* elements per level */
  int64_t nnzb_l[CDG_MAX_LEVELS];   /* stored n_p x n_p blocks of A_l */
  double h_avg, C_D;
  int64_t device_bytes;     /* size of the buffer cdg_bind_device needs */
  double setup_seconds[4];  /* mesh, level-0 assembly, agglomeration, coarsening */
  int32_t n_meshes;         /* 1, or the number of meshes of a batched handle */
  int32_t np_l[CDG_MAX_LEVELS];   /* basis functions per element on each level */
  int32_t n_plevels;        /* p-multigrid: levels of degree p..2 on the fine mesh (0 without) */
  int32_t solve_graph;      /* 1 once a CG solve (or a GMRES restart cycle) has run as a single CUDA
                               graph launch (a conditional WHILE node around one iteration or
                               Arnoldi step; convergence and residual histories decided on the
                               device), 0 before the first solve or when the driver refused that
                               graph (then graphs per iteration or step, host-driven) */
} cdg_info;

/* Defaults: p=2, gamma=1e4, V(1,1), omega=2/3, 4 levels, seed 0, FP64,
 * directional switch, flux coarsening, tol=1e-10, maxit=500, CG (restart 50
 * when GMRES is selected). */
void cdg_default_options(cdg_options* opt);

/* Host set-up (Sections 2-4.1): faces, switch, quadrature, bases, level-0 CDG
 * operator, Algorithm 2 hierarchy, transfers, flux-coarsened operators, block
 * inverses and the dense inverse of the coarsest operator.  Copies all inputs.
 * Errors: CDG_EINVAL, CDG_EMESH, CDG_ENOMEM. */
int cdg_create(const cdg_mesh* mesh, const cdg_options* opt, cdg_handle** out);
void cdg_destroy(cdg_handle* h);

/* Batched handle: n_meshes independent meshes (same dim, p and options, and
 * the same number of hierarchy levels) set up separately and solved together.
 * Every level is the block-diagonal union of the meshes' levels, so each kernel
 * of the solve phase processes all meshes in one launch; the CG keeps separate
 * scalars and convergence per mesh (a converged mesh stops changing).  Arrays
 * of a batched handle concatenate the meshes in order (elements, boundary
 * faces, dofs; offsets from cdg_batch_offsets); cdg_solve then writes
 * res_hist[n_meshes][maxit+1] and iters[n_meshes].  kappa, face_switch and
 * enumeration must be NULL.  The paper solves one mesh at a time; batching is
 * an execution choice of this library. */
int cdg_create_batched(const cdg_mesh* meshes, int32_t n_meshes, const cdg_options* opt, cdg_handle** out);
/* n_meshes, elem_offsets [n_meshes+1] and bface_offsets [n_meshes+1] (any may be NULL). */
int cdg_batch_offsets(const cdg_handle* h, int32_t* n_meshes, int64_t* elem_offsets, int64_t* bface_offsets);
const char* cdg_last_error(const cdg_handle* h);
int cdg_query(const cdg_handle* h, cdg_info* info);
/* Launch configuration chosen by the autotuner for one level (no counterpart in
 * the paper; an execution detail of this library).  out[13]: [0] FP64 level-0
 * apply and [1] FP64 level-0 residual (level 0 only), [2] V-cycle residual and
 * [3] V-cycle smoother sweep (V-cycle precision): blocks in flight per step of
 * the vector-load kernel; multi-right-hand-side kernels as (threads across
 * the right-hand sides, block rows per CTA): [4,5] smoother sweep, [6,7]
 * residual, [8,9] FP64 level-0 apply (level 0 only), and their right-hand
 * sides per thread: [10] smoother sweep, [11] residual, [12] FP64 level-0
 * apply.  0 = not applicable or not tuned yet.  Errors: CDG_EINVAL (bad level
 * or NULL), CDG_ESTATE (not bound). */
int cdg_tuning(const cdg_handle* h, int32_t level, int32_t* out);

/* Quadrature points at which the caller samples f, g_D and g_N (R3: collapsed
 * Gauss-Legendre rules of degree 2p): xq [n_elements][nq][dim] in user order,
 * xbq [n_bfaces][nfq][dim] in library boundary-face order (sorted by element,
 * then local face), btag [n_bfaces].  Any pointer may be NULL. */
int cdg_quadrature_points(const cdg_handle* h, double* xq, double* xbq, int32_t* btag);

/* Host copies of the set-up, for inspection and tests (any pointer may be
 * NULL).  perm [n_l]: tree position -> working index (level 0: user element);
 * parent [n_l] (tree order, -1 on the coarsest level); A_l in tree order as
 * BSR: rowptr [n_l+1], col [nnzb_l], val [nnzb_l][n_p(l)][n_p(l)] row-major
 * blocks; transfer blocks L [n_l][n_p(l)][n_p(l+1)] with
 * L_K = int_K phi_K psi_parent^T (between two degrees of a p-multigrid
 * hierarchy: the truncation [I; 0]).  n_p(l) is cdg_info.np_l[l]. */
int cdg_export_level(const cdg_handle* h, int32_t level, int64_t* perm, int32_t* parent,
                     int64_t* rowptr, int32_t* col, double* val, double* L);
/* Agglomeration of one level in working numbering (Algorithm 2 output):
 * parent [n_l] = index of the agglomerate on level l+1 in creation order. */
int cdg_export_agglomeration(const cdg_handle* h, int32_t level, int64_t* parent);

/* Changes the V-cycle precision of a handle (cdg_options.precision: 0, 1, or 2
 * for a handle with nrhs) without repeating the host set-up, which does not
 * depend on it (the paper fixes no precision; this is an execution option of
 * the library).  Releases the device binding: query cdg_info.device_bytes again
 * and call cdg_bind_device before the next device call.  Errors: CDG_EINVAL
 * (bad value, NULL handle). */
int cdg_set_precision(cdg_handle* h, int32_t precision);

/* Device binding: copies the hierarchy into dev_buffer (>= info.device_bytes
 * bytes, 256-byte aligned) on stream and synchronises it.  Errors: CDG_ENOMEM
 * (buffer too small), CDG_ECUDA. */
int cdg_bind_device(cdg_handle* h, void* dev_buffer, int64_t bytes, void* stream);

/* Right-hand side b (user order, [n_elements][n_p]) from f at the volume
 * points [n_elements][nq] and g_D, g_N at the boundary points
 * [n_bfaces][nfq] (NULL = zero), all device pointers:
 * b = int f v + int_{Gamma_D} kappa g_D (-dv/dn + C_D v) + int_{Gamma_N} g_N v. */
int cdg_rhs(cdg_handle* h, const double* f_q, const double* gD_q, const double* gN_q, double* b,
            void* stream);

/* Full solve (Section 4, Section 5 set-up): b from (f, g_D, g_N), then CG
 * preconditioned by one V-cycle per iteration from u0 (u holds u0 on entry
 * when use_u0 != 0, else u0 = 0) until ||r||/||b|| <= tol or maxit.  Writes u
 * (user order), res_hist[0..iters] (relative recurrence residuals, array of
 * maxit+1 entries) and *iters.  host_pointers != 0: f_q, gD_q, gN_q, u and
 * res_hist are host arrays (copied in and out inside the call); else device
 * arrays (res_hist may then be a host array too: it is always written from
 * the host).  The solve runs on a private stream of the handle, ordered after
 * the work already queued on `stream`; it returns when the solution is written.
 * With krylov = 1 the outer method is restarted GMRES(restart) with the V-cycle
 * as right preconditioner (Section 4), in the flexible form that stores the
 * preconditioned vectors; iterations count Arnoldi steps, res_hist[k] is the
 * least-squares residual estimate |g_{k+1}|/||b|| (the true residual after a
 * restart or at the end), and a happy breakdown ends the solve as converged.
 * Errors: CDG_ESTATE, CDG_ENOCONV, CDG_EBREAKDOWN (CG: p^T A p <= 0; GMRES: a
 * singular Hessenberg column; both: a non-finite residual), CDG_ECUDA. */
int cdg_solve(cdg_handle* h, const double* f_q, const double* gD_q, const double* gN_q, double* u,
              int32_t use_u0, double* res_hist, int32_t* iters, int32_t host_pointers, void* stream);

/* Many right-hand sides on one mesh (handle created with nrhs = R > 0; not for
 * batched handles): solves A_0 u_r = b(f_r) for r < R in one CG with per-column
 * scalars.  f_q [R][n_elements][nq] device (zero boundary data), u
 * [R][n_elements][n_p] device, res_hist [R][maxit+1] and iters [R] host.
 * Vectors are stored [element][n_p][R] on the device so every operator block
 * is read once per R columns; the V-cycle computes in FP32 on FP32 block copies
 * (precision 1) or on BF16 row-scaled smoother and transfer blocks with FP32
 * residual operator and block inverses (precision 2); the outer CG is FP64. */
int cdg_solve_multi(cdg_handle* h, const double* f_q, double* u, double* res_hist, int32_t* iters, void* stream);

/* y = A_0 x for the R columns of a handle created with nrhs = R (tree order,
 * [n_elements][n_p][R] FP64 device vectors), by the method cdg_solve_multi
 * uses (tc_fp64_apply or the FP64 CUDA-core apply); returns when y is
 * written.  Errors: CDG_ESTATE, CDG_ETIMEOUT (a tensor-core wait reached its
 * limit), CDG_ECUDA. */
int cdg_apply_multi(cdg_handle* h, const double* x, double* y, void* stream);

/* Same solve from a given load vector b (device, user order, [n_elements][n_p]). */
int cdg_solve_b(cdg_handle* h, const double* b, double* u, int32_t use_u0, double* res_hist,
                int32_t* iters, void* stream);

/* Adjoint (differentiation of the solve; the paper has no adjoint, it follows
 * from the primal form eq. primal_form, A_0(kappa) u = b(f, kappa)).  For a loss
 * L(u): lambda solves A_0^T lambda = dL/du; dL/df = (db/df)^T lambda and
 * dL/dkappa_K = lambda^T (db/dkappa_K - dA_0/dkappa_K u).  A_0 is symmetric, so
 * the adjoint solve is the same preconditioned CG.  All vectors device, user
 * order; these calls use the handle's CG work vectors (do not overlap them with
 * a solve on another stream). */
/* lambda [n_elements][n_p] from dLdu [n_elements][n_p]; as cdg_solve_b. */
int cdg_solve_adjoint(cdg_handle* h, const double* dLdu, double* lambda, double* res_hist, int32_t* iters,
                      void* stream);
/* dLdf_q [n_elements][nq]: sum_i w_q phi_i(x_q) lambda_K[i]. */
int cdg_rhs_adjoint(cdg_handle* h, const double* lambda, double* dLdf_q, void* stream);
/* dLdkappa [n_elements]: each term of A_0 and b is owned by one element and is
 * linear in its kappa (R7: volume term by its element, interior face by its
 * q-side, Dirichlet face by its element); gD_q as in cdg_rhs (NULL = 0). */
int cdg_kappa_gradient(cdg_handle* h, const double* lambda, const double* u, const double* gD_q, double* dLdkappa,
                       void* stream);

/* Per-level operations (device pointers, tree order, FP64): */
/* y = A_l x  (block-sparse apply, eq. primal_form and Section 4.1) */
int cdg_apply(cdg_handle* h, int32_t level, const double* x, double* y, void* stream);
/* y = A_l x with the FP32 copy of A_l that the FP32 V-cycle uses (precision 1 or 2
 * handles, levels below the coarsest); FP32 vectors.  CDG_EINVAL elsewhere. */
int cdg_apply_f32(cdg_handle* h, int32_t level, const float* x, float* y, void* stream);
/* y = b - A_l x */
int cdg_residual(cdg_handle* h, int32_t level, const double* x, const double* b, double* y,
                 void* stream);
/* y = x + omega D_l^{-1} (b - A_l x)  (damped block Jacobi, Section 4.3; y != x) */
int cdg_smooth(cdg_handle* h, int32_t level, const double* x, const double* b, double* y,
               void* stream);
/* bc = R r = sum over children K of L_K^T r_K  (level -> level+1, Section 3.4) */
int cdg_restrict(cdg_handle* h, int32_t level, const double* r, double* bc, void* stream);
/* x += L xc  (level+1 -> level injection, Section 3.4) */
int cdg_prolong(cdg_handle* h, int32_t level, const double* xc, double* x, void* stream);
/* x = A_n^{-1} b on the coarsest level (direct solve, Section 4.3): the dense
 * inverse times b, followed in an FP64 handle (precision 0) by one step of
 * iterative refinement x += A_n^{-1} (b - A_n x) with the block-sparse A_n, so
 * the result is that of a backward-stable solve (within cond(A_n) eps of a
 * factorisation-based one).  b and x must not alias. */
int cdg_coarse_solve(cdg_handle* h, const double* b, double* x, void* stream);
/* z = V(r): one V(nu_pre, nu_post) cycle on level 0 from a zero guess (R14),
 * in the handle's precision; r, z FP64 tree order. */
int cdg_vcycle(cdg_handle* h, const double* r, double* z, void* stream);
/* Permutations between user and tree order of level 0 (device). */
int cdg_to_tree(cdg_handle* h, const double* user, double* tree, void* stream);
int cdg_to_user(cdg_handle* h, const double* tree, double* user, void* stream);

/* Allocation-free variant of cdg_smooth (no counterpart in the paper: it exists
 * for callers that cannot allocate device memory at the point of the call --
 * code running while a memory pool is frozen or exhausted, or inside a host
 * callback -- and therefore cannot provide scratch space of their own).
 * Same result as cdg_smooth: y = x + omega D_l^{-1} (b - A_l x), device
 * pointers, tree order, FP64 handle.  The intermediate D_l^{-1} b is kept in
 * a fixed device array inside the library (CDG_STATIC_SCRATCH doubles = 8 MiB,
 * held by every GPU that loads the library until the process exits) instead of
 * the handle's buffer; levels with n_l * n_p > CDG_STATIC_SCRATCH are rejected
 * with CDG_EINVAL, and so is the coarsest level.  The first call on a device
 * looks up the array's device address with that device current, and so does
 * the first call after the current context changed (cudaDeviceReset, another
 * context made current); make those calls before any stream capture.  All calls share the one array: calls that overlap on the GPU (on
 * different streams, or from different threads) race and must be serialised
 * by the caller.  No device or host memory is allocated by this call. */
#define CDG_STATIC_SCRATCH (1 << 20)
int cdg_smooth_static(cdg_handle* h, int32_t level, const double* x, const double* b, double* y,
                      void* stream);

/* Failure injection for tests of the bounded device waits (no counterpart in
 * the paper).  Sets the iteration limit of the waits inside kernel loops of
 * this bound handle: the tcgen05 smoother sweep of cdg_solve_multi (precision
 * 2 with tensor_cores), the tcgen05 FP64 apply (tc_fp64_apply) and the grid
 * barriers of the persistent V-cycle (persistent_vcycle).  limit = 0 makes the first such wait give up at once;
 * the kernel then sets its error flag, waits (with its default limit) for the
 * tensor-core work it already issued, frees its tensor memory and returns, and
 * the solve returns CDG_ETIMEOUT.  limit < 0 restores the defaults.  Nothing
 * faults or hangs the GPU.  Holds until the next cdg_bind_device; a change
 * drops the handle's captured solve graphs (the next solve captures them
 * again).  Errors:
 * CDG_EINVAL (NULL handle), CDG_ESTATE (not bound). */
int cdg_set_wait_limit(cdg_handle* h, int32_t limit);

/* FP64 FMA throughput probe (no counterpart in the paper: it measures the
 * arithmetic bound of the FP64 block-sparse kernels on the device at hand).
 * Launches blocks x 256 threads, each running 16 independent FMA chains of
 * ceil(iters / 2) steps: blocks * 256 * 16 * ceil(iters / 2) FMAs in total.  The caller times the
 * launch on `stream` (e.g. with CUDA events) and divides.  sink: device pointer
 * to one double that the kernel writes only for inputs that never occur (keeps
 * the chains live).  Errors: CDG_EINVAL (blocks or iters < 1, NULL sink),
 * CDG_ECUDA. */
int cdg_fp64_fma_probe(int32_t blocks, int64_t iters, double* sink, void* stream);

/* Element-wise conversion of a device vector between binary64 and binary32
 * (no counterpart in the paper: the conversion the mixed-precision solves
 * apply at the edges of their FP32 V-cycle, Section 4.3 being run in two
 * precisions).  to_fp32 = 1: in is n doubles, out n floats, rounded to
 * nearest with ties to even; to_fp32 = 0: in is n floats, out n doubles
 * (exact).  The kernels build the results from the IEEE 754 bit fields with
 * integer operations; results equal the IEEE conversions for every input
 * (NaN payloads aside).  Asynchronous on `stream`.  Errors: CDG_EINVAL (NULL
 * pointer with n > 0, n < 0), CDG_ECUDA. */
int cdg_convert(const void* in, void* out, int64_t n, int32_t to_fp32, void* stream);

/* Number of CUDA kernels this library has launched in the process so far
 * (instrumentation for benchmarks; thread-safe, never reset). */
int64_t cdg_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* CDG_H_ */
