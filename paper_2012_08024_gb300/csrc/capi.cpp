// C ABI entry points (include/cdg.h): host set-up, queries and exports; the
// device entry points forward to device.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <vector>

#include "handle.h"

namespace {
thread_local std::string g_create_error;

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int fail(cdg_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

// No C++ exception crosses the C ABI: a host allocation that fails inside an
// entry point (staging vectors, graph bookkeeping) returns CDG_ENOMEM, anything
// else thrown returns CDG_EINVAL with its message.
int fail_quiet(cdg_handle* h, int code, const char* msg) noexcept {
  try {
    fail(h, code, msg);
  } catch (...) {
  }
  return code;
}

template <typename F>
int nothrow(cdg_handle* h, F&& f) noexcept {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fail_quiet(h, CDG_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail_quiet(h, CDG_EINVAL, e.what());
  } catch (...) {
    return fail_quiet(h, CDG_EINVAL, "unexpected exception");
  }
}
}  // namespace

static int check_options(const cdg_options* opt) {
  if (opt->p < 1 || opt->p > 6) return fail(nullptr, CDG_EINVAL, "p must be in [1, 6]");
  if (opt->max_levels < 1 || opt->max_levels > CDG_MAX_LEVELS)
    return fail(nullptr, CDG_EINVAL, "max_levels must be in [1, 16]");
  if (opt->nu_pre < 0 || opt->nu_post < 0 || opt->nu_pre + opt->nu_post < 1)
    return fail(nullptr, CDG_EINVAL, "need nu_pre, nu_post >= 0 and at least one smoothing step");
  if (!(opt->omega > 0) || !(opt->gamma > 0) || opt->maxit < 0 || !(opt->tol >= 0) || !std::isfinite(opt->omega) ||
      !std::isfinite(opt->gamma) || !std::isfinite(opt->tol))
    return fail(nullptr, CDG_EINVAL, "bad omega, gamma, tol or maxit");
  for (int32_t flag : {opt->switch_kind, opt->coarsen, opt->autotune, opt->solve_graph, opt->tensor_cores})
    if (flag != 0 && flag != 1)
      return fail(nullptr, CDG_EINVAL, "switch_kind, coarsen, autotune, solve_graph and tensor_cores are 0 or 1");
  if (opt->fuse_transfers < 0 || opt->fuse_transfers > 3)
    return fail(nullptr, CDG_EINVAL, "fuse_transfers must be in [0, 3]");
  if (opt->tc_fp64_apply != 0 && opt->tc_fp64_apply != 1)
    return fail(nullptr, CDG_EINVAL, "tc_fp64_apply is 0 or 1");
  if (opt->persistent_vcycle != 0 && opt->persistent_vcycle != 1)
    return fail(nullptr, CDG_EINVAL, "persistent_vcycle is 0 or 1");
  if (opt->precision < 0 || opt->precision > 2) return fail(nullptr, CDG_EINVAL, "precision must be 0, 1 or 2");
  if (opt->nrhs < 0 || opt->nrhs > 1024) return fail(nullptr, CDG_EINVAL, "nrhs must be in [0, 1024]");
  if (opt->precision == 2 && opt->nrhs == 0)
    return fail(nullptr, CDG_EINVAL, "precision 2 (BF16 blocks) is the multi-right-hand-side mode: set nrhs");
  if (opt->krylov < 0 || opt->krylov > 1) return fail(nullptr, CDG_EINVAL, "krylov must be 0 (CG) or 1 (GMRES)");
  if (opt->krylov == 1 && (opt->restart < 1 || opt->restart > 512))
    return fail(nullptr, CDG_EINVAL, "GMRES restart must be in [1, 512]");
  if (opt->pmg < 0 || opt->pmg > 1) return fail(nullptr, CDG_EINVAL, "pmg must be 0 or 1");
  if (opt->pmg && opt->p > 1 && opt->max_levels + opt->p - 1 > CDG_MAX_LEVELS)
    return fail(nullptr, CDG_EINVAL, "p-multigrid: max_levels + p - 1 must be at most 16");
  if (opt->pmg && opt->p > 1 && opt->nrhs)
    return fail(nullptr, CDG_EINVAL, "p-multigrid is not available with nrhs (cdg_solve_multi)");
  if (!std::isfinite(opt->beta) || !std::isfinite(opt->velocity[0]) || !std::isfinite(opt->velocity[1]) ||
      !std::isfinite(opt->velocity[2]))
    return fail(nullptr, CDG_EINVAL, "beta and velocity must be finite");
  if (opt->beta != 0.0 && opt->krylov != 1)
    return fail(nullptr, CDG_EINVAL, "convection makes A_0 non-symmetric: use GMRES (krylov = 1)");
  if (opt->beta != 0.0 && opt->nrhs)
    return fail(nullptr, CDG_EINVAL, "convection is not available with nrhs (cdg_solve_multi runs CG)");
  return CDG_OK;
}

static int check_mesh(const cdg_mesh* mesh) {
  if (mesh->dim != 2 && mesh->dim != 3) return fail(nullptr, CDG_EINVAL, "dim must be 2 or 3");
  if (mesh->n_elements <= 0 || mesh->n_vertices <= 0 || !mesh->xyz || !mesh->elem)
    return fail(nullptr, CDG_EINVAL, "empty mesh");
  if (mesh->n_bfaces < 0 || (mesh->n_bfaces > 0 && !mesh->bface))
    return fail(nullptr, CDG_EINVAL, "bad boundary face list");
  for (int64_t i = 0; i < mesh->n_vertices * mesh->dim; ++i)
    if (!std::isfinite(mesh->xyz[i])) return fail(nullptr, CDG_EINVAL, "vertex coordinates must be finite");
  return CDG_OK;
}

// Host set-up of one mesh (throws on bad input).  kappa / enumeration / switch
// are taken from opt only when use_arrays is set (single-mesh handles).
static void build_one(const cdg_mesh* mesh, const cdg_options* opt, bool use_arrays, cdg::Hierarchy& H) {
  cdg::Options& o = H.opt;
  o.p = opt->p;
  o.pmg = opt->pmg;
  o.beta = opt->beta;
  for (int c = 0; c < 3; ++c) o.vel[c] = opt->velocity[c];
  o.gamma = opt->gamma;
  o.nu_pre = opt->nu_pre;
  o.nu_post = opt->nu_post;
  o.omega = opt->omega;
  o.max_levels = opt->max_levels;
  o.seed = opt->seed;
  o.switch_kind = opt->switch_kind;
  o.coarsen = opt->coarsen;
  const int64_t ne = mesh->n_elements;
  if (use_arrays && opt->enumeration) {
    o.enumeration.assign(opt->enumeration, opt->enumeration + ne);
    std::vector<int64_t> e = o.enumeration;
    std::sort(e.begin(), e.end());
    if (std::adjacent_find(e.begin(), e.end()) != e.end())
      throw std::invalid_argument("the element enumeration must have distinct values");
  }
  if (use_arrays && opt->kappa) {
    o.kappa.assign(opt->kappa, opt->kappa + ne);
    for (double k : o.kappa)
      if (!(k > 0) || !std::isfinite(k)) throw std::invalid_argument("kappa must be positive and finite");
  }
  double t0 = now();
  cdg::build_mesh(mesh->dim, mesh->n_vertices, mesh->xyz, ne, mesh->elem, mesh->n_bfaces, mesh->bface,
                  mesh->btag, o, H.mesh);
  if (use_arrays && opt->face_switch) {
    const size_t nif = H.mesh.if_K1.size();
    o.face_switch.assign(opt->face_switch, opt->face_switch + nif);
    for (int8_t v : o.face_switch)
      if (v != 1 && v != -1) throw std::invalid_argument("face_switch entries must be +1 or -1");
    cdg::build_mesh(mesh->dim, mesh->n_vertices, mesh->xyz, ne, mesh->elem, mesh->n_bfaces, mesh->bface,
                    mesh->btag, o, H.mesh);
  }
  H.mono.init(mesh->dim, o.p);
  H.np = H.mono.np;
  // the device kernels hold one block row in at most one warp and are instantiated
  // for n_p = 3, 4, 6, 10, 15, 20, 21, 28: every 2D degree up to 6, 3D up to 3
  if (mesh->dim == 3 && o.p > 3) throw std::invalid_argument("tetrahedra support p <= 3 (n_p <= 20)");
  H.vrule = cdg::simplex_rule(mesh->dim, 2 * o.p);
  H.frule = cdg::simplex_rule(mesh->dim - 1, 2 * o.p);
  H.lev.assign(1, cdg::Level());
  double t1 = now();
  cdg::build_level0(H);
  double t2 = now();
  if (o.pmg && o.p > 1) {
    // p-multigrid (Section 4.4): the same discretisation at degrees p-1, ..., 2, then
    // the complete degree-1 hierarchy
    std::vector<cdg::Hierarchy> fine(o.p - 2);
    for (int q = o.p - 1; q >= 2; --q) {
      cdg::Hierarchy& F = fine[o.p - 1 - q];
      F.opt = o;
      F.opt.p = q;
      F.mesh = H.mesh;
      F.mono.init(mesh->dim, q);
      F.np = F.mono.np;
      F.vrule = cdg::simplex_rule(mesh->dim, 2 * q);
      F.frule = cdg::simplex_rule(mesh->dim - 1, 2 * q);
      F.lev.assign(1, cdg::Level());
      cdg::build_level0(F);
    }
    cdg_options o1 = *opt;
    o1.p = 1;
    o1.pmg = 0;
    cdg::Hierarchy H1;
    build_one(mesh, &o1, use_arrays, H1);
    double t3 = now();
    cdg::merge_pmg(H, fine, H1);
    cdg::build_rhs_data(H);
    double t4 = now();
    H.t_mesh = t1 - t0;
    H.t_assemble = t2 - t1 + (t3 - t2) - H1.t_agglomerate - H1.t_coarsen;
    H.t_agglomerate = H1.t_agglomerate;
    H.t_coarsen = H1.t_coarsen + (t4 - t3);
    return;
  }
  cdg::agglomerate(H);
  double t3 = now();
  cdg::coarsen(H);
  cdg::finalize_tree_order(H);
  cdg::build_rhs_data(H);
  double t4 = now();
  H.t_mesh = t1 - t0;
  H.t_assemble = t2 - t1;
  H.t_agglomerate = t3 - t2;
  H.t_coarsen = t4 - t3;
}

template <typename F>
static int guarded(cdg_handle* h, F&& f) {
  try {
    f();
  } catch (const std::invalid_argument& e) {
    delete h;
    return fail(nullptr, CDG_EINVAL, e.what());
  } catch (const std::domain_error& e) {
    delete h;
    return fail(nullptr, CDG_EMESH, e.what());
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(nullptr, CDG_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    delete h;
    return fail(nullptr, CDG_EMESH, e.what());
  }
  return CDG_OK;
}

static void quad_points(const cdg::Hierarchy& H, double* xq, double* xbq, int32_t* btag) {
  const cdg::Mesh0& m = H.mesh;
  const int d = m.d;
  if (xq) {
    const int nq = H.vrule.n();
    for (int64_t K = 0; K < m.ne; ++K) {
      const int64_t* ev = m.elem.data() + K * (d + 1);
      for (int q = 0; q < nq; ++q)
        for (int k = 0; k < d; ++k) {
          double s = m.xyz[ev[0] * d + k];
          for (int i = 0; i < d; ++i)
            s += H.vrule.x[(size_t)q * d + i] * (m.xyz[ev[i + 1] * d + k] - m.xyz[ev[0] * d + k]);
          xq[((size_t)K * nq + q) * d + k] = s;
        }
    }
  }
  const int nfq = H.frule.n();
  for (size_t b = 0; b < m.bf_K.size(); ++b) {
    if (btag) btag[b] = m.bf_tag[b];
    if (!xbq) continue;
    const double* xv = &m.bf_xv[b * d * d];
    for (int q = 0; q < nfq; ++q)
      for (int k = 0; k < d; ++k) {
        double s = xv[k];
        for (int i = 0; i < d - 1; ++i) s += H.frule.x[(size_t)q * (d - 1) + i] * (xv[(i + 1) * d + k] - xv[k]);
        xbq[((size_t)b * nfq + q) * d + k] = s;
      }
  }
}

extern "C" {

void cdg_default_options(cdg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->p = 2;
  o->gamma = 1e4;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->omega = 2.0 / 3.0;
  o->max_levels = 4;
  o->seed = 0;
  o->precision = 0;
  o->switch_kind = 0;
  o->coarsen = 0;
  o->tol = 1e-10;
  o->maxit = 500;
  o->krylov = 0;
  o->restart = 50;
  o->autotune = 1;
  o->tensor_cores = 1;
  o->solve_graph = 1;
  o->fuse_transfers = 0;
}

const char* cdg_last_error(const cdg_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

int cdg_create(const cdg_mesh* mesh, const cdg_options* opt, cdg_handle** out) {
  if (!out) return fail(nullptr, CDG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !opt) return fail(nullptr, CDG_EINVAL, "mesh or options NULL");
  int rc = check_options(opt);
  if (rc == CDG_OK) rc = check_mesh(mesh);
  if (rc != CDG_OK) return rc;
  cdg_handle* h = new (std::nothrow) cdg_handle();
  if (!h) return fail_quiet(nullptr, CDG_ENOMEM, "host allocation failed");
  h->opt = *opt;
  h->opt.face_switch = nullptr;
  h->opt.enumeration = nullptr;
  h->opt.kappa = nullptr;
  rc = guarded(h, [&] { build_one(mesh, opt, true, h->H); });
  if (rc != CDG_OK) return rc;
  // cdg_solve_multi is instantiated for the block sizes of 2D p <= 3 and 3D p <= 2
  const int np = h->H.np;
  if (opt->nrhs > 0 && np != 3 && np != 4 && np != 6 && np != 10) {
    delete h;
    return fail(nullptr, CDG_EINVAL, "nrhs > 0 (cdg_solve_multi) supports n_p = 3, 4, 6 or 10 (2D p <= 3, 3D p <= 2)");
  }
  *out = h;
  return CDG_OK;
}

int cdg_create_batched(const cdg_mesh* meshes, int32_t n_meshes, const cdg_options* opt, cdg_handle** out) {
  if (!out) return fail(nullptr, CDG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!meshes || !opt || n_meshes < 1) return fail(nullptr, CDG_EINVAL, "meshes, n_meshes or options invalid");
  if (opt->kappa || opt->face_switch || opt->enumeration || opt->nrhs)
    return fail(nullptr, CDG_EINVAL, "per-element arrays and nrhs are not supported for batched handles");
  if (opt->krylov != 0) return fail(nullptr, CDG_EINVAL, "batched handles solve with CG (krylov = 0)");
  if (opt->pmg != 0) return fail(nullptr, CDG_EINVAL, "p-multigrid is not available for batched handles");
  if (opt->beta != 0.0) return fail(nullptr, CDG_EINVAL, "convection is not available for batched handles");
  int rc = check_options(opt);
  for (int32_t m = 0; rc == CDG_OK && m < n_meshes; ++m) rc = check_mesh(&meshes[m]);
  if (rc != CDG_OK) return rc;
  cdg_handle* h = new (std::nothrow) cdg_handle();
  if (!h) return fail_quiet(nullptr, CDG_ENOMEM, "host allocation failed");
  h->opt = *opt;
  rc = guarded(h, [&] {
    std::vector<cdg::Hierarchy> subs(n_meshes);
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t m = 0; m < n_meshes; ++m) {
      try {
        build_one(&meshes[m], opt, false, subs[m]);
      } catch (...) {
        subs[m].lev.clear();   // reported below
      }
    }
    for (int32_t m = 0; m < n_meshes; ++m)
      if (subs[m].lev.empty()) build_one(&meshes[m], opt, false, subs[m]);   // rethrows with the message
    cdg::concat_hierarchies(subs, h->H);
  });
  if (rc != CDG_OK) return rc;
  *out = h;
  return CDG_OK;
}

int cdg_batch_offsets(const cdg_handle* h, int32_t* n_meshes, int64_t* elem_offsets, int64_t* bface_offsets) {
  if (!h) return CDG_EINVAL;
  const cdg::Hierarchy& H = h->H;
  const int32_t nseg = (int32_t)H.seg_rows[0].size() - 1;
  if (n_meshes) *n_meshes = nseg;
  if (elem_offsets) {
    if (H.subs.empty()) {
      elem_offsets[0] = 0;
      elem_offsets[1] = H.mesh.ne;
    } else {
      elem_offsets[0] = 0;
      for (int32_t m = 0; m < nseg; ++m) elem_offsets[m + 1] = elem_offsets[m] + H.subs[m].mesh.ne;
    }
  }
  if (bface_offsets)
    for (int32_t m = 0; m <= nseg; ++m) bface_offsets[m] = H.seg_bface[m];
  return CDG_OK;
}

void cdg_destroy(cdg_handle* h) {
  if (!h) return;
  dev_release(h);
  delete h;
}

int cdg_tuning(const cdg_handle* h, int32_t level, int32_t* out) {
  if (!h || !out) return CDG_EINVAL;
  if (!h->dev) {
    const_cast<cdg_handle*>(h)->err = "cdg_bind_device has not been called";
    return CDG_ESTATE;
  }
  if (level < 0 || level >= (int32_t)h->H.lev.size()) {
    const_cast<cdg_handle*>(h)->err = "level out of range";
    return CDG_EINVAL;
  }
  return nothrow(const_cast<cdg_handle*>(h), [&] { return dev_tuning(h, level, out); });
}

int cdg_query(const cdg_handle* h, cdg_info* info) {
  if (!h || !info) return CDG_EINVAL;
  const cdg::Hierarchy& H = h->H;
  std::memset(info, 0, sizeof(*info));
  info->dim = H.mesh.d;
  info->p = H.opt.p;
  info->n_p = H.np;
  info->n_levels = (int32_t)H.lev.size();
  info->nq = H.vrule.n();
  info->nfq = H.frule.n();
  info->n_elements = H.mesh.ne;
  info->n_interior_faces = (int64_t)H.mesh.if_K1.size();
  info->n_bfaces = (int64_t)H.mesh.bf_K.size();
  info->n_dofs = H.mesh.ne * H.np;
  for (size_t l = 0; l < H.lev.size(); ++l) {
    info->n_l[l] = H.lev[l].n;
    info->nnzb_l[l] = H.A_t[l].nnzb();
  }
  info->h_avg = H.mesh.h_avg;
  info->C_D = H.mesh.C_D;
  int64_t b = 0;
  dev_bytes(h, &b);
  info->device_bytes = b;
  info->setup_seconds[0] = H.t_mesh;
  info->setup_seconds[1] = H.t_assemble;
  info->setup_seconds[2] = H.t_agglomerate;
  info->setup_seconds[3] = H.t_coarsen;
  info->n_meshes = (int32_t)H.seg_rows[0].size() - 1;
  for (size_t l = 0; l < H.lev.size(); ++l) info->np_l[l] = H.np_l.empty() ? H.np : H.np_l[l];
  info->n_plevels = H.n_plevels;
  info->solve_graph = dev_solve_graph(h);
  return CDG_OK;
}

int cdg_quadrature_points(const cdg_handle* h, double* xq, double* xbq, int32_t* btag) {
  if (!h) return CDG_EINVAL;
  const cdg::Hierarchy& H = h->H;
  if (H.subs.empty()) {
    quad_points(H, xq, xbq, btag);
    return CDG_OK;
  }
  const int d = H.mesh.d, nq = H.vrule.n(), nfq = H.frule.n();
  size_t eo = 0, bo = 0;
  for (const cdg::Hierarchy& S : H.subs) {
    quad_points(S, xq ? xq + eo * nq * d : nullptr, xbq ? xbq + bo * nfq * d : nullptr, btag ? btag + bo : nullptr);
    eo += S.mesh.ne;
    bo += S.mesh.bf_K.size();
  }
  return CDG_OK;
}

int cdg_export_level(const cdg_handle* h, int32_t level, int64_t* perm, int32_t* parent, int64_t* rowptr,
                     int32_t* col, double* val, double* L) {
  if (!h) return CDG_EINVAL;
  const cdg::Hierarchy& H = h->H;
  if (level < 0 || level >= (int32_t)H.lev.size()) return CDG_EINVAL;
  const int64_t n = H.lev[level].n;
  const cdg::BSR& A = H.A_t[level];
  const bool last = level + 1 == (int32_t)H.lev.size();
  const int npf = H.np_l[level], npc = last ? npf : H.np_l[level + 1];
  const size_t nb2 = (size_t)npf * npc;
  if (perm) std::memcpy(perm, H.order[level].data(), sizeof(int64_t) * n);
  if (parent)
    for (int64_t k = 0; k < n; ++k) parent[k] = last ? -1 : H.parent_t[level][k];
  if (rowptr) std::memcpy(rowptr, A.rowptr.data(), sizeof(int64_t) * (n + 1));
  if (col) std::memcpy(col, A.col.data(), sizeof(int32_t) * A.col.size());
  if (val) std::memcpy(val, A.val.data(), sizeof(double) * A.val.size());
  if (L && !last) {
    if (H.L_t[level].empty()) {   // between two degrees: truncation of the nested bases
      std::memset(L, 0, sizeof(double) * n * nb2);
      for (int64_t k = 0; k < n; ++k)
        for (int i = 0; i < npc; ++i) L[k * nb2 + (size_t)i * npc + i] = 1.0;
    } else {
      std::memcpy(L, H.L_t[level].data(), sizeof(double) * n * nb2);
    }
  }
  return CDG_OK;
}

int cdg_export_agglomeration(const cdg_handle* h, int32_t level, int64_t* parent) {
  if (!h || !parent) return CDG_EINVAL;
  const cdg::Hierarchy& H = h->H;
  if (level < 0 || level + 1 >= (int32_t)H.lev.size() || H.lev[level].parent.empty()) return CDG_EINVAL;
  std::memcpy(parent, H.lev[level].parent.data(), sizeof(int64_t) * H.lev[level].n);
  return CDG_OK;
}

int cdg_bind_device(cdg_handle* h, void* buf, int64_t bytes, void* stream) {
  if (!h || !buf) return h ? fail(h, CDG_EINVAL, "buffer is NULL") : CDG_EINVAL;
  // an exception thrown part-way leaves no half-bound device state behind
  bool threw = true;
  const int rc = nothrow(h, [&] {
    const int r = dev_bind(h, buf, bytes, stream);
    threw = false;
    return r;
  });
  if (threw) dev_release(h);
  return rc;
}

int cdg_set_precision(cdg_handle* h, int32_t precision) {
  if (!h) return CDG_EINVAL;
  if (precision < 0 || precision > 2) return fail(h, CDG_EINVAL, "precision must be 0, 1 or 2");
  if (precision == 2 && h->opt.nrhs == 0)
    return fail(h, CDG_EINVAL, "precision 2 (BF16 blocks) is the multi-right-hand-side mode: set nrhs");
  return nothrow(h, [&] {
    dev_release(h);
    h->opt.precision = precision;
    return CDG_OK;
  });
}

int cdg_set_wait_limit(cdg_handle* h, int32_t limit) {
  if (!h) return CDG_EINVAL;
  return nothrow(h, [&] { return dev_set_wait_limit(h, limit); });
}

int cdg_fp64_fma_probe(int32_t blocks, int64_t iters, double* sink, void* stream) {
  if (blocks < 1 || iters < 1 || !sink) return CDG_EINVAL;
  return dev_fma_probe(blocks, iters, sink, stream);
}

int cdg_convert(const void* in, void* out, int64_t n, int32_t to_fp32, void* stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return CDG_EINVAL;
  return dev_convert(in, out, (long long)n, to_fp32 ? 1 : 0, stream);
}

int cdg_rhs(cdg_handle* h, const double* f_q, const double* gD, const double* gN, double* b, void* stream) {
  if (!h || !f_q || !b) return h ? fail(h, CDG_EINVAL, "NULL argument") : CDG_EINVAL;
  return nothrow(h, [&] { return dev_rhs(h, f_q, gD, gN, b, true, stream); });
}

int cdg_solve(cdg_handle* h, const double* f_q, const double* gD, const double* gN, double* u, int32_t use_u0,
              double* res_hist, int32_t* iters, int32_t host_pointers, void* stream) {
  if (!h || !f_q || !u) return h ? fail(h, CDG_EINVAL, "NULL argument") : CDG_EINVAL;
  return nothrow(h, [&] {
    std::vector<int> its(h->H.seg_rows.empty() ? 1 : h->H.seg_rows[0].size() - 1, 0);
    const int rc = dev_solve(h, f_q, gD, gN, nullptr, u, use_u0, res_hist, its.data(), host_pointers, stream);
    if (iters)
      for (size_t m = 0; m < its.size(); ++m) iters[m] = its[m];
    return rc;
  });
}

int cdg_solve_b(cdg_handle* h, const double* b, double* u, int32_t use_u0, double* res_hist, int32_t* iters,
                void* stream) {
  if (!h || !b || !u) return h ? fail(h, CDG_EINVAL, "NULL argument") : CDG_EINVAL;
  return nothrow(h, [&] {
    std::vector<int> its(h->H.seg_rows.empty() ? 1 : h->H.seg_rows[0].size() - 1, 0);
    const int rc = dev_solve(h, nullptr, nullptr, nullptr, b, u, use_u0, res_hist, its.data(), 0, stream);
    if (iters)
      for (size_t m = 0; m < its.size(); ++m) iters[m] = its[m];
    return rc;
  });
}

int cdg_apply(cdg_handle* h, int32_t level, const double* x, double* y, void* stream) {
  return nothrow(h, [&] { return dev_level_op(h, 0, level, x, nullptr, y, stream); });
}
int cdg_apply_f32(cdg_handle* h, int32_t level, const float* x, float* y, void* stream) {
  return nothrow(h, [&] { return dev_apply_f32(h, level, x, y, stream); });
}
int cdg_residual(cdg_handle* h, int32_t level, const double* x, const double* b, double* y, void* stream) {
  return nothrow(h, [&] { return dev_level_op(h, 1, level, x, b, y, stream); });
}
int cdg_smooth(cdg_handle* h, int32_t level, const double* x, const double* b, double* y, void* stream) {
  return nothrow(h, [&] { return dev_level_op(h, 2, level, x, b, y, stream); });
}
int cdg_restrict(cdg_handle* h, int32_t level, const double* r, double* bc, void* stream) {
  return nothrow(h, [&] { return dev_level_op(h, 3, level, r, nullptr, bc, stream); });
}
int cdg_prolong(cdg_handle* h, int32_t level, const double* xc, double* x, void* stream) {
  return nothrow(h, [&] { return dev_level_op(h, 4, level, xc, nullptr, x, stream); });
}
int cdg_coarse_solve(cdg_handle* h, const double* b, double* x, void* stream) {
  return nothrow(h, [&] { return dev_level_op(h, 5, -1, b, nullptr, x, stream); });
}
int cdg_vcycle(cdg_handle* h, const double* r, double* z, void* stream) {
  return nothrow(h, [&] { return dev_vcycle(h, r, z, stream); });
}
int cdg_to_tree(cdg_handle* h, const double* user, double* tree, void* stream) {
  return nothrow(h, [&] { return dev_permute(h, user, tree, true, stream); });
}
int cdg_to_user(cdg_handle* h, const double* tree, double* user, void* stream) {
  return nothrow(h, [&] { return dev_permute(h, tree, user, false, stream); });
}

int cdg_smooth_static(cdg_handle* h, int32_t level, const double* x, const double* b, double* y, void* stream) {
  return nothrow(h, [&] { return dev_smooth_static(h, level, x, b, y, stream); });
}

int cdg_solve_multi(cdg_handle* h, const double* f_q, double* u, double* res_hist, int32_t* iters, void* stream) {
  if (!h || !f_q || !u) return h ? fail(h, CDG_EINVAL, "NULL argument") : CDG_EINVAL;
  return nothrow(h, [&] {
    std::vector<int> its(h->opt.nrhs > 0 ? h->opt.nrhs : 1, 0);
    const int rc = dev_solve_multi(h, f_q, u, res_hist, its.data(), stream);
    if (iters)
      for (size_t r = 0; r < its.size() && h->opt.nrhs > 0; ++r) iters[r] = its[r];
    return rc;
  });
}

int cdg_apply_multi(cdg_handle* h, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return h ? fail(h, CDG_EINVAL, "NULL argument") : CDG_EINVAL;
  return nothrow(h, [&] { return dev_apply_multi(h, x, y, stream); });
}

int cdg_solve_adjoint(cdg_handle* h, const double* dLdu, double* lambda, double* res_hist, int32_t* iters,
                      void* stream) {
  // A_0 is symmetric: A^T lambda = dL/du is the same solve as A_0 u = b
  if (h && h->opt.beta != 0.0) return fail(h, CDG_EINVAL, "no adjoint with convection (A_0 is not symmetric)");
  return cdg_solve_b(h, dLdu, lambda, 0, res_hist, iters, stream);
}

int cdg_rhs_adjoint(cdg_handle* h, const double* lambda, double* dLdf_q, void* stream) {
  if (!h || !lambda || !dLdf_q) return h ? fail(h, CDG_EINVAL, "NULL argument") : CDG_EINVAL;
  return nothrow(h, [&] { return dev_adjoint(h, 0, lambda, nullptr, nullptr, dLdf_q, stream); });
}

int cdg_kappa_gradient(cdg_handle* h, const double* lambda, const double* u, const double* gD_q, double* dLdkappa,
                       void* stream) {
  if (!h || !lambda || !u || !dLdkappa) return h ? fail(h, CDG_EINVAL, "NULL argument") : CDG_EINVAL;
  if (h->opt.beta != 0.0) return fail(h, CDG_EINVAL, "no adjoint with convection (A_0 is not symmetric)");
  return nothrow(h, [&] { return dev_adjoint(h, 1, lambda, u, gD_q, dLdkappa, stream); });
}

int64_t cdg_kernel_launches(void) { return (int64_t)dev_launch_count(); }

}  // extern "C"
