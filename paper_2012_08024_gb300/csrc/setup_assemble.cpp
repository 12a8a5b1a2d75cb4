// Level-0 CDG operator A_0, discrete gradient G_0 and right-hand-side data
// (Section 2.2 eqs. edge_flux_interior, edge_flux_boundary, cdg_fluxes;
// Section 2.3 eqs. disc_grad, primal_form).
//
// Solved problem: -div(kappa grad u) = f (the paper's Laplace(u) = f with the
// sign that makes A symmetric positive definite).  On an interior face f with
// q-side a (switch S_a^b < 0) and u-side b, unit normal n out of a and jump
// [[u]] = u_a - u_b, the primal bilinear form collects
//   kappa_K int_K grad u . grad v                                   (volume)
//   -kappa_a int_f ([[u]] dn v_a + [[v]] dn u_a)                     (consistency)
//   +kappa_a sum_k (int_f [[u]] phi^a_k)(int_f [[v]] phi^a_k)        (lifting r_f on a)
//   +kappa_K int_f (-u dn v - v dn u + C_D u v)   on Dirichlet faces.
// The lifting identity uses the orthonormal basis of a and the flatness of f.
// G_0 (paper's sign): (G u)_{K,c,k} = int_K u d_c phi_k - int_{dK \ Gamma_D} u-hat phi_k n_c.
#include <algorithm>
#include <cmath>
#include <stdexcept>

#include "host_setup.h"

namespace cdg {

static void face_point(int d, const double* xv, const Rule& r, int q, double meas, double* x,
                       double& w) {
  const double* xi = r.x.data() + (size_t)q * (d - 1);
  for (int k = 0; k < d; ++k) {
    double s = xv[k];
    for (int i = 0; i < d - 1; ++i) s += xi[i] * (xv[(i + 1) * d + k] - xv[k]);
    x[k] = s;
  }
  w = r.w[q] * meas * (d == 3 ? 2.0 : 1.0);
}

static void vol_point(const Mesh0& m, i64 K, const Rule& r, int q, double* x, double& w) {
  const int d = m.d;
  const double* xi = r.x.data() + (size_t)q * d;
  const i64* ev = m.elem.data() + K * (d + 1);
  const double* v0 = m.xyz.data() + ev[0] * d;
  for (int k = 0; k < d; ++k) {
    double s = v0[k];
    for (int i = 0; i < d; ++i) s += xi[i] * (m.xyz[ev[i + 1] * d + k] - v0[k]);
    x[k] = s;
  }
  w = r.w[q] * m.vol[K] * (d == 2 ? 2.0 : 6.0);
}

static inline double kap(const Options& o, i64 K) { return o.kappa.empty() ? 1.0 : o.kappa[K]; }

// R18: the convection term beta v . grad u of -div(kappa grad u) + beta v . grad u
// = f in upwind DG form (constant v): on each element -int_K u beta v.grad w plus
// int_{dK} beta (v.n) u-hat w with u-hat the trace of the element the flow
// leaves; on the boundary u-hat = u_K at outflow and on Neumann faces, and g_D
// at Dirichlet inflow, which becomes a right-hand-side term (added to the
// boundary data that multiplies g_D).  Added to A_0 after its assembly.
static void add_convection(Hierarchy& H) {
  const Mesh0& m = H.mesh;
  const int d = m.d, np = H.np;
  const i64 ne = m.ne, nif = (i64)m.if_K1.size(), nbf = (i64)m.bf_K.size();
  const BasisSet& B = H.lev[0].basis;
  BSR& A = H.lev[0].A;
  const size_t nb2 = (size_t)np * np;
  const int nq = H.vrule.n(), nfq = H.frule.n();
  double bv[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < d; ++c) bv[c] = H.opt.beta * H.opt.vel[c];
  auto block = [&](i64 K, i64 J) {
    const auto first = A.col.begin() + A.rowptr[K], last = A.col.begin() + A.rowptr[K + 1];
    const auto it = std::lower_bound(first, last, (i32)J);
    if (it == last || *it != (i32)J) throw std::logic_error("convection block outside the pattern of A_0");
    return A.block(A.rowptr[K] + (it - first));
  };
  // volume: row K only
#pragma omp parallel for schedule(static)
  for (i64 K = 0; K < ne; ++K) {
    double* blk = block(K, K);
    double x[3], w, ph[64], g[64 * 3], vg[64];
    for (int q = 0; q < nq; ++q) {
      vol_point(m, K, H.vrule, q, x, w);
      basis_eval(H, B, K, x, ph);
      basis_grad(H, B, K, x, g);
      for (int i = 0; i < np; ++i) {
        double s = 0.0;
        for (int c = 0; c < d; ++c) s += bv[c] * g[i * d + c];
        vg[i] = s;
      }
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) blk[i * np + j] -= w * vg[i] * ph[j];
    }
  }
  // interior faces: two blocks each (rows K1 and K2), computed in parallel, added in face order
  std::vector<double> Fc((size_t)nif * 2 * nb2, 0.0);
#pragma omp parallel for schedule(static)
  for (i64 f = 0; f < nif; ++f) {
    const i64 K1 = m.if_K1[f], K2 = m.if_K2[f];
    double vn = 0.0;
    for (int c = 0; c < d; ++c) vn += bv[c] * m.if_n[f * d + c];
    if (vn == 0.0) continue;
    const i64 up = vn > 0 ? K1 : K2;   // the element the flow leaves
    double* b1 = &Fc[(f * 2 + 0) * nb2];
    double* b2 = &Fc[(f * 2 + 1) * nb2];
    for (int q = 0; q < nfq; ++q) {
      double x[3], w, p1[64], pu[64], p2[64];
      face_point(d, &m.if_xv[f * d * d], H.frule, q, m.if_meas[f], x, w);
      basis_eval(H, B, K1, x, p1);
      basis_eval(H, B, K2, x, p2);
      basis_eval(H, B, up, x, pu);
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
          b1[i * np + j] += vn * w * p1[i] * pu[j];    // row K1: + vn int u-hat w_1
          b2[i * np + j] -= vn * w * p2[i] * pu[j];    // row K2: - vn int u-hat w_2
        }
    }
  }
  for (i64 f = 0; f < nif; ++f) {
    double vn = 0.0;
    for (int c = 0; c < d; ++c) vn += bv[c] * m.if_n[f * d + c];
    if (vn == 0.0) continue;
    const i64 K1 = m.if_K1[f], K2 = m.if_K2[f], up = vn > 0 ? K1 : K2;
    double* a1 = block(K1, up);
    double* a2 = block(K2, up);
    for (size_t t = 0; t < nb2; ++t) {
      a1[t] += Fc[(f * 2 + 0) * nb2 + t];
      a2[t] += Fc[(f * 2 + 1) * nb2 + t];
    }
  }
  // boundary faces: outflow and Neumann faces keep u_K (block), Dirichlet inflow moves g_D
  // to the right-hand side
  std::vector<double> Bc((size_t)nbf * nb2, 0.0);
#pragma omp parallel for schedule(static)
  for (i64 bfi = 0; bfi < nbf; ++bfi) {
    const i64 K = m.bf_K[bfi];
    double vn = 0.0;
    for (int c = 0; c < d; ++c) vn += bv[c] * m.bf_n[bfi * d + c];
    if (vn == 0.0) continue;
    const bool keep = vn > 0 || m.bf_tag[bfi] == 1;
    double* rb = &H.rhs_bD[(size_t)bfi * nfq * np];
    for (int q = 0; q < nfq; ++q) {
      double x[3], w, ph[64];
      face_point(d, &m.bf_xv[bfi * d * d], H.frule, q, m.bf_meas[bfi], x, w);
      basis_eval(H, B, K, x, ph);
      if (keep) {
        for (int i = 0; i < np; ++i)
          for (int j = 0; j < np; ++j) Bc[bfi * nb2 + i * np + j] += vn * w * ph[i] * ph[j];
      } else {
        for (int i = 0; i < np; ++i) rb[q * np + i] += -vn * w * ph[i];
      }
    }
  }
  for (i64 bfi = 0; bfi < nbf; ++bfi) {
    double* a = block(m.bf_K[bfi], m.bf_K[bfi]);
    for (size_t t = 0; t < nb2; ++t) a[t] += Bc[bfi * nb2 + t];
  }
}

void build_level0(Hierarchy& H) {
  Mesh0& m = H.mesh;
  const int d = m.d, np = H.np, nvk = d + 1;
  const i64 ne = m.ne, nif = (i64)m.if_K1.size(), nbf = (i64)m.bf_K.size();
  if (!H.opt.kappa.empty() && (i64)H.opt.kappa.size() != ne)
    throw std::invalid_argument("kappa must have one value per element");
  Level& L0 = H.lev[0];
  std::vector<std::vector<i64>> members(ne);
  for (i64 K = 0; K < ne; ++K) members[K] = {K};
  make_bases(H, members, L0.basis);
  const BasisSet& B = L0.basis;
  const size_t nb2 = (size_t)np * np;
  // flux-form mass (R7): M_K = I / kappa_K per component, orthonormal basis
  L0.Mk.assign((size_t)ne * nb2, 0.0);
  L0.Minv.assign((size_t)ne * nb2, 0.0);
  for (i64 K = 0; K < ne; ++K)
    for (int i = 0; i < np; ++i) {
      L0.Mk[K * nb2 + i * np + i] = 1.0 / kap(H.opt, K);
      L0.Minv[K * nb2 + i * np + i] = kap(H.opt, K);
    }
  const int nq = H.vrule.n(), nfq = H.frule.n();

  // volume blocks and G volume blocks
  std::vector<double> Vb((size_t)ne * nb2), GVb((size_t)ne * d * nb2);
#pragma omp parallel for schedule(static)
  for (i64 K = 0; K < ne; ++K) {
    double x[3], w, ph[64], g[64 * 3];
    double* V = &Vb[K * nb2];
    double* GV = &GVb[K * d * nb2];
    const double kk = kap(H.opt, K);
    for (int q = 0; q < nq; ++q) {
      vol_point(m, K, H.vrule, q, x, w);
      basis_eval(H, B, K, x, ph);
      basis_grad(H, B, K, x, g);
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
          double s = 0.0;
          for (int c = 0; c < d; ++c) s += g[i * d + c] * g[j * d + c];
          V[i * np + j] += kk * w * s;
        }
      for (int c = 0; c < d; ++c)
        for (int k = 0; k < np; ++k)
          for (int j = 0; j < np; ++j) GV[(c * np + k) * np + j] += w * g[k * d + c] * ph[j];
    }
  }
  // interior face blocks: aa, ab, ba, bb of A; G blocks (a,b) and (b,b)
  std::vector<double> Fb((size_t)nif * 4 * nb2), FG((size_t)nif * 2 * d * nb2);
#pragma omp parallel for schedule(static)
  for (i64 f = 0; f < nif; ++f) {
    const i64 a = m.if_q[f], b = m.if_u[f];
    double n[3];
    const double sg = (a == m.if_K1[f]) ? 1.0 : -1.0;
    for (int k = 0; k < d; ++k) n[k] = sg * m.if_n[f * d + k];
    std::vector<double> pa((size_t)nfq * np), pb((size_t)nfq * np), dna((size_t)nfq * np), wq(nfq);
    for (int q = 0; q < nfq; ++q) {
      double x[3], g[64 * 3];
      face_point(d, &m.if_xv[f * d * d], H.frule, q, m.if_meas[f], x, wq[q]);
      basis_eval(H, B, a, x, &pa[q * np]);
      basis_eval(H, B, b, x, &pb[q * np]);
      basis_grad(H, B, a, x, g);
      for (int i = 0; i < np; ++i) {
        double s = 0.0;
        for (int c = 0; c < d; ++c) s += g[i * d + c] * n[c];
        dna[q * np + i] = s;
      }
    }
    double* aa = &Fb[(f * 4 + 0) * nb2];
    double* ab = &Fb[(f * 4 + 1) * nb2];
    double* ba = &Fb[(f * 4 + 2) * nb2];
    double* bb = &Fb[(f * 4 + 3) * nb2];
    std::vector<double> Qaa(nb2, 0.0), Qab(nb2, 0.0);
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) {
        double s_aa = 0, s_ab = 0, s_ba = 0, qaa = 0, qab = 0;
        for (int q = 0; q < nfq; ++q) {
          const double w = wq[q];
          s_aa += w * (dna[q * np + i] * pa[q * np + j] + pa[q * np + i] * dna[q * np + j]);
          s_ab += w * dna[q * np + i] * pb[q * np + j];
          s_ba += w * pb[q * np + i] * dna[q * np + j];
          qaa += w * pa[q * np + i] * pa[q * np + j];
          qab += w * pa[q * np + i] * pb[q * np + j];
        }
        aa[i * np + j] = -s_aa;
        ab[i * np + j] = s_ab;
        ba[i * np + j] = s_ba;
        Qaa[i * np + j] = qaa;
        Qab[i * np + j] = qab;
      }
    // lifting: [[u]] moments int_f [[u]] phi^a_k = Qaa[k,:] u_a - Qab[k,:] u_b
    const double kk = kap(H.opt, a);
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) {
        double s_aa = 0, s_ab = 0, s_ba = 0, s_bb = 0;
        for (int k = 0; k < np; ++k) {
          s_aa += Qaa[k * np + i] * Qaa[k * np + j];
          s_ab += Qaa[k * np + i] * Qab[k * np + j];
          s_ba += Qab[k * np + i] * Qaa[k * np + j];
          s_bb += Qab[k * np + i] * Qab[k * np + j];
        }
        aa[i * np + j] = kk * (aa[i * np + j] + s_aa);
        ab[i * np + j] = kk * (ab[i * np + j] - s_ab);
        ba[i * np + j] = kk * (ba[i * np + j] - s_ba);
        bb[i * np + j] = kk * s_bb;
      }
    // G: q-side a takes u-hat = u_b; u-side b takes its own trace (normal -n)
    double* Gab = &FG[(f * 2 + 0) * d * nb2];
    double* Gbb = &FG[(f * 2 + 1) * d * nb2];
    for (int k = 0; k < np; ++k)
      for (int j = 0; j < np; ++j) {
        double s_ab = 0, s_bb = 0;
        for (int q = 0; q < nfq; ++q) {
          s_ab += wq[q] * pa[q * np + k] * pb[q * np + j];
          s_bb += wq[q] * pb[q * np + k] * pb[q * np + j];
        }
        for (int c = 0; c < d; ++c) {
          Gab[(c * np + k) * np + j] = -n[c] * s_ab;
          Gbb[(c * np + k) * np + j] = n[c] * s_bb;
        }
      }
  }
  // boundary faces: Dirichlet block of A, Neumann block of G, rhs data
  std::vector<double> Db((size_t)nbf * nb2, 0.0), NG((size_t)nbf * d * nb2, 0.0);
  H.rhs_bD.assign((size_t)nbf * nfq * np, 0.0);
#pragma omp parallel for schedule(static)
  for (i64 bfi = 0; bfi < nbf; ++bfi) {
    const i64 K = m.bf_K[bfi];
    const double* n = &m.bf_n[bfi * d];
    const double kk = kap(H.opt, K);
    std::vector<double> ph((size_t)nfq * np), dn((size_t)nfq * np), wq(nfq);
    for (int q = 0; q < nfq; ++q) {
      double x[3], g[64 * 3];
      face_point(d, &m.bf_xv[bfi * d * d], H.frule, q, m.bf_meas[bfi], x, wq[q]);
      basis_eval(H, B, K, x, &ph[q * np]);
      basis_grad(H, B, K, x, g);
      for (int i = 0; i < np; ++i) {
        double s = 0.0;
        for (int c = 0; c < d; ++c) s += g[i * d + c] * n[c];
        dn[q * np + i] = s;
      }
    }
    double* rb = &H.rhs_bD[(size_t)bfi * nfq * np];
    if (m.bf_tag[bfi] == 0) {
      double* D = &Db[bfi * nb2];
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
          double s = 0.0;
          for (int q = 0; q < nfq; ++q)
            s += wq[q] * (-dn[q * np + j] * ph[q * np + i] - ph[q * np + j] * dn[q * np + i] +
                          m.C_D * ph[q * np + i] * ph[q * np + j]);
          D[i * np + j] = kk * s;
        }
      for (int q = 0; q < nfq; ++q)
        for (int i = 0; i < np; ++i)
          rb[q * np + i] = kk * wq[q] * (-dn[q * np + i] + m.C_D * ph[q * np + i]);
    } else {
      double* G = &NG[bfi * d * nb2];
      for (int k = 0; k < np; ++k)
        for (int j = 0; j < np; ++j) {
          double s = 0.0;
          for (int q = 0; q < nfq; ++q) s += wq[q] * ph[q * np + k] * ph[q * np + j];
          for (int c = 0; c < d; ++c) G[(c * np + k) * np + j] = -n[c] * s;
        }
      for (int q = 0; q < nfq; ++q)
        for (int i = 0; i < np; ++i) rb[q * np + i] = wq[q] * ph[q * np + i];
    }
  }
  // volume rhs data
  H.rhs_vol.assign((size_t)ne * nq * np, 0.0);
#pragma omp parallel for schedule(static)
  for (i64 K = 0; K < ne; ++K)
    for (int q = 0; q < nq; ++q) {
      double x[3], w, ph[64];
      vol_point(m, K, H.vrule, q, x, w);
      basis_eval(H, B, K, x, ph);
      for (int i = 0; i < np; ++i) H.rhs_vol[((size_t)K * nq + q) * np + i] = w * ph[i];
    }

  // unit-kappa pieces of A_0 owned by each element (for d A_0 / d kappa)
  H.kappa_w.assign(ne, 1.0);
  for (i64 K = 0; K < ne; ++K) H.kappa_w[K] = kap(H.opt, K);
  H.dk_own.assign((size_t)ne * nb2, 0.0);
  H.dk_ptr.assign(ne + 1, 0);
  for (i64 f = 0; f < nif; ++f) ++H.dk_ptr[m.if_q[f] + 1];
  for (i64 K = 0; K < ne; ++K) H.dk_ptr[K + 1] += H.dk_ptr[K];
  H.dk_nbr.assign(nif, 0);
  H.dk_blk.assign((size_t)nif * 3 * nb2, 0.0);
  {
    std::vector<i64> fill(H.dk_ptr.begin(), H.dk_ptr.end() - 1);
    for (i64 f = 0; f < nif; ++f) {   // ascending face order inside each element
      const i64 K = m.if_q[f];
      const i64 t = fill[K]++;
      H.dk_nbr[t] = m.if_u[f];
      const double ik = 1.0 / kap(H.opt, K);
      for (size_t e = 0; e < nb2; ++e) {
        H.dk_own[K * nb2 + e] += ik * Fb[(f * 4 + 0) * nb2 + e];
        H.dk_blk[(t * 3 + 0) * nb2 + e] = ik * Fb[(f * 4 + 1) * nb2 + e];
        H.dk_blk[(t * 3 + 1) * nb2 + e] = ik * Fb[(f * 4 + 2) * nb2 + e];
        H.dk_blk[(t * 3 + 2) * nb2 + e] = ik * Fb[(f * 4 + 3) * nb2 + e];
      }
    }
  }
  for (i64 K = 0; K < ne; ++K) {
    const double ik = 1.0 / kap(H.opt, K);
    for (size_t e = 0; e < nb2; ++e) H.dk_own[K * nb2 + e] += ik * Vb[K * nb2 + e];
  }
  for (i64 bfi = 0; bfi < nbf; ++bfi)
    if (m.bf_tag[bfi] == 0) {
      const i64 K = m.bf_K[bfi];
      const double ik = 1.0 / kap(H.opt, K);
      for (size_t e = 0; e < nb2; ++e) H.dk_own[K * nb2 + e] += ik * Db[bfi * nb2 + e];
    }

  // assemble A_0 rows: diagonal + face neighbours, sorted columns
  BSR& A = L0.A;
  A.nrows = A.ncols = ne;
  A.br = A.bc = np;
  A.rowptr.assign(ne + 1, 0);
  for (i64 K = 0; K < ne; ++K) A.rowptr[K + 1] = A.rowptr[K] + 1 + (i64)m.nbrs[K].size();
  A.col.resize(A.rowptr[ne]);
  A.val.assign((size_t)A.rowptr[ne] * nb2, 0.0);
  BSR& G = L0.G;
  G.nrows = G.ncols = ne;
  G.br = d * np;
  G.bc = np;
  G.rowptr.assign(ne + 1, 0);
  for (i64 K = 0; K < ne; ++K) {
    int nq_side = 0;
    for (int l = 0; l < nvk; ++l) {
      i64 f = m.elem_face[K * nvk + l];
      if (f >= 0 && m.if_q[f] == K) ++nq_side;
    }
    G.rowptr[K + 1] = G.rowptr[K] + 1 + nq_side;
  }
  G.col.resize(G.rowptr[ne]);
  G.val.assign((size_t)G.rowptr[ne] * d * nb2, 0.0);
#pragma omp parallel for schedule(static)
  for (i64 K = 0; K < ne; ++K) {
    // A row
    std::vector<i64> cols = m.nbrs[K];
    cols.push_back(K);
    std::sort(cols.begin(), cols.end());
    const i64 r0 = A.rowptr[K];
    for (size_t t = 0; t < cols.size(); ++t) A.col[r0 + t] = (i32)cols[t];
    auto slot = [&](i64 J) {
      return r0 + (i64)(std::lower_bound(cols.begin(), cols.end(), J) - cols.begin());
    };
    double* diag = A.block(slot(K));
    for (size_t t = 0; t < nb2; ++t) diag[t] = Vb[K * nb2 + t];
    for (int l = 0; l < nvk; ++l) {
      i64 f = m.elem_face[K * nvk + l];
      if (f >= 0) {
        const bool isq = m.if_q[f] == K;
        const i64 J = isq ? m.if_u[f] : m.if_q[f];
        const double* dd = &Fb[(f * 4 + (isq ? 0 : 3)) * nb2];
        const double* od = &Fb[(f * 4 + (isq ? 1 : 2)) * nb2];
        double* off = A.block(slot(J));
        for (size_t t = 0; t < nb2; ++t) {
          diag[t] += dd[t];
          off[t] += od[t];
        }
      } else {
        const i64 bfi = -(f + 1);
        if (m.bf_tag[bfi] == 0)
          for (size_t t = 0; t < nb2; ++t) diag[t] += Db[bfi * nb2 + t];
      }
    }
    // G row: own block first, then u-sides of faces where K is the q-side (sorted)
    std::vector<std::pair<i64, i64>> qf;   // (neighbour, face)
    for (int l = 0; l < nvk; ++l) {
      i64 f = m.elem_face[K * nvk + l];
      if (f >= 0 && m.if_q[f] == K) qf.push_back({m.if_u[f], f});
    }
    std::vector<i64> gcols = {K};
    for (auto& pr : qf) gcols.push_back(pr.first);
    std::sort(gcols.begin(), gcols.end());
    const i64 g0 = G.rowptr[K];
    for (size_t t = 0; t < gcols.size(); ++t) G.col[g0 + t] = (i32)gcols[t];
    auto gslot = [&](i64 J) {
      return g0 + (i64)(std::lower_bound(gcols.begin(), gcols.end(), J) - gcols.begin());
    };
    double* gd = G.block(gslot(K));
    for (size_t t = 0; t < d * nb2; ++t) gd[t] = GVb[K * d * nb2 + t];
    for (int l = 0; l < nvk; ++l) {
      i64 f = m.elem_face[K * nvk + l];
      if (f >= 0) {
        if (m.if_q[f] == K) {
          double* go = G.block(gslot(m.if_u[f]));
          const double* src = &FG[(f * 2 + 0) * d * nb2];
          for (size_t t = 0; t < d * nb2; ++t) go[t] += src[t];
        } else {
          const double* src = &FG[(f * 2 + 1) * d * nb2];
          for (size_t t = 0; t < d * nb2; ++t) gd[t] += src[t];
        }
      } else {
        const i64 bfi = -(f + 1);
        if (m.bf_tag[bfi] == 1)
          for (size_t t = 0; t < d * nb2; ++t) gd[t] += NG[bfi * d * nb2 + t];
      }
    }
  }
  if (H.opt.beta != 0.0) add_convection(H);
}

}  // namespace cdg
