// Quadrature, modal bases and level-0 mesh topology (Sections 2.2, 3.3).
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>
#include <stdexcept>

#include "host_setup.h"

namespace cdg {

// Gauss-Legendre points on [-1, 1] by Newton's method on the three-term
// recurrence, returned in ascending order.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) p0 = 1.0;
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static void gl01(int n, std::vector<double>& t, std::vector<double>& w) {
  gauss_legendre(n, t, w);
  for (int i = 0; i < n; ++i) {
    t[i] = 0.5 * (t[i] + 1.0);
    w[i] *= 0.5;
  }
}

// Collapsed (Duffy) product rule exact to total degree k on the unit simplex.
Rule simplex_rule(int dim, int k) {
  Rule r;
  r.dim = dim;
  auto cdiv = [](int a) { return (a + 1) / 2; };   // ceil(a/2)
  std::vector<double> a, wa, b, wb, c, wc;
  if (dim == 1) {
    gl01(cdiv(k + 1), a, wa);
    r.x = a;
    r.w = wa;
    return r;
  }
  gl01(cdiv(k + 1), a, wa);
  gl01(cdiv(k + 2), b, wb);
  if (dim == 2) {
    for (size_t i = 0; i < a.size(); ++i)
      for (size_t j = 0; j < b.size(); ++j) {
        r.x.push_back(a[i] * (1 - b[j]));
        r.x.push_back(b[j]);
        r.w.push_back(wa[i] * wb[j] * (1 - b[j]));
      }
    return r;
  }
  gl01(cdiv(k + 3), c, wc);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; j < b.size(); ++j)
      for (size_t l = 0; l < c.size(); ++l) {
        r.x.push_back(a[i] * (1 - b[j]) * (1 - c[l]));
        r.x.push_back(b[j] * (1 - c[l]));
        r.x.push_back(c[l]);
        r.w.push_back(wa[i] * wb[j] * wc[l] * (1 - b[j]) * (1 - c[l]) * (1 - c[l]));
      }
  return r;
}

void Monomials::init(int dim, int deg) {
  d = dim;
  p = deg;
  e.clear();
  for (int t = 0; t <= deg; ++t) {
    // all exponent tuples of total degree t, descending lexicographic order
    std::vector<std::array<int, 3>> layer;
    for (int a0 = t; a0 >= 0; --a0) {
      if (dim == 2) {
        layer.push_back({a0, t - a0, 0});
      } else {
        for (int a1 = t - a0; a1 >= 0; --a1) layer.push_back({a0, a1, t - a0 - a1});
      }
    }
    for (auto& a : layer)
      for (int k = 0; k < dim; ++k) e.push_back(a[k]);
  }
  np = (int)e.size() / dim;
}

static inline double ipow(double y, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= y;
  return r;
}

void Monomials::eval(const double* y, double* m) const {
  for (int j = 0; j < np; ++j) {
    double v = 1.0;
    for (int k = 0; k < d; ++k) v *= ipow(y[k], e[j * d + k]);
    m[j] = v;
  }
}

void Monomials::grad(const double* y, double inv_h, double* g) const {
  for (int j = 0; j < np; ++j)
    for (int k = 0; k < d; ++k) {
      int ek = e[j * d + k];
      if (ek == 0) {
        g[j * d + k] = 0.0;
        continue;
      }
      double v = ek * inv_h;
      for (int i = 0; i < d; ++i) v *= ipow(y[i], i == k ? ek - 1 : e[j * d + i]);
      g[j * d + k] = v;
    }
}

// ---------------------------------------------------------------- dense helpers
bool cholesky(int n, double* a) {
  for (int j = 0; j < n; ++j) {
    double s = a[j * n + j];
    for (int k = 0; k < j; ++k) s -= a[j * n + k] * a[j * n + k];
    if (!(s > 0.0)) return false;
    double ljj = std::sqrt(s);
    a[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = a[i * n + j];
      for (int k = 0; k < j; ++k) t -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = t / ljj;
    }
    for (int i = 0; i < j; ++i) a[i * n + j] = 0.0;
  }
  return true;
}

void lower_inverse(int n, const double* l, double* inv) {
  std::fill(inv, inv + (size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    for (int i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= l[(size_t)i * n + k] * inv[(size_t)k * n + c];
      inv[(size_t)i * n + c] = s / l[(size_t)i * n + i];
    }
  }
}

// Gauss-Jordan inverse with partial pivoting; false if singular to working precision.
bool lu_inverse(int n, const double* a, double* inv) {
  std::vector<double> m(a, a + (size_t)n * n);
  std::fill(inv, inv + (size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  double scale = 0.0;
  for (size_t t = 0; t < (size_t)n * n; ++t) scale = std::max(scale, std::fabs(a[t]));
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(m[(size_t)r * n + c]) > std::fabs(m[(size_t)piv * n + c])) piv = r;
    if (!(std::fabs(m[(size_t)piv * n + c]) > 1e-14 * scale)) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(m[(size_t)piv * n + k], m[(size_t)c * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)c * n + k]);
      }
    const double d = 1.0 / m[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      m[(size_t)c * n + k] *= d;
      inv[(size_t)c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = m[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        m[(size_t)r * n + k] -= f * m[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  return true;
}

bool spd_inverse(int n, const double* a, double* inv) {
  std::vector<double> l(a, a + (size_t)n * n), li((size_t)n * n);
  if (!cholesky(n, l.data())) return false;
  lower_inverse(n, l.data(), li.data());
  // inv = li^T li
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int k = i; k < n; ++k) s += li[(size_t)k * n + i] * li[(size_t)k * n + j];
      inv[(size_t)i * n + j] = s;
      inv[(size_t)j * n + i] = s;
    }
  return true;
}

// ---------------------------------------------------------------- bases
static void simplex_map(int d, const double* v, const Rule& r, int q, double* x, double& wphys,
                        double absdet) {
  const double* xi = r.x.data() + (size_t)q * d;
  for (int k = 0; k < d; ++k) {
    double s = v[k];
    for (int i = 0; i < d; ++i) s += xi[i] * (v[(i + 1) * d + k] - v[k]);
    x[k] = s;
  }
  wphys = r.w[q] * absdet;
}

static double simplex_absdet(int d, const double* v) {
  if (d == 2) {
    double a = v[2] - v[0], b = v[3] - v[1], c = v[4] - v[0], e = v[5] - v[1];
    return std::fabs(a * e - b * c);
  }
  double m[9];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) m[i * 3 + k] = v[(i + 1) * 3 + k] - v[k];
  double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
               m[2] * (m[3] * m[7] - m[4] * m[6]);
  return std::fabs(det);
}

static void simplex_coords(const Mesh0& m, i64 K, double* v) {
  for (int i = 0; i <= m.d; ++i)
    for (int k = 0; k < m.d; ++k) v[i * m.d + k] = m.xyz[m.elem[K * (m.d + 1) + i] * m.d + k];
}

void basis_eval(const Hierarchy& H, const BasisSet& B, i64 e, const double* x, double* phi) {
  const int d = B.d, np = B.np;
  double y[3] = {0.0, 0.0, 0.0}, mval[64];
  const double ih = 1.0 / B.h[e];
  for (int k = 0; k < d; ++k) y[k] = (x[k] - B.c[e * d + k]) * ih;
  H.mono.eval(y, mval);
  const double* T = B.T.data() + (size_t)e * np * np;
  for (int i = 0; i < np; ++i) {
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s += T[i * np + j] * mval[j];
    phi[i] = s;
  }
}

void basis_grad(const Hierarchy& H, const BasisSet& B, i64 e, const double* x, double* gphi) {
  const int d = B.d, np = B.np;
  double y[3] = {0.0, 0.0, 0.0}, g[64 * 3];
  const double ih = 1.0 / B.h[e];
  for (int k = 0; k < d; ++k) y[k] = (x[k] - B.c[e * d + k]) * ih;
  H.mono.grad(y, ih, g);
  const double* T = B.T.data() + (size_t)e * np * np;
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < d; ++k) {
      double s = 0.0;
      for (int j = 0; j <= i; ++j) s += T[i * np + j] * g[j * d + k];
      gphi[i * d + k] = s;
    }
}

void make_bases(Hierarchy& H, const std::vector<std::vector<i64>>& members, BasisSet& B) {
  const Mesh0& m = H.mesh;
  const int d = m.d, np = H.np;
  const i64 n = (i64)members.size();
  B.d = d;
  B.np = np;
  B.c.assign(n * d, 0.0);
  B.h.assign(n, 0.0);
  B.vol.assign(n, 0.0);
  B.T.assign((size_t)n * np * np, 0.0);
  bool bad = false;
#pragma omp parallel for schedule(dynamic, 64)
  for (i64 e = 0; e < n; ++e) {
    double v[12], cen[3] = {0, 0, 0}, vol = 0.0;
    for (i64 K : members[e]) {
      const double vk = m.vol[K];
      simplex_coords(m, K, v);
      for (int k = 0; k < d; ++k) {
        double s = 0.0;
        for (int i = 0; i <= d; ++i) s += v[i * d + k];
        cen[k] += vk * s / (d + 1);
      }
      vol += vk;
    }
    for (int k = 0; k < d; ++k) cen[k] /= vol;
    double h = 0.0;
    for (i64 K : members[e])
      for (int i = 0; i <= d; ++i) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
          double t = m.xyz[m.elem[K * (d + 1) + i] * d + k] - cen[k];
          s += t * t;
        }
        h = std::max(h, std::sqrt(s));
      }
    std::vector<double> gram((size_t)np * np, 0.0), mv(np);
    const double ih = 1.0 / h;
    for (i64 K : members[e]) {
      simplex_coords(m, K, v);
      const double ad = simplex_absdet(d, v);
      for (int q = 0; q < H.vrule.n(); ++q) {
        double x[3], w, y[3];
        simplex_map(d, v, H.vrule, q, x, w, ad);
        for (int k = 0; k < d; ++k) y[k] = (x[k] - cen[k]) * ih;
        H.mono.eval(y, mv.data());
        for (int i = 0; i < np; ++i)
          for (int j = 0; j <= i; ++j) gram[i * np + j] += w * mv[i] * mv[j];
      }
    }
    for (int i = 0; i < np; ++i)
      for (int j = i + 1; j < np; ++j) gram[i * np + j] = gram[j * np + i];
    if (!cholesky(np, gram.data())) {
#pragma omp atomic write
      bad = true;
      continue;
    }
    lower_inverse(np, gram.data(), B.T.data() + (size_t)e * np * np);
    for (int k = 0; k < d; ++k) B.c[e * d + k] = cen[k];
    B.h[e] = h;
    B.vol[e] = vol;
  }
  if (bad) throw std::runtime_error("basis Gram matrix not positive definite (degenerate element)");
}

// ---------------------------------------------------------------- mesh topology
static void face_normal(int d, const double* fv, const double* opp, double* n, double& meas) {
  if (d == 2) {
    double tx = fv[2] - fv[0], ty = fv[3] - fv[1];
    n[0] = ty;
    n[1] = -tx;
    meas = std::sqrt(tx * tx + ty * ty);
  } else {
    double a[3], b[3];
    for (int k = 0; k < 3; ++k) {
      a[k] = fv[3 + k] - fv[k];
      b[k] = fv[6 + k] - fv[k];
    }
    n[0] = a[1] * b[2] - a[2] * b[1];
    n[1] = a[2] * b[0] - a[0] * b[2];
    n[2] = a[0] * b[1] - a[1] * b[0];
    meas = 0.5 * std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  }
  double nn = 0.0, s = 0.0;
  for (int k = 0; k < d; ++k) nn += n[k] * n[k];
  nn = std::sqrt(nn);
  for (int k = 0; k < d; ++k) {
    n[k] /= nn;
    s += n[k] * (opp[k] - fv[k]);
  }
  if (s > 0)
    for (int k = 0; k < d; ++k) n[k] = -n[k];
}

static void local_face(const Mesh0& m, i64 K, int l, double* fv, double* opp) {
  const int d = m.d;
  int c = 0;
  for (int j = 0; j <= d; ++j) {
    const double* p = m.xyz.data() + m.elem[K * (d + 1) + j] * d;
    if (j == l) {
      for (int k = 0; k < d; ++k) opp[k] = p[k];
    } else {
      for (int k = 0; k < d; ++k) fv[c * d + k] = p[k];
      ++c;
    }
  }
}

void build_mesh(const int dim, i64 nv, const double* xyz, i64 ne, const i64* elem, i64 nbf,
                const i64* bface, const i32* btag, const Options& opt, Mesh0& m) {
  if (dim != 2 && dim != 3) throw std::invalid_argument("dim must be 2 or 3");
  if (nv <= 0 || ne <= 0 || !xyz || !elem) throw std::invalid_argument("empty mesh");
  const int d = dim, nvk = d + 1;
  m.d = d;
  m.nv = nv;
  m.ne = ne;
  m.xyz.assign(xyz, xyz + nv * d);
  m.elem.assign(elem, elem + ne * nvk);
  for (i64 i = 0; i < ne * nvk; ++i)
    if (m.elem[i] < 0 || m.elem[i] >= nv) throw std::invalid_argument("element vertex index out of range");
  m.vol.assign(ne, 0.0);
  bool degenerate = false;
  for (i64 K = 0; K < ne; ++K) {
    double v[12];
    simplex_coords(m, K, v);
    double emax = 0.0;
    for (int i = 1; i <= d; ++i) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += (v[i * d + k] - v[k]) * (v[i * d + k] - v[k]);
      emax = std::max(emax, std::sqrt(s));
    }
    double ad = simplex_absdet(d, v);
    if (!(ad > 1e-12 * std::pow(emax, d))) degenerate = true;
    m.vol[K] = ad / (d == 2 ? 2.0 : 6.0);
  }
  if (degenerate) throw std::domain_error("degenerate or inverted element (zero volume)");
  // faces: sort (sorted vertex tuple, element, local face)
  struct FK {
    std::array<i64, 3> key;
    i64 K;
    int l;
  };
  std::vector<FK> fk((size_t)ne * nvk);
  for (i64 K = 0; K < ne; ++K)
    for (int l = 0; l < nvk; ++l) {
      FK& f = fk[K * nvk + l];
      int c = 0;
      f.key = {-1, -1, -1};
      for (int j = 0; j < nvk; ++j)
        if (j != l) f.key[c++] = m.elem[K * nvk + j];
      std::sort(f.key.begin(), f.key.begin() + d);
      f.K = K;
      f.l = l;
    }
  std::sort(fk.begin(), fk.end(), [](const FK& a, const FK& b) {
    if (a.key != b.key) return a.key < b.key;
    if (a.K != b.K) return a.K < b.K;
    return a.l < b.l;
  });
  // boundary tags
  std::vector<std::pair<std::array<i64, 3>, int>> tags;
  for (i64 i = 0; i < nbf; ++i) {
    std::array<i64, 3> k = {-1, -1, -1};
    for (int j = 0; j < d; ++j) k[j] = bface[i * d + j];
    std::sort(k.begin(), k.begin() + d);
    const int t = btag ? btag[i] : 0;
    if (t != 0 && t != 1) throw std::invalid_argument("btag must be 0 (Dirichlet) or 1 (Neumann)");
    tags.push_back({k, t});
  }
  std::sort(tags.begin(), tags.end());
  for (size_t i = 1; i < tags.size(); ++i)
    if (tags[i].first == tags[i - 1].first) throw std::invalid_argument("a boundary face is listed twice in bface");
  std::vector<char> tag_used(tags.size(), 0);
  struct IF {
    i64 K1, K2;
    int l1, l2;
  };
  struct BF {
    i64 K;
    int l, tag;
  };
  std::vector<IF> ifs;
  std::vector<BF> bfs;
  for (size_t i = 0; i < fk.size();) {
    size_t j = i;
    while (j < fk.size() && fk[j].key == fk[i].key) ++j;
    if (j - i == 2) {
      ifs.push_back({fk[i].K, fk[i + 1].K, fk[i].l, fk[i + 1].l});
    } else if (j - i == 1) {
      int tag = 0;
      auto it = std::lower_bound(tags.begin(), tags.end(), std::make_pair(fk[i].key, INT32_MIN));
      if (it != tags.end() && it->first == fk[i].key) {
        tag = it->second;
        tag_used[it - tags.begin()] = 1;
      }
      bfs.push_back({fk[i].K, fk[i].l, tag});
    } else {
      throw std::domain_error("non-manifold face shared by more than two elements");
    }
    i = j;
  }
  for (char u : tag_used)
    if (!u) throw std::invalid_argument("a bface entry is not a boundary face of the mesh");
  std::sort(ifs.begin(), ifs.end(), [](const IF& a, const IF& b) {
    return a.K1 != b.K1 ? a.K1 < b.K1 : a.K2 < b.K2;
  });
  std::sort(bfs.begin(), bfs.end(), [](const BF& a, const BF& b) {
    return a.K != b.K ? a.K < b.K : a.l < b.l;
  });
  const i64 nif = (i64)ifs.size(), nb = (i64)bfs.size();
  m.if_K1.resize(nif); m.if_K2.resize(nif); m.if_l1.resize(nif); m.if_l2.resize(nif);
  m.if_n.resize(nif * d); m.if_meas.resize(nif); m.if_xv.resize(nif * d * d);
  m.if_S1.resize(nif); m.if_q.resize(nif); m.if_u.resize(nif);
  m.elem_face.assign(ne * nvk, 0);
  m.nbrs.assign(ne, {});
  const double wdir[3] = {1.0, std::sqrt(2.0), std::sqrt(3.0)};
  if (!opt.face_switch.empty() && (i64)opt.face_switch.size() != nif)
    throw std::invalid_argument("face_switch must have one entry per interior face");
  for (i64 f = 0; f < nif; ++f) {
    const IF& F = ifs[f];
    m.if_K1[f] = F.K1; m.if_K2[f] = F.K2; m.if_l1[f] = F.l1; m.if_l2[f] = F.l2;
    double opp[3];
    local_face(m, F.K1, F.l1, &m.if_xv[f * d * d], opp);
    face_normal(d, &m.if_xv[f * d * d], opp, &m.if_n[f * d], m.if_meas[f]);
    int S;
    if (!opt.face_switch.empty()) {
      S = opt.face_switch[f] > 0 ? 1 : -1;
    } else if (opt.switch_kind == 1) {
      i64 N1 = opt.enumeration.empty() ? F.K1 : opt.enumeration[F.K1];
      i64 N2 = opt.enumeration.empty() ? F.K2 : opt.enumeration[F.K2];
      S = N1 > N2 ? 1 : -1;
    } else {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += m.if_n[f * d + k] * wdir[k];
      if (std::fabs(s) < 1e-12) S = F.K1 > F.K2 ? 1 : -1;
      else S = s > 0 ? 1 : -1;
    }
    m.if_S1[f] = (int8_t)S;
    m.if_q[f] = S < 0 ? F.K1 : F.K2;
    m.if_u[f] = S < 0 ? F.K2 : F.K1;
    m.elem_face[F.K1 * nvk + F.l1] = f;
    m.elem_face[F.K2 * nvk + F.l2] = f;
    m.nbrs[F.K1].push_back(F.K2);
    m.nbrs[F.K2].push_back(F.K1);
  }
  m.bf_K.resize(nb); m.bf_l.resize(nb); m.bf_tag.resize(nb);
  m.bf_n.resize(nb * d); m.bf_meas.resize(nb); m.bf_xv.resize(nb * d * d);
  double hsum = 0.0;
  i64 nd = 0;
  for (i64 b = 0; b < nb; ++b) {
    m.bf_K[b] = bfs[b].K; m.bf_l[b] = bfs[b].l; m.bf_tag[b] = bfs[b].tag;
    double opp[3];
    local_face(m, bfs[b].K, bfs[b].l, &m.bf_xv[b * d * d], opp);
    face_normal(d, &m.bf_xv[b * d * d], opp, &m.bf_n[b * d], m.bf_meas[b]);
    m.elem_face[bfs[b].K * nvk + bfs[b].l] = -(1 + b);
    if (bfs[b].tag == 0) {
      hsum += d * m.vol[bfs[b].K] / m.bf_meas[b];
      ++nd;
    }
  }
  if (nd == 0) throw std::domain_error("the Dirichlet boundary must have positive measure");
  for (auto& v : m.nbrs) std::sort(v.begin(), v.end());
  m.h_avg = hsum / nd;
  m.C_D = opt.gamma / m.h_avg;
}

}  // namespace cdg
