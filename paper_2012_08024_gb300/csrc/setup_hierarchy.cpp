// Agglomeration hierarchy (Sections 3.1-3.2, Algorithms 1-2), transfers
// (Section 3.4) and flux coarsening (Section 4.1), then the tree numbering used
// on the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <stdexcept>
#include <string>

#include "host_setup.h"

namespace cdg {

// SplitMix64 finaliser (Steele, Lea & Flood): tie-break keys for the random
// choices of Algorithm 2, made reproducible across implementations.
uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static inline uint64_t tie_key(uint64_t seed, int level, i64 e_min, i64 cand) {
  return splitmix64(seed ^ ((uint64_t)level << 48) ^ ((uint64_t)e_min << 20) ^ (uint64_t)cand);
}

// One pass of Algorithm 2.  Pops the unprocessed element with the fewest
// unprocessed neighbours (ties: lowest index).  With >= 2 such neighbours it
// groups the unprocessed elements around the vertex of e_min touching most of
// them; otherwise it appends e_min to the smallest adjacent block, or, when no
// block is adjacent yet, groups as before (one neighbour) or stands alone.
std::vector<std::vector<i64>> greedy_agglomerate(const std::vector<std::vector<i64>>& verts,
                                                 const std::vector<std::vector<i64>>& nbrs,
                                                 uint64_t seed, int level) {
  const i64 n = (i64)verts.size();
  i64 vmax_id = 0;
  for (auto& vs : verts)
    for (i64 v : vs) vmax_id = std::max(vmax_id, v + 1);
  // vertex -> elements incidence (CSR, element ids ascending)
  std::vector<i64> iptr(vmax_id + 1, 0), inc;
  for (auto& vs : verts)
    for (i64 v : vs) ++iptr[v + 1];
  for (i64 v = 0; v < vmax_id; ++v) iptr[v + 1] += iptr[v];
  inc.resize(iptr[vmax_id]);
  {
    std::vector<i64> fill(iptr.begin(), iptr.end() - 1);
    for (i64 e = 0; e < n; ++e)
      for (i64 v : verts[e]) inc[fill[v]++] = e;
  }
  std::vector<i64> c(vmax_id);
  for (i64 v = 0; v < vmax_id; ++v) c[v] = iptr[v + 1] - iptr[v];
  std::vector<i64> N(n);
  std::vector<char> inP(n, 1);
  std::vector<i64> block_of(n, -1);
  using Entry = std::pair<i64, i64>;
  std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> heap;
  for (i64 e = 0; e < n; ++e) {
    N[e] = (i64)nbrs[e].size();
    heap.push({N[e], e});
  }
  std::vector<std::vector<i64>> blocks;
  auto remove = [&](i64 e) {
    inP[e] = 0;
    for (i64 v : verts[e]) --c[v];
  };
  auto decrement = [&](i64 e) {
    for (i64 e2 : nbrs[e])
      if (inP[e2]) {
        --N[e2];
        heap.push({N[e2], e2});
      }
  };
  while (!heap.empty()) {
    Entry top = heap.top();
    heap.pop();
    const i64 e_min = top.second;
    if (!inP[e_min] || top.first != N[e_min]) continue;
    remove(e_min);
    bool star = N[e_min] >= 2;
    if (!star) {
      i64 best = -1;
      size_t bsize = 0;
      uint64_t bkey = 0;
      for (i64 e2 : nbrs[e_min]) {
        const i64 B = block_of[e2];
        if (B < 0) continue;
        const size_t sz = blocks[B].size();
        const uint64_t key = tie_key(seed, level, e_min, B);
        if (best < 0 || sz < bsize || (sz == bsize && (key < bkey || (key == bkey && B < best)))) {
          best = B;
          bsize = sz;
          bkey = key;
        }
      }
      if (best >= 0) {
        blocks[best].push_back(e_min);
        block_of[e_min] = best;
        decrement(e_min);
        continue;
      }
      if (N[e_min] >= 1) {
        star = true;
      } else {
        block_of[e_min] = (i64)blocks.size();
        blocks.push_back({e_min});
        continue;
      }
    }
    i64 vbest = -1, cbest = 0;
    uint64_t kbest = 0;
    for (i64 v : verts[e_min]) {
      const uint64_t key = tie_key(seed, level, e_min, v);
      if (vbest < 0 || c[v] > cbest || (c[v] == cbest && (key < kbest || (key == kbest && v < vbest)))) {
        vbest = v;
        cbest = c[v];
        kbest = key;
      }
    }
    std::vector<i64> E = {e_min};
    for (i64 t = iptr[vbest]; t < iptr[vbest + 1]; ++t)
      if (inP[inc[t]]) E.push_back(inc[t]);   // ascending (incidence is ascending)
    for (size_t t = 1; t < E.size(); ++t) remove(E[t]);
    const i64 Bn = (i64)blocks.size();
    for (i64 e : E) block_of[e] = Bn;
    blocks.push_back(E);
    for (i64 e : E) decrement(e);
  }
  return blocks;
}

void agglomerate(Hierarchy& H) {
  const Mesh0& m = H.mesh;
  Level& L0 = H.lev[0];
  L0.n = m.ne;
  L0.verts.resize(m.ne);
  L0.members.resize(m.ne);
  for (i64 K = 0; K < m.ne; ++K) {
    L0.verts[K].assign(m.elem.begin() + K * (m.d + 1), m.elem.begin() + (K + 1) * (m.d + 1));
    std::sort(L0.verts[K].begin(), L0.verts[K].end());
    L0.members[K] = {K};
  }
  L0.nbrs = m.nbrs;
  while ((int)H.lev.size() < H.opt.max_levels && H.lev.back().n > 1) {
    Level& F = H.lev.back();
    const int l = (int)H.lev.size() - 1;
    auto blocks = greedy_agglomerate(F.verts, F.nbrs, H.opt.seed, l);
    Level Cn;
    Cn.n = (i64)blocks.size();
    F.parent.assign(F.n, -1);
    for (i64 B = 0; B < Cn.n; ++B)
      for (i64 e : blocks[B]) F.parent[e] = B;
    Cn.verts.resize(Cn.n);
    Cn.members.resize(Cn.n);
    Cn.nbrs.resize(Cn.n);
    for (i64 B = 0; B < Cn.n; ++B) {
      for (i64 e : blocks[B]) {
        Cn.verts[B].insert(Cn.verts[B].end(), F.verts[e].begin(), F.verts[e].end());
        Cn.members[B].insert(Cn.members[B].end(), F.members[e].begin(), F.members[e].end());
        for (i64 e2 : F.nbrs[e])
          if (F.parent[e2] != B) Cn.nbrs[B].push_back(F.parent[e2]);
      }
      auto uniq = [](std::vector<i64>& v) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
      };
      uniq(Cn.verts[B]);
      uniq(Cn.nbrs[B]);
    }
    H.lev.push_back(std::move(Cn));
  }
  // tree numbering
  const int nl = (int)H.lev.size();
  H.order.assign(nl, {});
  H.pos.assign(nl, {});
  for (int l = nl - 1; l >= 0; --l) {
    const i64 n = H.lev[l].n;
    std::vector<i64>& ord = H.order[l];
    ord.resize(n);
    for (i64 e = 0; e < n; ++e) ord[e] = e;
    if (l < nl - 1) {
      const std::vector<i64>& pp = H.pos[l + 1];
      const std::vector<i64>& par = H.lev[l].parent;
      std::stable_sort(ord.begin(), ord.end(), [&](i64 a, i64 b) {
        const i64 pa = pp[par[a]], pb = pp[par[b]];
        return pa != pb ? pa < pb : a < b;
      });
    }
    H.pos[l].assign(n, 0);
    for (i64 k = 0; k < n; ++k) H.pos[l][ord[k]] = k;
  }
}

// ------------------------------------------------------------------ coarsening
static void matmul_acc(int m, int k, int n, const double* A, const double* B, double* C, double s) {
  // C[m][n] += s * A[m][k] B[k][n]
  for (int i = 0; i < m; ++i)
    for (int p = 0; p < k; ++p) {
      const double a = s * A[i * k + p];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[i * n + j] += a * B[p * n + j];
    }
}

static void matTmul_acc(int k, int m, int n, const double* A, const double* B, double* C, double s) {
  // C[m][n] += s * A[k][m]^T B[k][n]
  for (int p = 0; p < k; ++p)
    for (int i = 0; i < m; ++i) {
      const double a = s * A[p * m + i];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[i * n + j] += a * B[p * n + j];
    }
}

static void simplex_vertices(const Mesh0& m, i64 K, double* v) {
  for (int i = 0; i <= m.d; ++i)
    for (int k = 0; k < m.d; ++k) v[i * m.d + k] = m.xyz[m.elem[K * (m.d + 1) + i] * m.d + k];
}

void coarsen(Hierarchy& H) {
  const Mesh0& m = H.mesh;
  const int d = m.d, np = H.np;
  const size_t nb2 = (size_t)np * np;
  const int nlev = (int)H.lev.size();
  for (int l = 0; l + 1 < nlev; ++l) {
    Level& F = H.lev[l];
    Level& Cn = H.lev[l + 1];
    make_bases(H, Cn.members, Cn.basis);
    // prolongation blocks L_K = int_K phi_K psi_parent^T
    F.Lblk.assign((size_t)F.n * nb2, 0.0);
#pragma omp parallel for schedule(dynamic, 64)
    for (i64 K = 0; K < F.n; ++K) {
      const i64 A = F.parent[K];
      double* LK = &F.Lblk[K * nb2];
      double v[12], x[3], pf[64], pc[64];
      for (i64 s : F.members[K]) {
        simplex_vertices(m, s, v);
        const double sc = m.vol[s] * (d == 2 ? 2.0 : 6.0);
        for (int q = 0; q < H.vrule.n(); ++q) {
          const double* xi = &H.vrule.x[(size_t)q * d];
          for (int k = 0; k < d; ++k) {
            double t = v[k];
            for (int i = 0; i < d; ++i) t += xi[i] * (v[(i + 1) * d + k] - v[k]);
            x[k] = t;
          }
          const double w = H.vrule.w[q] * sc;
          basis_eval(H, F.basis, K, x, pf);
          basis_eval(H, Cn.basis, A, x, pc);
          for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) LK[i * np + j] += w * pf[i] * pc[j];
        }
      }
    }
    // children lists (creation order is irrelevant for the sums below: each
    // coarse row sums its children in ascending working index)
    std::vector<std::vector<i64>> children(Cn.n);
    for (i64 K = 0; K < F.n; ++K) children[F.parent[K]].push_back(K);
    const bool flux = H.opt.coarsen == 0;
    const int gq = d * np;                 // q-rows per element
    const size_t gb = (size_t)gq * np;     // G block size
    // flux-form mass of level l+1: Mk_A = sum_{K in A} L_K^T Mk_K L_K (kappa-weighted, R7)
    Cn.Mk.assign((size_t)Cn.n * nb2, 0.0);
    Cn.Minv.assign((size_t)Cn.n * nb2, 0.0);
    bool mbad = false;
#pragma omp parallel for schedule(dynamic, 16)
    for (i64 A = 0; A < Cn.n; ++A) {
      std::vector<double> tmp(nb2);
      for (i64 K : children[A]) {
        std::fill(tmp.begin(), tmp.end(), 0.0);
        matmul_acc(np, np, np, &F.Mk[K * nb2], &F.Lblk[K * nb2], tmp.data(), 1.0);
        matTmul_acc(np, np, np, &F.Lblk[K * nb2], tmp.data(), &Cn.Mk[A * nb2], 1.0);
      }
      if (!spd_inverse(np, &Cn.Mk[A * nb2], &Cn.Minv[A * nb2])) mbad = true;
    }
    if (mbad) throw std::runtime_error("coarse flux-form mass matrix not positive definite");
    // GL = G_l L (per fine q-row, columns = coarse parents); WL = M_l^{-1} GL
    std::vector<i64> glptr(F.n + 1, 0);
    std::vector<i32> glcol;
    std::vector<double> glval, wlval;
    BSR& G = F.G;
    if (flux) {
      std::vector<std::vector<i32>> rc(F.n);
      for (i64 K = 0; K < F.n; ++K) {
        for (i64 b = G.rowptr[K]; b < G.rowptr[K + 1]; ++b) rc[K].push_back((i32)F.parent[G.col[b]]);
        std::sort(rc[K].begin(), rc[K].end());
        rc[K].erase(std::unique(rc[K].begin(), rc[K].end()), rc[K].end());
        glptr[K + 1] = glptr[K] + (i64)rc[K].size();
      }
      glcol.resize(glptr[F.n]);
      glval.assign((size_t)glptr[F.n] * gb, 0.0);
      wlval.assign((size_t)glptr[F.n] * gb, 0.0);
#pragma omp parallel for schedule(static)
      for (i64 K = 0; K < F.n; ++K) {
        std::copy(rc[K].begin(), rc[K].end(), glcol.begin() + glptr[K]);
        for (i64 b = G.rowptr[K]; b < G.rowptr[K + 1]; ++b) {
          const i64 J = G.col[b];
          const i32 B = (i32)F.parent[J];
          const i64 s = glptr[K] + (std::lower_bound(rc[K].begin(), rc[K].end(), B) - rc[K].begin());
          matmul_acc(gq, np, np, G.block(b), &F.Lblk[J * nb2], &glval[s * gb], 1.0);
        }
        for (i64 t = glptr[K]; t < glptr[K + 1]; ++t)
          for (int c = 0; c < d; ++c)
            matmul_acc(np, np, np, &F.Minv[K * nb2], &glval[t * gb + (size_t)c * nb2],
                       &wlval[t * gb + (size_t)c * nb2], 1.0);
      }
      // G_{l+1}[A, B] = sum_{K in A} (I_d (x) L_K)^T GL[K, B]
      BSR& Gc = Cn.G;
      Gc.nrows = Gc.ncols = Cn.n;
      Gc.br = gq;
      Gc.bc = np;
      Gc.rowptr.assign(Cn.n + 1, 0);
      std::vector<std::vector<i32>> cc(Cn.n);
      for (i64 A = 0; A < Cn.n; ++A) {
        for (i64 K : children[A])
          for (i64 t = glptr[K]; t < glptr[K + 1]; ++t) cc[A].push_back(glcol[t]);
        std::sort(cc[A].begin(), cc[A].end());
        cc[A].erase(std::unique(cc[A].begin(), cc[A].end()), cc[A].end());
        Gc.rowptr[A + 1] = Gc.rowptr[A] + (i64)cc[A].size();
      }
      Gc.col.resize(Gc.rowptr[Cn.n]);
      Gc.val.assign((size_t)Gc.rowptr[Cn.n] * gb, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
      for (i64 A = 0; A < Cn.n; ++A) {
        std::copy(cc[A].begin(), cc[A].end(), Gc.col.begin() + Gc.rowptr[A]);
        for (i64 K : children[A])
          for (i64 t = glptr[K]; t < glptr[K + 1]; ++t) {
            const i64 s = Gc.rowptr[A] + (std::lower_bound(cc[A].begin(), cc[A].end(), glcol[t]) - cc[A].begin());
            for (int c = 0; c < d; ++c)
              matTmul_acc(np, np, np, &F.Lblk[K * nb2], &glval[t * gb + (size_t)c * nb2],
                          Gc.block(s) + (size_t)c * nb2, 1.0);
          }
      }
    }
    std::vector<double> wcval;
    if (flux) {
      wcval.assign(Cn.G.val.size(), 0.0);
#pragma omp parallel for schedule(static)
      for (i64 A = 0; A < Cn.n; ++A)
        for (i64 t = Cn.G.rowptr[A]; t < Cn.G.rowptr[A + 1]; ++t)
          for (int c = 0; c < d; ++c)
            matmul_acc(np, np, np, &Cn.Minv[A * nb2], Cn.G.block(t) + (size_t)c * nb2,
                       &wcval[t * gb + (size_t)c * nb2], 1.0);
    }
    // transposed patterns: fine rows K with GL[K, B1] != 0; coarse rows A with Gc[A, B1] != 0
    std::vector<std::vector<std::pair<i64, i64>>> glT(flux ? Cn.n : 0), gcT(flux ? Cn.n : 0);
    if (flux) {
      for (i64 K = 0; K < F.n; ++K)
        for (i64 t = glptr[K]; t < glptr[K + 1]; ++t) glT[glcol[t]].push_back({K, t});
      for (i64 A = 0; A < Cn.n; ++A)
        for (i64 t = Cn.G.rowptr[A]; t < Cn.G.rowptr[A + 1]; ++t) gcT[Cn.G.col[t]].push_back({A, t});
    }
    // coarse operator rows
    const BSR& Af = F.A;
    std::vector<std::vector<i32>> acols(Cn.n);
    for (i64 B1 = 0; B1 < Cn.n; ++B1) {
      std::vector<i32>& cl = acols[B1];
      for (i64 K : children[B1])
        for (i64 b = Af.rowptr[K]; b < Af.rowptr[K + 1]; ++b) cl.push_back((i32)F.parent[Af.col[b]]);
      if (flux) {
        for (auto& kt : glT[B1])
          for (i64 t = glptr[kt.first]; t < glptr[kt.first + 1]; ++t) cl.push_back(glcol[t]);
        for (auto& at : gcT[B1])
          for (i64 t = Cn.G.rowptr[at.first]; t < Cn.G.rowptr[at.first + 1]; ++t) cl.push_back(Cn.G.col[t]);
      }
      std::sort(cl.begin(), cl.end());
      cl.erase(std::unique(cl.begin(), cl.end()), cl.end());
    }
    BSR& Ac = Cn.A;
    Ac.nrows = Ac.ncols = Cn.n;
    Ac.br = Ac.bc = np;
    Ac.rowptr.assign(Cn.n + 1, 0);
    for (i64 B1 = 0; B1 < Cn.n; ++B1) Ac.rowptr[B1 + 1] = Ac.rowptr[B1] + (i64)acols[B1].size();
    Ac.col.resize(Ac.rowptr[Cn.n]);
    Ac.val.assign((size_t)Ac.rowptr[Cn.n] * nb2, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
    for (i64 B1 = 0; B1 < Cn.n; ++B1) {
      const std::vector<i32>& cl = acols[B1];
      std::copy(cl.begin(), cl.end(), Ac.col.begin() + Ac.rowptr[B1]);
      auto slot = [&](i32 B2) {
        return Ac.rowptr[B1] + (i64)(std::lower_bound(cl.begin(), cl.end(), B2) - cl.begin());
      };
      std::vector<double> tmp(nb2);
      // L^T A_l L
      for (i64 K : children[B1])
        for (i64 b = Af.rowptr[K]; b < Af.rowptr[K + 1]; ++b) {
          const i64 J = Af.col[b];
          std::fill(tmp.begin(), tmp.end(), 0.0);
          matmul_acc(np, np, np, Af.block(b), &F.Lblk[J * nb2], tmp.data(), 1.0);
          matTmul_acc(np, np, np, &F.Lblk[K * nb2], tmp.data(), Ac.block(slot((i32)F.parent[J])), 1.0);
        }
      if (flux) {
        // - (G_l L)^T (G_l L)
        for (auto& kt : glT[B1]) {
          const i64 K = kt.first;
          const double* g1 = &glval[kt.second * gb];
          for (i64 t = glptr[K]; t < glptr[K + 1]; ++t)
            matTmul_acc(gq, np, np, g1, &wlval[t * gb], Ac.block(slot(glcol[t])), -1.0);
        }
        // + G_{l+1}^T G_{l+1}
        for (auto& at : gcT[B1]) {
          const i64 A = at.first;
          const double* g1 = Cn.G.block(at.second);
          for (i64 t = Cn.G.rowptr[A]; t < Cn.G.rowptr[A + 1]; ++t)
            matTmul_acc(gq, np, np, g1, &wcval[t * gb], Ac.block(slot(Cn.G.col[t])), 1.0);
        }
      }
    }
    // G_l is only needed to build level l+1
    std::vector<i64>().swap(F.G.rowptr);
    std::vector<double>().swap(F.G.val);
    std::vector<i32>().swap(F.G.col);
  }
}

// ------------------------------------------------------------------ tree order
void tree_level(Hierarchy& H, int l, int np, bool last) {
  const size_t nb2 = (size_t)np * np;
  const Level& Lv = H.lev[l];
  const BSR& A = Lv.A;
  BSR& T = H.A_t[l];
  const i64 n = Lv.n;
  T.nrows = T.ncols = n;
  T.br = T.bc = np;
  T.rowptr.assign(n + 1, 0);
  for (i64 k = 0; k < n; ++k) {
    const i64 r = H.order[l][k];
    T.rowptr[k + 1] = T.rowptr[k] + (A.rowptr[r + 1] - A.rowptr[r]);
  }
  T.col.resize(T.rowptr[n]);
  T.val.resize((size_t)T.rowptr[n] * nb2);
  bool notspd = false;
  if (!last) H.Dinv_t[l].assign((size_t)n * nb2, 0.0);
#pragma omp parallel for schedule(static)
  for (i64 k = 0; k < n; ++k) {
    const i64 r = H.order[l][k];
    std::vector<std::pair<i32, i64>> cb;
    for (i64 b = A.rowptr[r]; b < A.rowptr[r + 1]; ++b) cb.push_back({(i32)H.pos[l][A.col[b]], b});
    std::sort(cb.begin(), cb.end());
    for (size_t t = 0; t < cb.size(); ++t) {
      T.col[T.rowptr[k] + t] = cb[t].first;
      std::memcpy(T.block(T.rowptr[k] + t), A.block(cb[t].second), nb2 * sizeof(double));
      if (cb[t].first == k && !last) {
        // flux-coarsened operators need not be definite (observed on 3D meshes):
        // fall back to a pivoted inverse when the Cholesky factorisation fails
        // (a non-symmetric operator, with convection, always takes the pivoted inverse)
        const bool sym = H.opt.beta == 0.0;
        if (!(sym && spd_inverse(np, A.block(cb[t].second), &H.Dinv_t[l][k * nb2])) &&
            !lu_inverse(np, A.block(cb[t].second), &H.Dinv_t[l][k * nb2]))
          notspd = true;
      }
    }
  }
  if (notspd) throw std::runtime_error("singular diagonal block on level " + std::to_string(l));
  if (!last) {
    // row-scaled off-diagonal operator Ahat = D^{-1} (A - D) used by the smoother:
    // x + omega D^{-1}(b - A x) = x + omega (D^{-1} b - x - Ahat x)
    BSR& S = H.Ahat_t[l];
    S.nrows = S.ncols = n;
    S.br = S.bc = np;
    S.rowptr.assign(n + 1, 0);
    for (i64 k = 0; k < n; ++k) S.rowptr[k + 1] = S.rowptr[k] + (T.rowptr[k + 1] - T.rowptr[k] - 1);
    S.col.resize(S.rowptr[n]);
    S.val.assign((size_t)S.rowptr[n] * nb2, 0.0);
#pragma omp parallel for schedule(static)
    for (i64 k = 0; k < n; ++k) {
      i64 o = S.rowptr[k];
      const double* Di = &H.Dinv_t[l][k * nb2];
      for (i64 b = T.rowptr[k]; b < T.rowptr[k + 1]; ++b) {
        if (T.col[b] == k) continue;
        S.col[o] = T.col[b];
        const double* Ab = T.block(b);
        double* Sb = S.block(o);
        for (int i = 0; i < np; ++i)
          for (int j = 0; j < np; ++j) {
            double acc = 0.0;
            for (int m = 0; m < np; ++m) acc += Di[i * np + m] * Ab[m * np + j];
            Sb[i * np + j] = acc;
          }
        ++o;
      }
    }
  }
}

void finalize_tree_order(Hierarchy& H) {
  const int nlev = (int)H.lev.size();
  const int np = H.np;
  H.np_l.assign(nlev, np);
  const size_t nb2 = (size_t)np * np;
  H.A_t.assign(nlev, BSR());
  H.Dinv_t.assign(nlev, {});
  H.Ahat_t.assign(nlev, BSR());
  H.L_t.assign(nlev, {});
  H.parent_t.assign(nlev, {});
  H.childptr_t.assign(nlev, {});
  for (int l = 0; l < nlev; ++l) {
    const Level& Lv = H.lev[l];
    const i64 n = Lv.n;
    tree_level(H, l, np, l + 1 == nlev);
    if (l + 1 < nlev) {
      H.L_t[l].resize((size_t)n * nb2);
      H.parent_t[l].resize(n);
      for (i64 k = 0; k < n; ++k) {
        const i64 r = H.order[l][k];
        std::memcpy(&H.L_t[l][k * nb2], &Lv.Lblk[r * nb2], nb2 * sizeof(double));
        H.parent_t[l][k] = (i32)H.pos[l + 1][Lv.parent[r]];
      }
      std::vector<i32>& cp = H.childptr_t[l + 1];
      cp.assign(H.lev[l + 1].n + 1, 0);
      for (i64 k = 0; k < n; ++k) ++cp[H.parent_t[l][k] + 1];
      for (i64 a = 0; a < H.lev[l + 1].n; ++a) cp[a + 1] += cp[a];
    }
  }
  H.seg_rows.assign(nlev, {});
  for (int l = 0; l < nlev; ++l) H.seg_rows[l] = {0, H.lev[l].n};
  H.seg_bface = {0, (i64)H.mesh.bf_K.size()};
  // coarsest: dense SPD inverse
  const Level& Cl = H.lev.back();
  const i64 nc = Cl.n * np;
  if (nc > 16384) throw std::runtime_error("coarsest level too large for the dense solve; raise max_levels");
  std::vector<double> dense((size_t)nc * nc, 0.0);
  const BSR& T = H.A_t.back();
  for (i64 k = 0; k < Cl.n; ++k)
    for (i64 b = T.rowptr[k]; b < T.rowptr[k + 1]; ++b)
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j)
          dense[(size_t)(k * np + i) * nc + T.col[b] * np + j] = T.block(b)[i * np + j];
  H.coarse_inv.assign((size_t)nc * nc, 0.0);
  if (!(H.opt.beta == 0.0 && spd_inverse((int)nc, dense.data(), H.coarse_inv.data())) &&
      !lu_inverse((int)nc, dense.data(), H.coarse_inv.data()))
    throw std::runtime_error("singular coarsest operator");
  H.seg_coarse = {0, (i64)H.coarse_inv.size()};
}

// p-multigrid hierarchy (Section 4.4; reading R17).  Levels 0..P-1 hold the
// CDG operator rediscretised at degrees p, p-1, ..., 2 on the fine mesh (every
// element its own coarse element; the transfer between consecutive degrees is
// the truncation [I; 0] of the nested orthonormal bases, applied on the device
// without stored blocks), followed by the whole degree-1 hierarchy H1.  On
// entry H.lev[0] holds degree p and fine[i].lev[0] degree p-1-i (working order).
void merge_pmg(Hierarchy& H, std::vector<Hierarchy>& fine, Hierarchy& H1) {
  const int P = 1 + (int)fine.size();
  const int nh = (int)H1.lev.size();
  const int nlev = P + nh;
  const i64 ne = H.mesh.ne;
  std::vector<Level> lev;
  lev.reserve(nlev);
  lev.push_back(std::move(H.lev[0]));
  H.np_l.assign(1, H.np);
  for (Hierarchy& F : fine) {
    lev.push_back(std::move(F.lev[0]));
    H.np_l.push_back(F.np);
  }
  for (Level& L : H1.lev) {
    lev.push_back(std::move(L));
    H.np_l.push_back(H1.np);
  }
  H.lev = std::move(lev);
  H.n_plevels = P;
  for (int l = 0; l < P; ++l) {
    Level& L = H.lev[l];
    L.n = ne;
    L.parent.resize(ne);
    for (i64 K = 0; K < ne; ++K) L.parent[K] = K;
  }
  H.order.assign(P, H1.order[0]);
  H.pos.assign(P, H1.pos[0]);
  for (int h = 0; h < nh; ++h) {
    H.order.push_back(H1.order[h]);
    H.pos.push_back(H1.pos[h]);
  }
  H.A_t.assign(nlev, BSR());
  H.Dinv_t.assign(nlev, {});
  H.Ahat_t.assign(nlev, BSR());
  H.L_t.assign(nlev, {});
  H.parent_t.assign(nlev, {});
  H.childptr_t.assign(nlev, {});
  std::vector<i32> ident(ne), identp(ne + 1);
  for (i64 K = 0; K < ne; ++K) ident[K] = (i32)K;
  for (i64 K = 0; K <= ne; ++K) identp[K] = (i32)K;
  for (int l = 0; l < P; ++l) {
    tree_level(H, l, H.np_l[l], false);
    H.parent_t[l] = ident;
    H.childptr_t[l + 1] = identp;
  }
  for (int h = 0; h < nh; ++h) {
    const int l = P + h;
    H.A_t[l] = std::move(H1.A_t[h]);
    H.Dinv_t[l] = std::move(H1.Dinv_t[h]);
    H.Ahat_t[l] = std::move(H1.Ahat_t[h]);
    H.L_t[l] = std::move(H1.L_t[h]);
    H.parent_t[l] = std::move(H1.parent_t[h]);
    if (h > 0) H.childptr_t[l] = std::move(H1.childptr_t[h]);
  }
  H.seg_rows.assign(nlev, {});
  for (int l = 0; l < nlev; ++l) H.seg_rows[l] = {0, H.lev[l].n};
  H.seg_bface = {0, (i64)H.mesh.bf_K.size()};
  H.coarse_inv = std::move(H1.coarse_inv);
  H.seg_coarse = {0, (i64)H.coarse_inv.size()};
}

void build_rhs_data(Hierarchy& H) {
  const Mesh0& m = H.mesh;
  const int np = H.np, nq = H.vrule.n();
  const i64 ne = m.ne;
  const size_t nb2 = (size_t)np * np;
  // d A / d kappa pieces to tree order (rows and neighbour indices)
  {
    const std::vector<i64>& ord = H.order[0];
    const std::vector<i64>& pos = H.pos[0];
    std::vector<double> own((size_t)ne * nb2), blk(H.dk_blk.size()), kap(ne);
    std::vector<i64> ptr(ne + 1, 0), nbr(H.dk_nbr.size());
    for (i64 k = 0; k < ne; ++k) ptr[k + 1] = ptr[k] + (H.dk_ptr[ord[k] + 1] - H.dk_ptr[ord[k]]);
    for (i64 k = 0; k < ne; ++k) {
      const i64 K = ord[k];
      kap[k] = H.kappa_w[K];
      std::memcpy(&own[k * nb2], &H.dk_own[K * nb2], nb2 * sizeof(double));
      for (i64 t = H.dk_ptr[K], o = ptr[k]; t < H.dk_ptr[K + 1]; ++t, ++o) {
        nbr[o] = pos[H.dk_nbr[t]];
        std::memcpy(&blk[o * 3 * nb2], &H.dk_blk[t * 3 * nb2], 3 * nb2 * sizeof(double));
      }
    }
    H.dk_own.swap(own);
    H.dk_blk.swap(blk);
    H.dk_ptr.swap(ptr);
    H.dk_nbr.swap(nbr);
    H.kappa_w.swap(kap);
  }
  // volume data to tree order
  std::vector<double> v((size_t)ne * nq * np);
  for (i64 k = 0; k < ne; ++k)
    std::memcpy(&v[(size_t)k * nq * np], &H.rhs_vol[(size_t)H.order[0][k] * nq * np],
                sizeof(double) * nq * np);
  H.rhs_vol.swap(v);
  // boundary faces of every tree row
  H.rhs_bptr.assign(ne + 1, 0);
  for (size_t b = 0; b < m.bf_K.size(); ++b) ++H.rhs_bptr[H.pos[0][m.bf_K[b]] + 1];
  for (i64 k = 0; k < ne; ++k) H.rhs_bptr[k + 1] += H.rhs_bptr[k];
  H.rhs_bface.assign(m.bf_K.size(), 0);
  std::vector<i64> fill(H.rhs_bptr.begin(), H.rhs_bptr.end() - 1);
  for (size_t b = 0; b < m.bf_K.size(); ++b) H.rhs_bface[fill[H.pos[0][m.bf_K[b]]]++] = (i64)b;
}

}  // namespace cdg
