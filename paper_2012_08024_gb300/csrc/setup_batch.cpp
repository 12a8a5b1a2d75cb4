// Batched handles: many independent meshes solved together.  The per-mesh
// hierarchies are built as usual and concatenated level by level into one
// block-diagonal hierarchy (one segment per mesh), so every kernel of the solve
// phase processes all meshes in one launch; the CG keeps one set of scalars
// per segment.
#include <stdexcept>

#include "host_setup.h"

namespace cdg {

template <typename T>
static void append(std::vector<T>& dst, const std::vector<T>& src) {
  dst.insert(dst.end(), src.begin(), src.end());
}

static void append_bsr(BSR& dst, const BSR& src, i64 row_off, i64 col_off) {
  if (dst.rowptr.empty()) dst.rowptr.push_back(0);
  const i64 base = dst.rowptr.back();
  for (i64 r = 0; r < src.nrows; ++r) dst.rowptr.push_back(base + src.rowptr[r + 1]);
  for (i32 c : src.col) dst.col.push_back((i32)(c + col_off));
  append(dst.val, src.val);
  dst.nrows += src.nrows;
  dst.ncols += src.ncols;
  dst.br = src.br;
  dst.bc = src.bc;
  (void)row_off;
}

void concat_hierarchies(std::vector<Hierarchy>& subs, Hierarchy& B) {
  if (subs.empty()) throw std::invalid_argument("no meshes");
  const Hierarchy& F = subs[0];
  const int nlev = (int)F.lev.size();
  for (const Hierarchy& S : subs)
    if ((int)S.lev.size() != nlev || S.np != F.np || S.mesh.d != F.mesh.d)
      throw std::invalid_argument("batched meshes need the same dimension, degree and number of levels");
  B.opt = F.opt;
  B.mono = F.mono;
  B.vrule = F.vrule;
  B.frule = F.frule;
  B.np = F.np;
  B.np_l.assign(nlev, F.np);
  B.mesh.d = F.mesh.d;
  B.lev.assign(nlev, Level());
  B.A_t.assign(nlev, BSR());
  B.Ahat_t.assign(nlev, BSR());
  B.Dinv_t.assign(nlev, {});
  B.L_t.assign(nlev, {});
  B.parent_t.assign(nlev, {});
  B.childptr_t.assign(nlev, {});
  B.seg_rows.assign(nlev, {0});
  B.order.assign(nlev, {});
  B.seg_coarse = {0};
  B.seg_bface = {0};
  B.rhs_bptr = {0};
  B.dk_ptr = {0};
  i64 elem_off = 0, bf_off = 0;
  std::vector<i64> row_off(nlev, 0);
  for (Hierarchy& S : subs) {
    for (int l = 0; l < nlev; ++l) {
      const i64 ro = row_off[l];
      append_bsr(B.A_t[l], S.A_t[l], ro, ro);
      if (l + 1 < nlev) {
        append_bsr(B.Ahat_t[l], S.Ahat_t[l], ro, ro);
        append(B.Dinv_t[l], S.Dinv_t[l]);
        append(B.L_t[l], S.L_t[l]);
        for (i32 pa : S.parent_t[l]) B.parent_t[l].push_back((i32)(pa + row_off[l + 1]));
      }
      if (l > 0) {
        std::vector<i32>& cp = B.childptr_t[l];
        if (cp.empty()) cp.push_back(0);
        for (size_t a = 1; a < S.childptr_t[l].size(); ++a) cp.push_back((i32)(S.childptr_t[l][a] + row_off[l - 1]));
      }
      B.lev[l].n += S.lev[l].n;
    }
    for (int l = 0; l < nlev; ++l) {
      row_off[l] += S.lev[l].n;
      B.seg_rows[l].push_back(row_off[l]);
    }
    append(B.coarse_inv, S.coarse_inv);
    B.seg_coarse.push_back((i64)B.coarse_inv.size());
    // tree order of every level: mesh by mesh (level 0: user elements)
    for (int l = 0; l < nlev; ++l)
      for (i64 w : S.order[l]) B.order[l].push_back(w + row_off[l] - S.lev[l].n);
    append(B.rhs_vol, S.rhs_vol);
    const i64 nbf = (i64)S.mesh.bf_K.size();
    for (size_t k = 1; k < S.rhs_bptr.size(); ++k) B.rhs_bptr.push_back(B.rhs_bptr.back() + S.rhs_bptr[k] - S.rhs_bptr[k - 1]);
    for (i64 bf : S.rhs_bface) B.rhs_bface.push_back(bf + bf_off);
    append(B.rhs_bD, S.rhs_bD);
    for (int t : S.mesh.bf_tag) B.mesh.bf_tag.push_back(t);
    append(B.dk_own, S.dk_own);
    for (size_t k = 1; k < S.dk_ptr.size(); ++k) B.dk_ptr.push_back(B.dk_ptr.back() + S.dk_ptr[k] - S.dk_ptr[k - 1]);
    for (i64 J : S.dk_nbr) B.dk_nbr.push_back(J + elem_off);
    append(B.dk_blk, S.dk_blk);
    append(B.kappa_w, S.kappa_w);
    elem_off += S.mesh.ne;
    bf_off += nbf;
    B.seg_bface.push_back(bf_off);
    B.t_mesh += S.t_mesh;
    B.t_assemble += S.t_assemble;
    B.t_agglomerate += S.t_agglomerate;
    B.t_coarsen += S.t_coarsen;
    // keep only what the host-side queries need from each mesh
    Hierarchy keep;
    keep.mesh = std::move(S.mesh);
    keep.vrule = S.vrule;
    keep.frule = S.frule;
    keep.np = S.np;
    keep.lev.assign(S.lev.size(), Level());
    for (size_t l = 0; l < S.lev.size(); ++l) keep.lev[l].n = S.lev[l].n;
    S = std::move(keep);
  }
  B.mesh.ne = elem_off;
  B.mesh.bf_K.assign(bf_off, 0);
  B.subs = std::move(subs);
}

}  // namespace cdg
