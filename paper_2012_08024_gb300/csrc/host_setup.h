// Host-side set-up of the CDG agglomeration multigrid hierarchy.
//
// Everything here runs once per mesh on the CPU: simplex quadrature, orthonormal
// modal bases on elements and agglomerates (Section 3.3), the level-0 CDG
// operator and discrete gradient (Section 2), greedy agglomeration (Section 3.2,
// Algorithms 1-2), transfers (Section 3.4) and flux coarsening (Section 4.1).
// The result is a stack of block-sparse levels in "tree order" (children of every
// agglomerate contiguous) that the device solver uploads once.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace cdg {

using i64 = int64_t;
using i32 = int32_t;

// ---------------------------------------------------------------- quadrature
struct Rule {            // reference simplex rule: points [n][dim], weights [n]
  int dim = 0;
  std::vector<double> x, w;
  int n() const { return (int)w.size(); }
};
Rule simplex_rule(int dim, int degree);

// ---------------------------------------------------------------- bases
struct Monomials {       // exponent table, graded by degree, descending lex inside
  int d = 0, p = 0, np = 0;
  std::vector<int> e;    // [np][d]
  void init(int dim, int deg);
  void eval(const double* y, double* m) const;               // y = (x - c)/h
  void grad(const double* y, double inv_h, double* g) const; // g [np][d]
};

struct BasisSet {        // one orthonormal basis per element/agglomerate of a level
  int d = 0, np = 0;
  std::vector<double> c;   // [n][d] centroid
  std::vector<double> h;   // [n]
  std::vector<double> T;   // [n][np][np], phi = T m, lower triangular
  std::vector<double> vol; // [n]
};

// ---------------------------------------------------------------- sparse blocks
struct BSR {             // block compressed rows, blocks row-major
  i64 nrows = 0, ncols = 0;
  int br = 0, bc = 0;
  std::vector<i64> rowptr;
  std::vector<i32> col;
  std::vector<double> val;
  i64 nnzb() const { return (i64)col.size(); }
  const double* block(i64 b) const { return val.data() + b * (i64)br * bc; }
  double* block(i64 b) { return val.data() + b * (i64)br * bc; }
};

// ---------------------------------------------------------------- options
struct Options {
  int p = 2;
  double gamma = 1e4;
  int nu_pre = 1, nu_post = 1;
  double omega = 2.0 / 3.0;
  int max_levels = 4;
  uint64_t seed = 0;
  int switch_kind = 0;               // 0 directional (consistent), 1 natural
  std::vector<int8_t> face_switch;   // optional, per interior face (library order)
  std::vector<i64> enumeration;      // optional element enumeration for the natural switch
  int coarsen = 0;                   // 0 flux, 1 primal
  std::vector<double> kappa;         // optional per-element diffusion (input order)
  int pmg = 0;                       // 1: degrees p, p-1, ..., 2 on the fine mesh before the p = 1 hierarchy
  double beta = 0.0;                 // convection beta v . grad u (upwind DG, constant v)
  double vel[3] = {0.0, 0.0, 0.0};
};

// ---------------------------------------------------------------- level-0 mesh
struct Mesh0 {
  int d = 0;
  i64 nv = 0, ne = 0;
  std::vector<double> xyz;
  std::vector<i64> elem;
  std::vector<double> vol;
  // interior faces sorted by (K1, K2), K1 < K2
  std::vector<i64> if_K1, if_K2, if_q, if_u;
  std::vector<int> if_l1, if_l2;
  std::vector<double> if_n, if_meas, if_xv;   // normal out of K1, measure, vertex coords [nf][d][d]
  std::vector<int8_t> if_S1;                  // S_{K1}^{K2}
  // boundary faces sorted by (K, local face)
  std::vector<i64> bf_K;
  std::vector<int> bf_l, bf_tag;
  std::vector<double> bf_n, bf_meas, bf_xv;
  // element -> faces: elem_face[K*(d+1)+l] = interior face id, or -(1+boundary id)
  std::vector<i64> elem_face;
  std::vector<std::vector<i64>> nbrs;
  double h_avg = 0, C_D = 0;
};

struct Level {           // one multigrid level, working numbering
  i64 n = 0;
  std::vector<std::vector<i64>> verts;    // fine vertex ids of each element
  std::vector<std::vector<i64>> nbrs;     // face neighbours
  std::vector<std::vector<i64>> members;  // level-0 elements inside
  std::vector<i64> parent;                // -> next level (working ids)
  BasisSet basis;
  BSR A, G;                               // operator, discrete gradient (paper sign)
  std::vector<double> Lblk;               // [n][np][np] prolongation to this level from parent
  std::vector<double> Mk, Minv;           // [n][np][np] flux-form mass block (per component) and inverse
};

struct Hierarchy {
  Options opt;
  Mesh0 mesh;
  Monomials mono;
  Rule vrule, frule;
  int np = 0;                     // basis functions per element on level 0
  std::vector<Level> lev;
  // p-multigrid: the first n_plevels levels are degrees p, p-1, ..., 2 on the fine mesh
  // (rediscretised; truncation transfers), then the degree-1 agglomeration hierarchy
  int n_plevels = 0;
  std::vector<int> np_l;          // basis functions per element, per level
  // tree numbering: order[l][final] = working id; pos[l][working] = final
  std::vector<std::vector<i64>> order, pos;
  // level data in tree order (what the device uses)
  std::vector<BSR> A_t;                       // per level
  std::vector<std::vector<double>> Dinv_t;    // per level except coarsest: [n][np][np]
  std::vector<BSR> Ahat_t;                    // per level except coarsest: D^{-1} A without the diagonal blocks
  std::vector<std::vector<double>> L_t;       // per level except coarsest
  std::vector<std::vector<i32>> parent_t;     // per level except coarsest
  std::vector<std::vector<i32>> childptr_t;   // per level except finest: [n+1]
  std::vector<double> coarse_inv;             // dense inverse of the coarsest operator
  // right-hand side data (tree order of level 0)
  std::vector<double> rhs_vol;                // [ne][nq][np] = w_q phi_i(x_q)
  std::vector<i64> rhs_bptr;                  // [ne+1] boundary faces of each element
  std::vector<i64> rhs_bface;                 // boundary face ids
  std::vector<double> rhs_bD, rhs_bN;         // [nbf][nfq][np]
  // d A_0 / d kappa_K (R7: A_0 is linear in kappa), per element, unit-kappa pieces:
  // own block (volume + Dirichlet faces + q-side diagonal parts) and, for each
  // face where K is the q-side, the (K,J), (J,K), (J,J) blocks.  Working order
  // after build_level0, tree order (rows and J) after build_rhs_data.
  std::vector<double> dk_own;                 // [ne][np][np]
  std::vector<i64> dk_ptr;                    // [ne+1] q-faces of each element
  std::vector<i64> dk_nbr;                    // neighbour J of each q-face
  std::vector<double> dk_blk;                 // [nq_faces][3][np][np]: KJ, JK, JJ
  std::vector<double> kappa_w;                // kappa per element (working order), 1 if none
  // segments: independent meshes of a batched handle (one segment otherwise)
  std::vector<std::vector<i64>> seg_rows;     // [level][nseg+1] first tree row of each segment
  std::vector<i64> seg_coarse;                // [nseg+1] offsets of each dense inverse in coarse_inv
  std::vector<i64> seg_bface;                 // [nseg+1] first boundary face of each segment
  std::vector<Hierarchy> subs;                // per-mesh set-ups of a batched handle (mesh data only)
  // timings
  double t_mesh = 0, t_assemble = 0, t_agglomerate = 0, t_coarsen = 0;
};

// Concatenates finalized per-mesh hierarchies (same dim, p and level count)
// into one block-diagonal hierarchy with one segment per mesh.
void concat_hierarchies(std::vector<Hierarchy>& subs, Hierarchy& B);

// stage functions (each throws std::runtime_error with a message on bad input)
void build_mesh(const int dim, i64 nv, const double* xyz, i64 ne, const i64* elem, i64 nbf,
                const i64* bface, const i32* btag, const Options& opt, Mesh0& m);
void build_level0(Hierarchy& H);
void agglomerate(Hierarchy& H);
void coarsen(Hierarchy& H);
void finalize_tree_order(Hierarchy& H);
// tree-order operator of level l with n_p = np, and (unless last) its block
// inverses and the row-scaled smoother operator Ahat
void tree_level(Hierarchy& H, int l, int np, bool last);
// p-multigrid hierarchy: H holds level 0 at degree p (built), fine[q] the
// rediscretised operators of degrees p-1, ..., 2, H1 the degree-1 hierarchy
void merge_pmg(Hierarchy& H, std::vector<Hierarchy>& fine, Hierarchy& H1);
void build_rhs_data(Hierarchy& H);

// basis helpers
void basis_eval(const Hierarchy& H, const BasisSet& B, i64 e, const double* x, double* phi);
void basis_grad(const Hierarchy& H, const BasisSet& B, i64 e, const double* x, double* gphi);
void make_bases(Hierarchy& H, const std::vector<std::vector<i64>>& members, BasisSet& B);

uint64_t splitmix64(uint64_t x);
std::vector<std::vector<i64>> greedy_agglomerate(const std::vector<std::vector<i64>>& verts,
                                                 const std::vector<std::vector<i64>>& nbrs,
                                                 uint64_t seed, int level);

// small dense helpers
bool cholesky(int n, double* a);                  // in place, lower; false if not SPD
void lower_inverse(int n, const double* l, double* inv);
bool spd_inverse(int n, const double* a, double* inv);
bool lu_inverse(int n, const double* a, double* inv);    // partial pivoting; false if singular

}  // namespace cdg
