// Internal declarations shared by the host set-up (setup.cpp) and the CUDA side (igamg.cu).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "igamg.h"

namespace igamg {

// A 1D banded matrix with half-width hw: entry (i, j) lives at v[i*(2hw+1) + (j-i+hw)].
struct Band {
  int rows = 0, cols = 0, hw = 0;
  std::vector<double> v;
  void init(int r, int c, int h) {
    rows = r; cols = c; hw = h;
    v.assign((size_t)r * (2 * h + 1), 0.0);
  }
  double get(int i, int j) const {
    if (i < 0 || i >= rows || j < 0 || j >= cols) return 0.0;
    int d = j - i + hw;
    if (d < 0 || d > 2 * hw) return 0.0;
    return v[(size_t)i * (2 * hw + 1) + d];
  }
  void add(int i, int j, double x);
};

// Per-level 1D factors of the Kronecker form of K_l (2D, identity map, constant sigma, nu):
//   A_xx = X1 (x) Mq + X2 (x) Y2   [x-factor (x) y-factor],  A_yy = Mq (x) X1 + Y2 (x) X2,
//   B_x  = D (x) Mq,  B_y = Mq (x) D,  m = mq (x) mq.
// X1 = sigma M_p + nu S_p, X2 = nu M_p (degree p); Mq = M_{p-1}, Y2 = S_{p-1} + W_{p-1} with
// W the Nitsche wall terms of Sec. 3.3 (penalty C_I / h_fine on every level).
struct Level1D {
  int n = 0, p = 0, q = 0;
  Band X1, X2, Mq, Y2, D;     // all stored with half-width p
  std::vector<double> mq;     // int N^q_k, k = 0..n+q-1
  std::vector<double> dcoef;  // d/dx of degree-p splines: p/(t_{k+p}-t_k), k = 1..n+p-1 -> [k-1]
};

// 1D prolongation (fine x coarse) in two banded views.
struct Transfer1D {
  int nf = 0, nc = 0;          // rows (fine) and columns (coarse) of this view
  static constexpr int WP = 3; // max nonzeros per fine row
  static constexpr int WR = 5; // max nonzeros per coarse column
  std::vector<int> c0;         // per fine row: first coarse column
  std::vector<double> pv;      // nf * WP
  std::vector<int> f0;         // per coarse column: first fine row
  std::vector<double> rv;      // nc * WR
};

struct PatchTables {
  int n_patches = 0, maxl = 0, n_cls = 0, n_colours = 0, n_cls8 = 0;
  std::vector<int> dofs;       // n_patches * maxl (global dof ids, -1 padded), colour-major
  std::vector<int> cls;        // n_patches: index into cinv8 (8-DOF patches) or cinv (others)
  std::vector<int> nloc;       // per class of cinv: n_v + n_q
  std::vector<double> cinv;    // n_cls * maxl * maxl: leading block of the bordered inverse
  std::vector<double> cinv8;   // n_cls8 * 64: the same for 8-DOF patches, packed 8 x 8
  std::vector<int> colour_off; // n_colours + 1
  std::vector<int> n8;         // per colour: patches with 4+4 DOFs, stored first in the colour
  std::vector<int> d2p_off;    // dof -> list of (patch * maxl + local row), CSR over dofs
  std::vector<int> d2p_idx;
};

// Row stencils of K_l by row class.  A row's class is the pair of 1D position classes
// of its two indices (cls1 below): positions within T of either end are their own class,
// all others share the translation-invariant interior class.  Coefficients of neighbours
// outside the index range are stored as zero.
// Every record has the same length RU = B0 + B1 + 1 so that all row kinds run the same
// unconditional loops: box 0 (B0 = (2p+1)(2p-1) entries), box 1 (B1 = 2p(2p-1)), then the
// lambda coefficient; boxes are stored x-major (y fastest), shorter boxes zero-padded.
//   u_x rows: box 0 = A_xx over u_x (dx in -p..p, dy in -q..q), box 1 = -B_x over p
//             (kx in -p..p-1, dy in -q..q), last 0
//   u_y rows: box 0 = A_yy over u_y (dx in -q..q, dy in -p..p), box 1 = -B_y over p
//             (dx in -q..q, ky in -p..p-1), last 0
//   p rows:   box 0 = B_x^T over u_x (s in -q..p, dy in -q..q), box 1 = B_y^T over u_y
//             (dx in -q..q, s in -q..p), last m_k
struct Stencils {
  int T = 0, NC = 0, B0 = 0, B1 = 0, RU = 0;
  std::vector<double> sx, sy, sp;
};

inline int cls1(int i, int last, int T) { return i < T ? i : (last - i < T ? 2 * T - (last - i) : T); }

struct LevelHost {
  Level1D f;
  igamg_sizes sz{};
  PatchTables pt;
  Stencils st;
  // General (non-Kronecker) operators, e.g. generalized Oseen: one stencil record of RU
  // coefficients per row (rows 0 .. n_total-2, same layout as the class records); empty
  // when the class stencils describe the level.
  std::vector<double> rows;
};

struct HierarchyHost {
  int p = 0, L = 0, n_fine = 0;
  double sigma = 0, nu = 0, cpen = 0;
  std::vector<LevelHost> lev;          // 0 = coarsest
  std::vector<Transfer1D> tp_free;     // [l] : level l-1 -> l, degree p, interior indices
  std::vector<Transfer1D> tq;          // [l] : degree p-1, all indices
  std::vector<double> coarse_inv;      // ndof0 x ndof0
  int ndof0 = 0;
  // load vector tables on the finest level: per 1D basis i and local element k (0..d),
  // values times quadrature weight at the G points; G = p+2
  int G = 0;
  std::vector<double> lv_p, lv_q;      // (n+p)*(p+1)*G and (n+q)*(q+1)*G
  std::vector<double> quad_x;          // n*G abscissae (finest level)
};

// Builds everything; returns IGAMG_OK or an error code with a message in err.
int build_hierarchy(const igamg_problem& pr, HierarchyHost& H, std::string& err);
igamg_sizes level_sizes(int p, int n);
double k_entry(const Level1D& L, const igamg_sizes& s, long long g1, long long g2);
// entry (g1, g2) of a level given by per-row stencil records
double k_entry_rows(const LevelHost& lv, int p, long long g1, long long g2);
// 1D factors of one level with n elements; pen_over_nu = C_I / h_fine.
void build_level1d(int p, int n, double sigma, double nu, double pen_over_nu, Level1D& L);
void build_stencils(int p, const Level1D& L, const igamg_sizes& s, Stencils& st);

}  // namespace igamg
