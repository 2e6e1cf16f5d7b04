// Internal declarations shared by the host set-up (setup.cpp) and the CUDA side (igamg.cu).
#pragma once
#include <cstdint>
#include <functional>
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
  std::vector<int> pos;         // 2D: per patch its streamfunction position a | b << 16
  std::vector<int> d2p_off;    // dof -> list of (patch * maxl + local row), CSR over dofs
  std::vector<int> d2p_idx;
  // Row-flat view for the row-parallel colour kernel: each colour is cut into blocks of
  // row_slots slots (128, 256, or 1024 on levels whose largest patch has more than 256 rows),
  // one slot per local row; a patch's rows sit in consecutive slots of one block (blocks
  // are padded instead of splitting a patch).
  int row_slots = 0;                // 0: no row-flat view (a patch larger than 1024 rows)
  std::vector<int> slot_g;          // dof of the slot's row, or -1 (padding)
  std::vector<int> slot_c;          // the patch's class: its matrix in cinv_all
  std::vector<unsigned> slot_kb;    // local row k | nl << 10 | (slot of the patch's row 0 in the block) << 20
  std::vector<int> colour_blk;      // n_colours + 1: first block of each colour
  std::vector<double> cinv_all;     // every class (8-DOF classes after the others), nl x nl packed
  std::vector<long long> cinv_off;  // offset of each class's matrix in cinv_all
};

// Fills the row-flat view (slot_*, colour_blk, cinv_all) from dofs / cls / nloc / cinv / cinv8.
void build_row_slots(PatchTables& pt);

// Schedule of the pipelined sweep (2D): patch positions 1..nint cut into tiles of tw x tw,
// tiles row-major (ntx per row); for tile t and colour c, list[off[t*C+c] .. off[t*C+c+1])
// holds the patch indices of that colour in the tile, its n8[t*C+c] 8-DOF patches first.
struct TileTables {
  int tw = 0, ntx = 0, nty = 0;
  std::vector<int> list, off, n8;
};
void build_tile_tables(const PatchTables& pt, int nint, int tw, TileTables& tt);

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
  // Mapped domains only (empty otherwise): per velocity row (0 .. n_ux+n_uy-1) the 2p x 2p
  // coefficients coupling it to the other velocity component (the third box of the record).
  std::vector<double> ext;
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
  // mapped domains: the finest level's quadrature points in physical coordinates, (2, nG, nG)
  // [component][eta point][xi point], and J^T there, (nG, nG, 2, 2) [.][.][k][i] = dX_i/dxi_k,
  // which turns f into the parametric load (J^T f)
  int geometry = 0;
  std::vector<double> quad_xy, jt;
  // generalized Oseen on the square: the finest level's advection term applied element by
  // element (matrix-free) needs, per element e and local basis function a, the 1D basis values
  // and derivatives at the element's G Gauss points, [(e*(d+1)+a)*G + g] for d = p (adv_bp,
  // adv_dp) and d = p-1 (adv_bq, adv_dq), and the Gauss weight times beta at every Gauss
  // point, (2, nG, nG) [component][y point][x point]; empty otherwise
  std::vector<double> adv_bp, adv_dp, adv_bq, adv_dq, adv_beta;
};

// Builds everything; returns IGAMG_OK or an error code with a message in err.
int build_hierarchy(const igamg_problem& pr, HierarchyHost& H, std::string& err);
// What the colour kernels rely on: every patch DOF is a row of the level (not lambda);
// within one colour no DOF appears twice (same-colour updates never touch the same entry);
// and no two patches of one colour are coupled through K.  The last is checked the way the
// method argues it (Sec. 5.2: subdomains of one colour overlap only on sets of measure
// zero): the element boxes spanned by the supports of each patch's DOFs must not share an
// element with another patch of the same colour.  Two basis functions whose supports share
// no element have a zero entry in every block of K (volume terms, Nitsche wall terms and,
// on coarse levels, the Galerkin products of functions supported inside the same boxes),
// so a patch's local residual never reads a value that a same-colour patch writes, and a
// colour's patches may run in any order or at once with the sequential sweep's result.
// support(g, lo, hi): element index range [lo, hi] of DOF g's support per direction;
// n_elem: elements per direction (dims beyond the level's dimension = 1).
bool validate_patch_tables(const PatchTables& pt, long long n_rows, std::string& err,
                           const std::function<void(long long, int*, int*)>& support, const int* n_elem);
igamg_sizes level_sizes(int p, int n);
double k_entry(const Level1D& L, const igamg_sizes& s, long long g1, long long g2);
// entry (g1, g2) of a level given by per-row stencil records
double k_entry_rows(const LevelHost& lv, int p, long long g1, long long g2);
// 1D factors of one level with n elements; pen_over_nu = C_I / h_fine.
void build_level1d(int p, int n, double sigma, double nu, double pen_over_nu, Level1D& L);
void build_stencils(int p, const Level1D& L, const igamg_sizes& s, Stencils& st);

// helpers of setup.cpp shared with the 3D set-up
std::vector<double> knots(int d, int n);
void span_values(const std::vector<double>& t, int d, int s, double x, double* N);
void span_derivs(const std::vector<double>& t, int d, int s, double x, double* dN);
void gauss01(int m, std::vector<double>& x, std::vector<double>& w);
bool invert(std::vector<double> A, int n, std::vector<double>& Ainv);
std::vector<double> prolong_dense(int d, int nc, int& nfb, int& ncb);
bool make_transfer(const std::vector<double>& P, int nfb, int ncb, int off, Transfer1D& T);

// ---- 3D (unit cube) ----------------------------------------------------------------------
// Layout of U on a level with n elements per direction, q = p-1, ni = n+p-2, nq = n+p-1:
//   u_x: (z: nq) x (y: nq) x (x: ni, full indices 1..ni), x fastest; u_y: nq x ni x nq;
//   u_z: ni x nq x nq; p: nq^3; lambda.  Component c is degree p along axis c.
struct Sizes3 {
  int n = 0, p = 0, ni = 0, nq = 0;
  long long n_uc = 0, n_u = 0, n_p = 0, n_total = 0;
};
Sizes3 sizes3(int p, int n);

// Row records of K_l by row class, one table per row kind (u_x, u_y, u_z, p rows); a
// class is the triple of 1D position classes (cls1) of the row's indices.  Every record
// has RU = B0 + 2 B1 + 1 entries: three boxes of neighbours, each "long" along one axis
// (entries ordered long-axis slowest, then axis (c+1)%3, then (c+2)%3 fastest), then the
// lambda coefficient.
//   u_c rows: box 0 = A_cc over u_c (long axis c, offsets -p..p; -q..q across),
//             box 1 = -B_c over p (long axis c, -p..p-1), box 2 = zeros (over p)
//   p rows:   box k = B_k^T over u_k (long axis k, offsets -q..p; -q..q across; box 0
//             holds 2p of its 2p+1 long positions), lambda coefficient m_k last
// B0 = (2p+1)(2q+1)^2, B1 = 2p(2q+1)^2.  Neighbours outside the index range have zero
// coefficients.  cmap[kind][class] -> record index (compact: only classes that occur).
struct Stencils3 {
  int T = 0, NC = 0, B0 = 0, B1 = 0, RU = 0;
  std::vector<int> cmap[4];
  std::vector<double> rec[4];
};

struct LevelHost3 {
  Level1D f;
  Sizes3 sz;
  igamg_sizes pub{};
  PatchTables pt;
  Stencils3 st;
  // generalized Oseen only (empty otherwise): per velocity row, box 0 of the advection part
  // (fine level: assembled; coarse levels: R A P of the level above), and per row (all rows
  // but lambda) the full record = class record + advection, as the kernels read it
  std::vector<double> adv;
  std::vector<double> rows;
  // mapped domains only (empty otherwise): per u_x / u_y row (0 .. 2 n_uc - 1) the
  // 2p x 2p x (2p-1) coefficients coupling it to the other of the two components
  std::vector<double> ext;
};

struct HierarchyHost3 {
  int p = 0, L = 0, n_fine = 0;
  double sigma = 0, nu = 0, cpen = 0;
  std::vector<LevelHost3> lev;
  std::vector<Transfer1D> tp_free, tq;
  std::vector<double> coarse_inv;
  int ndof0 = 0;
  int G = 0;
  std::vector<double> lv_p, lv_q, quad_x;
  // mapped domains: physical quadrature points (3, nG, nG, nG) [component][z][y][x] and
  // J^T there, (nG^3, 3, 3) [.][k][i] = dX_i/dxi_k (the load is int (J^T f) . v_hat)
  int geometry = 0;
  std::vector<double> quad_xyz, jt;
};

int build_hierarchy3(const igamg_problem& pr, HierarchyHost3& H, std::string& err);
// the finest level's 1D factors and row records only (no patches, transfers, coarse inverse)
int build_level_only3(const igamg_problem& pr, HierarchyHost3& H, std::string& err);
double k_entry3(const Level1D& L, const Sizes3& s, long long g1, long long g2);
// entry (g1, g2) evaluated from the row records, as the GPU kernels do
double k_entry3_records(const LevelHost3& lv, int p, long long g1, long long g2);
// the full hierarchy without patch tables and coarse inverse (host inspection of operators)
int build_operators3(const igamg_problem& pr, HierarchyHost3& H, std::string& err);

}  // namespace igamg
