// Host-side set-up of the multigrid hierarchy (Sec. 4-5 of arXiv 1705.09282), in FP64.
//
// Route taken here (different from a plain 2D assembly on purpose): on the unit square
// with constant sigma, nu every block of K is a sum of Kronecker products of 1D banded
// matrices, so each level keeps only its 1D factors.  Coarse operators are the Galerkin
// products R K P of Sec. 5.1; for this bilinear form they equal the same form on the
// coarse spline space with the Nitsche penalty of the finest mesh (the coarse space is a
// subspace of the fine one and every integral is exact), which is how they are built.
// Knot-insertion prolongations (Sec. 4.4) are obtained by collocation at the fine
// Greville abscissae (Schoenberg-Whitney), not by inserting knots one at a time.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <atomic>
#include <map>
#include <thread>
#include <utility>

#include "igamg3d.h"
#include "igamg_internal.h"

namespace igamg {

void Band::add(int i, int j, double x) {
  int d = j - i + hw;
  if (i < 0 || i >= rows || j < 0 || j >= cols || d < 0 || d > 2 * hw) {
    if (x != 0.0) std::fprintf(stderr, "igamg: band overflow (%d,%d)\n", i, j);
    return;
  }
  v[(size_t)i * (2 * hw + 1) + d] += x;
}

// ---- shared helpers (also used by the 3D set-up) ----

std::vector<double> knots(int d, int n) {
  std::vector<double> t(n + 2 * d + 1);
  for (int k = 0; k < (int)t.size(); ++k) {
    int m = k - d;
    t[k] = m <= 0 ? 0.0 : (m >= n ? 1.0 : (double)m / n);
  }
  return t;
}

// Values of the d+1 B-splines that are nonzero on knot span s (t_s <= x <= t_{s+1}),
// i.e. N_{s-d..s}(x), by the triangular form of the Cox-de Boor recursion (Sec. 4.2).
void span_values(const std::vector<double>& t, int d, int s, double x, double* N) {
  double left[8], right[8];
  N[0] = 1.0;
  for (int j = 1; j <= d; ++j) {
    left[j] = x - t[s + 1 - j];
    right[j] = t[s + j] - x;
    double carry = 0.0;
    for (int r = 0; r < j; ++r) {
      double tmp = N[r] / (right[r + 1] + left[j - r]);
      N[r] = carry + right[r + 1] * tmp;
      carry = left[j - r] * tmp;
    }
    N[j] = carry;
  }
}

// Derivatives of N_{s-d..s} on span s: N'_{i,d} = d/(t_{i+d}-t_i) N_{i,d-1} - d/(t_{i+d+1}-t_{i+1}) N_{i+1,d-1}.
void span_derivs(const std::vector<double>& t, int d, int s, double x, double* dN) {
  if (d == 0) { dN[0] = 0.0; return; }
  double Nl[8];
  span_values(t, d - 1, s, x, Nl);  // N_{s-d+1..s, d-1}
  for (int k = 0; k <= d; ++k) {
    int i = s - d + k;
    double a = 0.0, b = 0.0;
    if (k >= 1) { double h = t[i + d] - t[i]; if (h > 0) a = d / h * Nl[k - 1]; }
    if (k <= d - 1) { double h = t[i + d + 1] - t[i + 1]; if (h > 0) b = d / h * Nl[k]; }
    dN[k] = a - b;
  }
}

// Gauss-Legendre rule with m points on [0,1] (Newton on the Legendre recurrence).
void gauss01(int m, std::vector<double>& x, std::vector<double>& w) {
  x.resize(m); w.resize(m);
  for (int i = 0; i < m; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= m; ++k) { double pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = pk; }
      if (m == 1) { p1 = z; p0 = 1.0; }
      dp = m * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= m; ++k) { double pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = pk; }
    dp = m * (z * p1 - p0) / (z * z - 1.0);
    x[m - 1 - i] = 0.5 * (z + 1.0);
    w[m - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2/((1-z^2) P'^2)) / 2
  }
}

// In-place LU with partial pivoting of a dense n x n row-major matrix; returns false on
// a pivot below tol * max|entry|.
bool lu_inplace(std::vector<double>& A, int n, std::vector<int>& piv) {
  double amax = 0.0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int r = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > std::fabs(A[(size_t)r * n + k])) r = i;
    piv[k] = r;
    if (!(std::fabs(A[(size_t)r * n + k]) > 1e-14 * amax)) return false;
    if (r != k) for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)r * n + j]);
    double inv = 1.0 / A[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] * inv;
      A[(size_t)i * n + k] = l;
      if (l != 0.0)
        for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return true;
}

void lu_solve(const std::vector<double>& LU, const std::vector<int>& piv, int n, double* b) {
  for (int k = 0; k < n; ++k) { std::swap(b[k], b[piv[k]]); }
  for (int i = 1; i < n; ++i) { double s = b[i]; for (int j = 0; j < i; ++j) s -= LU[(size_t)i * n + j] * b[j]; b[i] = s; }
  for (int i = n - 1; i >= 0; --i) { double s = b[i]; for (int j = i + 1; j < n; ++j) s -= LU[(size_t)i * n + j] * b[j]; b[i] = s / LU[(size_t)i * n + i]; }
}

// Explicit inverse via LU; false if singular.
bool invert(std::vector<double> A, int n, std::vector<double>& Ainv) {
  std::vector<int> piv;
  if (!lu_inplace(A, n, piv)) return false;
  Ainv.assign((size_t)n * n, 0.0);
  std::vector<double> col(n);
  for (int j = 0; j < n; ++j) {
    std::fill(col.begin(), col.end(), 0.0);
    col[j] = 1.0;
    lu_solve(A, piv, n, col.data());
    for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + j] = col[i];
  }
  return true;
}



// 1D factors on n elements (all integrals by (p+2)-point Gauss, exact for these polynomials).
void build_level1d(int p, int n, double sigma, double nu, double pen_over_nu, Level1D& L) {
  const int q = p - 1;
  L.n = n; L.p = p; L.q = q;
  auto tp = knots(p, n), tq = knots(q, n);
  std::vector<double> gx, gw;
  gauss01(p + 2, gx, gw);
  Band Mp, Sp, Sq, Wq;
  Mp.init(n + p, n + p, p); Sp.init(n + p, n + p, p);
  L.Mq.init(n + q, n + q, p); Sq.init(n + q, n + q, p); Wq.init(n + q, n + q, p);
  L.D.init(n + p, n + q, p);
  const double h = 1.0 / n;
  for (int e = 0; e < n; ++e) {
    for (int g = 0; g < (int)gx.size(); ++g) {
      double x = (e + gx[g]) * h, w = gw[g] * h;
      double Np[8], dNp[8], Nq[8], dNq[8];
      span_values(tp, p, e + p, x, Np); span_derivs(tp, p, e + p, x, dNp);
      span_values(tq, q, e + q, x, Nq); span_derivs(tq, q, e + q, x, dNq);
      for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= p; ++b) {
          Mp.add(e + a, e + b, w * Np[a] * Np[b]);
          Sp.add(e + a, e + b, w * dNp[a] * dNp[b]);
        }
      for (int a = 0; a <= q; ++a)
        for (int b = 0; b <= q; ++b) {
          L.Mq.add(e + a, e + b, w * Nq[a] * Nq[b]);
          Sq.add(e + a, e + b, w * dNq[a] * dNq[b]);
        }
      for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= q; ++b) L.D.add(e + a, e + b, w * dNp[a] * Nq[b]);
    }
  }
  // Nitsche wall terms for the tangential component, Sec. 3.3, per unit nu:
  //   sum over walls x0 in {0,1} with outward normal s = -1 / +1:
  //   -s (N_i N_j' + N_i' N_j)(x0) + (C_I / h_fine) N_i(x0) N_j(x0)
  for (int wall = 0; wall < 2; ++wall) {
    double x0 = wall ? 1.0 : 0.0, s = wall ? 1.0 : -1.0;
    int span = wall ? (n - 1 + q) : q;
    double Nq[8], dNq[8];
    span_values(tq, q, span, x0, Nq); span_derivs(tq, q, span, x0, dNq);
    int base = span - q;
    for (int a = 0; a <= q; ++a)
      for (int b = 0; b <= q; ++b)
        Wq.add(base + a, base + b, -s * (Nq[a] * dNq[b] + dNq[a] * Nq[b]) + pen_over_nu * Nq[a] * Nq[b]);
  }
  L.X1.init(n + p, n + p, p); L.X2.init(n + p, n + p, p); L.Y2.init(n + q, n + q, p);
  for (size_t k = 0; k < Mp.v.size(); ++k) {
    L.X1.v[k] = sigma * Mp.v[k] + nu * Sp.v[k];
    L.X2.v[k] = nu * Mp.v[k];
  }
  for (size_t k = 0; k < Sq.v.size(); ++k) L.Y2.v[k] = Sq.v[k] + Wq.v[k];
  L.mq.resize(n + q);
  for (int k = 0; k < n + q; ++k) L.mq[k] = (tq[k + q + 1] - tq[k]) / (q + 1);
  L.dcoef.resize(n + q);
  for (int k = 1; k <= n + q; ++k) L.dcoef[k - 1] = p / (tp[k + p] - tp[k]);
}



// Dense 1D prolongation (fine x coarse) for midpoint refinement, by collocation.
std::vector<double> prolong_dense(int d, int nc, int& nfb, int& ncb) {
  int nf = 2 * nc;
  nfb = nf + d; ncb = nc + d;
  auto tf = knots(d, nf), tc = knots(d, nc);
  std::vector<double> Bf((size_t)nfb * nfb, 0.0), Bc((size_t)nfb * ncb, 0.0);
  for (int r = 0; r < nfb; ++r) {
    double g = 0.0;
    if (d == 0) g = (tf[r] + tf[r + 1]) / 2;
    else { for (int k = 1; k <= d; ++k) g += tf[r + k]; g /= d; }
    int sf = std::min(std::max((int)std::floor(g * nf), 0), nf - 1) + d;
    int sc = std::min(std::max((int)std::floor(g * nc), 0), nc - 1) + d;
    double N[8];
    span_values(tf, d, sf, g, N);
    for (int k = 0; k <= d; ++k) Bf[(size_t)r * nfb + sf - d + k] = N[k];
    span_values(tc, d, sc, g, N);
    for (int k = 0; k <= d; ++k) Bc[(size_t)r * ncb + sc - d + k] = N[k];
  }
  std::vector<int> piv;
  if (!lu_inplace(Bf, nfb, piv)) return {};
  std::vector<double> P((size_t)nfb * ncb), col(nfb);
  for (int j = 0; j < ncb; ++j) {
    for (int r = 0; r < nfb; ++r) col[r] = Bc[(size_t)r * ncb + j];
    lu_solve(Bf, piv, nfb, col.data());
    for (int r = 0; r < nfb; ++r) P[(size_t)r * ncb + j] = std::fabs(col[r]) < 1e-13 ? 0.0 : col[r];
  }
  return P;
}

bool make_transfer(const std::vector<double>& P, int nfb, int ncb, int off, Transfer1D& T) {
  // view rows/cols [off, nfb-off) x [off, ncb-off)
  T.nf = nfb - 2 * off; T.nc = ncb - 2 * off;
  T.c0.assign(T.nf, 0); T.pv.assign((size_t)T.nf * Transfer1D::WP, 0.0);
  T.f0.assign(T.nc, 0); T.rv.assign((size_t)T.nc * Transfer1D::WR, 0.0);
  auto at = [&](int f, int c) { return P[(size_t)(f + off) * ncb + (c + off)]; };
  // entries outside the view must vanish (interior coarse functions do not touch the
  // fine boundary functions)
  if (off) for (int c = 0; c < T.nc; ++c) { if (P[(size_t)0 * ncb + c + off] != 0.0 || P[(size_t)(nfb - 1) * ncb + c + off] != 0.0) return false; }
  for (int f = 0; f < T.nf; ++f) {
    int first = -1, last = -1;
    for (int c = 0; c < T.nc; ++c) if (at(f, c) != 0.0) { if (first < 0) first = c; last = c; }
    if (first < 0) first = last = 0;
    if (last - first + 1 > Transfer1D::WP) return false;
    first = std::min(first, std::max(0, T.nc - Transfer1D::WP));
    T.c0[f] = first;
    for (int k = 0; k < Transfer1D::WP; ++k) { int c = first + k; T.pv[(size_t)f * Transfer1D::WP + k] = (c < T.nc) ? at(f, c) : 0.0; }
  }
  for (int c = 0; c < T.nc; ++c) {
    int first = -1, last = -1;
    for (int f = 0; f < T.nf; ++f) if (at(f, c) != 0.0) { if (first < 0) first = f; last = f; }
    if (first < 0) first = last = 0;
    if (last - first + 1 > Transfer1D::WR) return false;
    first = std::min(first, std::max(0, T.nf - Transfer1D::WR));
    T.f0[c] = first;
    for (int k = 0; k < Transfer1D::WR; ++k) { int f = first + k; T.rv[(size_t)c * Transfer1D::WR + k] = (f < T.nf) ? at(f, c) : 0.0; }
  }
  return true;
}

// ---- DOF numbering and single matrix entries of K_l from the 1D factors ---------------
struct Dof { int blk; int x, y; };  // blk 0 u_x, 1 u_y, 2 p, 3 lambda; x,y = full 1D indices

Dof decode(const igamg_sizes& s, long long g) {
  Dof d{};
  if (g < s.n_ux) { d.blk = 0; d.y = (int)(g / s.nx_ux); d.x = (int)(g % s.nx_ux) + 1; }
  else if (g < s.n_ux + s.n_uy) { long long r = g - s.n_ux; d.blk = 1; d.y = (int)(r / s.nx_uy) + 1; d.x = (int)(r % s.nx_uy); }
  else if (g < s.n_ux + s.n_uy + s.n_p) { long long r = g - s.n_ux - s.n_uy; d.blk = 2; d.y = (int)(r / s.n_pdir); d.x = (int)(r % s.n_pdir); }
  else { d.blk = 3; d.x = d.y = 0; }
  return d;
}

long long gid(const igamg_sizes& s, int blk, int x, int y) {
  switch (blk) {
    case 0: if (x < 1 || x > s.nx_ux) return -1; return (long long)y * s.nx_ux + (x - 1);
    case 1: if (y < 1 || y > s.ny_uy) return -1; return s.n_ux + (long long)(y - 1) * s.nx_uy + x;
    case 2: return s.n_ux + s.n_uy + (long long)y * s.n_pdir + x;
    default: return s.n_total - 1;
  }
}



double k_entry(const Level1D& L, const igamg_sizes& s, long long g1, long long g2) {
  Dof a = decode(s, g1), b = decode(s, g2);
  auto m = [&](const Dof& d) { return L.mq[d.x] * L.mq[d.y]; };
  if (a.blk == 0 && b.blk == 0) return L.X1.get(a.x, b.x) * L.Mq.get(a.y, b.y) + L.X2.get(a.x, b.x) * L.Y2.get(a.y, b.y);
  if (a.blk == 1 && b.blk == 1) return L.Mq.get(a.x, b.x) * L.X1.get(a.y, b.y) + L.Y2.get(a.x, b.x) * L.X2.get(a.y, b.y);
  if (a.blk == 0 && b.blk == 2) return -L.D.get(a.x, b.x) * L.Mq.get(a.y, b.y);
  if (a.blk == 1 && b.blk == 2) return -L.Mq.get(a.x, b.x) * L.D.get(a.y, b.y);
  if (a.blk == 2 && b.blk == 0) return L.D.get(b.x, a.x) * L.Mq.get(b.y, a.y);
  if (a.blk == 2 && b.blk == 1) return L.Mq.get(b.x, a.x) * L.D.get(b.y, a.y);
  if (a.blk == 2 && b.blk == 3) return m(a);
  if (a.blk == 3 && b.blk == 2) return m(b);
  return 0.0;
}

namespace {


// ---- general per-row operators (generalized Oseen) ----------------------------------------
// Record index of column c in the stencil record of row r (layout of Stencils), or -1.
int box_index(int p, const Dof& r, const Dof& c) {
  const int q = p - 1, WQ = 2 * q + 1, WPP = 2 * p + 1, B0 = WPP * WQ, RU = B0 + 2 * p * WQ + 1;
  int dx = c.x - r.x, dy = c.y - r.y;
  if (r.blk == 0) {
    if (c.blk == 0 && dx >= -p && dx <= p && dy >= -q && dy <= q) return (dx + p) * WQ + dy + q;
    if (c.blk == 2 && dx >= -p && dx <= p - 1 && dy >= -q && dy <= q) return B0 + (dx + p) * WQ + dy + q;
  } else if (r.blk == 1) {
    if (c.blk == 1 && dx >= -q && dx <= q && dy >= -p && dy <= p) return (dx + q) * WPP + dy + p;
    if (c.blk == 2 && dx >= -q && dx <= q && dy >= -p && dy <= p - 1) return B0 + (dx + q) * (2 * p) + dy + p;
  } else if (r.blk == 2) {
    if (c.blk == 0 && dx >= -q && dx <= p && dy >= -q && dy <= q) return (dx + q) * WQ + dy + q;
    if (c.blk == 1 && dx >= -q && dx <= q && dy >= -q && dy <= p) return B0 + (dx + q) * (2 * p) + dy + q;
    if (c.blk == 3) return RU - 1;
  }
  return -1;
}

// Inverse of box_index: the column of record entry e of row r (blk = -1 if none / outside).
Dof box_col(const igamg_sizes& s, int p, const Dof& r, int e) {
  const int q = p - 1, WQ = 2 * q + 1, WPP = 2 * p + 1, B0 = WPP * WQ, RU = B0 + 2 * p * WQ + 1;
  const int nint = s.n + p - 2, lastq = s.n + q - 1;
  Dof c{-1, 0, 0};
  auto ok_free = [&](int v) { return v >= 1 && v <= nint; };
  auto ok_q = [&](int v) { return v >= 0 && v <= lastq; };
  if (e == RU - 1) { if (r.blk == 2) c.blk = 3; return c; }
  if (r.blk == 0) {
    if (e < B0) { c = {0, r.x + e / WQ - p, r.y + e % WQ - q}; if (!ok_free(c.x) || !ok_q(c.y)) c.blk = -1; }
    else { int f = e - B0; c = {2, r.x + f / WQ - p, r.y + f % WQ - q}; if (!ok_q(c.x) || !ok_q(c.y)) c.blk = -1; }
  } else if (r.blk == 1) {
    if (e < B0) { c = {1, r.x + e / WPP - q, r.y + e % WPP - p}; if (!ok_q(c.x) || !ok_free(c.y)) c.blk = -1; }
    else { int f = e - B0; c = {2, r.x + f / (2 * p) - q, r.y + f % (2 * p) - p}; if (!ok_q(c.x) || !ok_q(c.y)) c.blk = -1; }
  } else if (r.blk == 2) {
    if (e < B0) {
      if (e >= 2 * p * WQ) return c;
      c = {0, r.x + e / WQ - q, r.y + e % WQ - q}; if (!ok_free(c.x) || !ok_q(c.y)) c.blk = -1;
    } else { int f = e - B0; c = {1, r.x + f / (2 * p) - q, r.y + f % (2 * p) - q}; if (!ok_q(c.x) || !ok_free(c.y)) c.blk = -1; }
  }
  return c;
}

// Per-row records of a level given by its class stencils (the Stokes part).
void rows_from_classes(int p, const LevelHost& lv, std::vector<double>& rows) {
  const Stencils& st = lv.st;
  const int n = lv.sz.n, RU = st.RU, NC = st.NC, T = st.T;
  const int lastp = n + p - 1, lastq = n + p - 2;
  long long nr = lv.sz.n_total - 1;
  rows.assign((size_t)nr * RU, 0.0);
  for (long long g = 0; g < nr; ++g) {
    Dof d = decode(lv.sz, g);
    const double* src;
    if (d.blk == 0) src = &st.sx[(size_t)(cls1(d.x, lastp, T) * NC + cls1(d.y, lastq, T)) * RU];
    else if (d.blk == 1) src = &st.sy[(size_t)(cls1(d.x, lastq, T) * NC + cls1(d.y, lastp, T)) * RU];
    else src = &st.sp[(size_t)(cls1(d.x, lastq, T) * NC + cls1(d.y, lastq, T)) * RU];
    std::copy(src, src + RU, &rows[(size_t)g * RU]);
  }
}

// + int v . (beta . grad u) for both velocity blocks (Sec. 3.1, generalized Oseen), beta at
// the (p+2)-point Gauss points, layout (2, n*G, n*G) [component][y point][x point].
void add_advection(int p, const LevelHost& lv, const double* beta, std::vector<double>& rows) {
  const int q = p - 1, n = lv.sz.n, G = p + 2, nG = n * G;
  const int WQ = 2 * q + 1, WPP = 2 * p + 1, RU = WPP * WQ + 2 * p * WQ + 1;
  std::vector<double> gx, gw;
  gauss01(G, gx, gw);
  auto tp = knots(p, n), tq = knots(q, n);
  const double* bxs = beta;
  const double* bys = beta + (size_t)nG * nG;
  for (int ey = 0; ey < n; ++ey)
    for (int ex = 0; ex < n; ++ex)
      for (int gyi = 0; gyi < G; ++gyi)
        for (int gxi = 0; gxi < G; ++gxi) {
          double x = (ex + gx[gxi]) / n, y = (ey + gx[gyi]) / n, w = gw[gxi] * gw[gyi] / ((double)n * n);
          double bx = bxs[(size_t)(ey * G + gyi) * nG + ex * G + gxi], by = bys[(size_t)(ey * G + gyi) * nG + ex * G + gxi];
          double Npx[8], dNpx[8], Nqx[8], dNqx[8], Npy[8], dNpy[8], Nqy[8], dNqy[8];
          span_values(tp, p, ex + p, x, Npx); span_derivs(tp, p, ex + p, x, dNpx);
          span_values(tq, q, ex + q, x, Nqx); span_derivs(tq, q, ex + q, x, dNqx);
          span_values(tp, p, ey + p, y, Npy); span_derivs(tp, p, ey + p, y, dNpy);
          span_values(tq, q, ey + q, y, Nqy); span_derivs(tq, q, ey + q, y, dNqy);
          for (int a = 0; a <= p; ++a)          // u_x: degree p in x, q in y
            for (int b = 0; b <= q; ++b) {
              long long g = gid(lv.sz, 0, ex + a, ey + b);
              if (g < 0) continue;
              double phi = w * Npx[a] * Nqy[b];
              for (int a2 = 0; a2 <= p; ++a2)
                for (int b2 = 0; b2 <= q; ++b2) {
                  if (gid(lv.sz, 0, ex + a2, ey + b2) < 0) continue;
                  double adv = bx * dNpx[a2] * Nqy[b2] + by * Npx[a2] * dNqy[b2];
                  rows[(size_t)g * RU + (a2 - a + p) * WQ + (b2 - b + q)] += phi * adv;
                }
            }
          for (int a = 0; a <= q; ++a)          // u_y: degree q in x, p in y
            for (int b = 0; b <= p; ++b) {
              long long g = gid(lv.sz, 1, ex + a, ey + b);
              if (g < 0) continue;
              double phi = w * Nqx[a] * Npy[b];
              for (int a2 = 0; a2 <= q; ++a2)
                for (int b2 = 0; b2 <= p; ++b2) {
                  if (gid(lv.sz, 1, ex + a2, ey + b2) < 0) continue;
                  double adv = bx * dNqx[a2] * Npy[b2] + by * Nqx[a2] * dNpy[b2];
                  rows[(size_t)g * RU + (a2 - a + q) * WPP + (b2 - b + p)] += phi * adv;
                }
            }
        }
}

// ---- mapped domains (Sec. 4.3 push-forwards; Sec. 6.2's quarter annulus) ----------------
// Third record box of a velocity row: its coupling to the other velocity component,
// 2p x 2p entries.  u_x row (x, y) -> u_y column (x + dx, y + dy), dx in [-p, q],
// dy in [-q, p]; u_y row -> u_x column, dx in [-q, p], dy in [-p, q].
int ext_index(int p, const Dof& r, const Dof& c) {
  const int q = p - 1, W = 2 * p;
  const int dx = c.x - r.x, dy = c.y - r.y;
  if (r.blk == 0 && c.blk == 1 && dx >= -p && dx <= q && dy >= -q && dy <= p) return (dx + p) * W + dy + q;
  if (r.blk == 1 && c.blk == 0 && dx >= -q && dx <= p && dy >= -p && dy <= q) return (dx + q) * W + dy + p;
  return -1;
}

Dof ext_col(const igamg_sizes& s, int p, const Dof& r, int e) {
  const int q = p - 1, W = 2 * p, nint = s.n + p - 2, lastq = s.n + q - 1;
  Dof c{-1, 0, 0};
  if (r.blk == 0) {
    c = {1, r.x + e / W - p, r.y + e % W - q};
    if (c.x < 0 || c.x > lastq || c.y < 1 || c.y > nint) c.blk = -1;
  } else if (r.blk == 1) {
    c = {0, r.x + e / W - q, r.y + e % W - p};
    if (c.x < 1 || c.x > nint || c.y < 0 || c.y > lastq) c.blk = -1;
  }
  return c;
}

// F(xi, eta) = r(xi) C(eta), r = ri + (ro - ri) xi, C the rational quadratic Bezier quarter
// circle (control points (1,0), (1,1), (0,1), weights 1, 1/sqrt(2), 1).  X[i], DF[i][k] =
// dX_i/dxi_k, D2[i][k][l] = d^2 X_i / dxi_k dxi_l.
void annulus_map(double ri, double ro, double xi, double eta, double X[2], double DF[2][2], double D2[2][2][2]) {
  const double w = std::sqrt(0.5), t = eta, u = 1.0 - eta;
  // homogeneous numerator N(t) and weight W(t) with their derivatives
  const double Nx = u * u + w * 2 * t * u, Ny = w * 2 * t * u + t * t;
  const double dNx = -2 * u + w * (2 - 4 * t), dNy = w * (2 - 4 * t) + 2 * t;
  const double ddNx = 2 - 4 * w, ddNy = -4 * w + 2;
  const double Wt = u * u + w * 2 * t * u + t * t, dW = -2 * u + w * (2 - 4 * t) + 2 * t, ddW = 4 - 4 * w;
  const double C[2] = {Nx / Wt, Ny / Wt};
  const double A[2] = {dNx * Wt - Nx * dW, dNy * Wt - Ny * dW};          // C' = A / W^2
  const double dA[2] = {ddNx * Wt - Nx * ddW, ddNy * Wt - Ny * ddW};
  double dC[2], ddC[2];
  for (int i = 0; i < 2; ++i) {
    dC[i] = A[i] / (Wt * Wt);
    ddC[i] = dA[i] / (Wt * Wt) - 2 * A[i] * dW / (Wt * Wt * Wt);
  }
  const double dr = ro - ri, r = ri + dr * xi;
  for (int i = 0; i < 2; ++i) {
    X[i] = r * C[i];
    DF[i][0] = dr * C[i];
    DF[i][1] = r * dC[i];
    D2[i][0][0] = 0.0;
    D2[i][0][1] = D2[i][1][0] = dr * dC[i];
    D2[i][1][1] = r * ddC[i];
  }
}

namespace {
// Values and physical gradients of the pushed-forward velocity basis v = N a_c / det J
// (a_c = column c of DF) from the parametric value N and gradient (N_xi, N_eta).
struct Pushed { double v[2], g[2][2], divh; };

inline Pushed push_velocity(double N, double Nxi, double Neta, int c, const double DF[2][2], const double D2[2][2][2],
                            double J, const double dJ[2], const double inv[2][2]) {
  Pushed o;
  const double dN[2] = {Nxi, Neta};
  double G[2][2];                                     // d v_i / d xi_k
  for (int i = 0; i < 2; ++i) {
    const double a = DF[i][c];
    o.v[i] = N * a / J;
    for (int k = 0; k < 2; ++k) G[i][k] = dN[k] * a / J + N * D2[i][c][k] / J - N * a * dJ[k] / (J * J);
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) o.g[i][j] = G[i][0] * inv[0][j] + G[i][1] * inv[1][j];
  o.divh = dN[c];
  return o;
}

struct Geo { double X[2], DF[2][2], D2[2][2][2], J, dJ[2], inv[2][2]; };

inline Geo geo_at(double ri, double ro, double xi, double eta) {
  Geo g;
  annulus_map(ri, ro, xi, eta, g.X, g.DF, g.D2);
  g.J = g.DF[0][0] * g.DF[1][1] - g.DF[0][1] * g.DF[1][0];
  for (int k = 0; k < 2; ++k)
    g.dJ[k] = g.D2[0][0][k] * g.DF[1][1] + g.DF[0][0] * g.D2[1][1][k] - g.D2[0][1][k] * g.DF[1][0] - g.DF[0][1] * g.D2[1][0][k];
  g.inv[0][0] = g.DF[1][1] / g.J; g.inv[0][1] = -g.DF[0][1] / g.J;
  g.inv[1][0] = -g.DF[1][0] / g.J; g.inv[1][1] = g.DF[0][0] / g.J;
  return g;
}

// free velocity functions of element (ex, ey) at one point: global ids and pushed values
struct LocalVel { int n = 0; long long gid[32]; Dof d[32]; Pushed f[32]; };

void local_velocity(const igamg_sizes& sz, int p, int ex, int ey, const std::vector<double>& tp,
                    const std::vector<double>& tq, double xi, double eta, const Geo& G, LocalVel& out) {
  const int q = p - 1;
  double Npx[8], dNpx[8], Nqx[8], dNqx[8], Npy[8], dNpy[8], Nqy[8], dNqy[8];
  span_values(tp, p, ex + p, xi, Npx); span_derivs(tp, p, ex + p, xi, dNpx);
  span_values(tq, q, ex + q, xi, Nqx); span_derivs(tq, q, ex + q, xi, dNqx);
  span_values(tp, p, ey + p, eta, Npy); span_derivs(tp, p, ey + p, eta, dNpy);
  span_values(tq, q, ey + q, eta, Nqy); span_derivs(tq, q, ey + q, eta, dNqy);
  out.n = 0;
  for (int a = 0; a <= p; ++a)                        // u_x: degree p in xi, q in eta
    for (int b = 0; b <= q; ++b) {
      long long g = gid(sz, 0, ex + a, ey + b);
      if (g < 0) continue;
      out.gid[out.n] = g; out.d[out.n] = {0, ex + a, ey + b};
      out.f[out.n++] = push_velocity(Npx[a] * Nqy[b], dNpx[a] * Nqy[b], Npx[a] * dNqy[b], 0, G.DF, G.D2, G.J, G.dJ, G.inv);
    }
  for (int a = 0; a <= q; ++a)                        // u_y: degree q in xi, p in eta
    for (int b = 0; b <= p; ++b) {
      long long g = gid(sz, 1, ex + a, ey + b);
      if (g < 0) continue;
      out.gid[out.n] = g; out.d[out.n] = {1, ex + a, ey + b};
      out.f[out.n++] = push_velocity(Nqx[a] * Npy[b], dNqx[a] * Npy[b], Nqx[a] * dNpy[b], 1, G.DF, G.D2, G.J, G.dJ, G.inv);
    }
}
}  // namespace

// Adds K(row = test gid ti, column = trial gid tj) += val into the level's records.
static void put_entry(int p, const igamg_sizes& sz, std::vector<double>& rows, std::vector<double>& ext,
                      const Dof& r, long long ti, const Dof& c, double val) {
  const int q = p - 1, RU = (2 * p + 1) * (2 * q + 1) + 2 * p * (2 * q + 1) + 1, BX = 4 * p * p;
  int idx = box_index(p, r, c);
  if (idx >= 0) { rows[(size_t)ti * RU + idx] += val; return; }
  idx = ext_index(p, r, c);
  if (idx >= 0) ext[(size_t)ti * BX + idx] += val;
  (void)sz;
}

// Fine-level operator of generalized Stokes on the quarter annulus, in record form:
// sigma (u, v) + nu (grad u, grad v) - (div v, p) + (div u, q) on the physical domain,
// integrated over the parametric square with (p+2)-point Gauss rules; Nitsche terms
// -nu (grad u n).v - nu (grad v n).u + C_I nu / h u.v on the four walls, h = det J /
// (|tangent| n); the multiplier column m_j = int q_j dx = int q_hat_j dxi.  Also fills the
// physical quadrature points and J^T there for the load vector.
void assemble_mapped(int p, LevelHost& lv, double sigma, double nu, double cpen, double ri, double ro,
                     HierarchyHost& H) {
  const int q = p - 1, n = lv.sz.n, G = p + 2, nG = n * G;
  const int RU = (2 * p + 1) * (2 * q + 1) + 2 * p * (2 * q + 1) + 1, BX = 4 * p * p;
  const long long nu_rows = lv.sz.n_ux + lv.sz.n_uy, nr = lv.sz.n_total - 1;
  lv.rows.assign((size_t)nr * RU, 0.0);
  lv.ext.assign((size_t)nu_rows * BX, 0.0);
  std::vector<double> gx, gw;
  gauss01(G, gx, gw);
  auto tp = knots(p, n), tq = knots(q, n);
  auto& rows = lv.rows;
  auto& ext = lv.ext;
  // volume terms: an element row ey writes only the records of functions with y index in
  // [ey, ey + p], so element rows p + 2 apart never share a record; p + 2 sequential phases,
  // each spreading its element rows (ey = phase mod p + 2) over the threads
  unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  const int phases = p + 2;
  for (int ph = 0; ph < phases; ++ph) {
    std::vector<int> eys;
    for (int ey = ph; ey < n; ey += phases) eys.push_back(ey);
    auto work = [&](size_t i0, size_t i1) {
      LocalVel lvv;
      for (size_t ii = i0; ii < i1; ++ii) {
        const int ey = eys[ii];
        for (int ex = 0; ex < n; ++ex)
          for (int gyi = 0; gyi < G; ++gyi)
            for (int gxi = 0; gxi < G; ++gxi) {
              const double xi = (ex + gx[gxi]) / n, eta = (ey + gx[gyi]) / n;
              const double w = gw[gxi] * gw[gyi] / ((double)n * n);
              Geo g = geo_at(ri, ro, xi, eta);
              local_velocity(lv.sz, p, ex, ey, tp, tq, xi, eta, g, lvv);
              double Nqx[8], Nqy[8];
              span_values(tq, q, ex + q, xi, Nqx);
              span_values(tq, q, ey + q, eta, Nqy);
              const double wJ = w * g.J;
              for (int i = 0; i < lvv.n; ++i) {
                const Pushed& a = lvv.f[i];
                for (int j = 0; j < lvv.n; ++j) {
                  const Pushed& b = lvv.f[j];
                  double m = sigma * (a.v[0] * b.v[0] + a.v[1] * b.v[1]);
                  double k = a.g[0][0] * b.g[0][0] + a.g[0][1] * b.g[0][1] + a.g[1][0] * b.g[1][0] + a.g[1][1] * b.g[1][1];
                  put_entry(p, lv.sz, rows, ext, lvv.d[i], lvv.gid[i], lvv.d[j], wJ * (m + nu * k));
                }
                // b(v, q) = int div v q dx = int divhat vhat qhat / det J dxi
                for (int ka = 0; ka <= q; ++ka)
                  for (int kb = 0; kb <= q; ++kb) {
                    const long long gq = gid(lv.sz, 2, ex + ka, ey + kb);
                    const Dof dq{2, ex + ka, ey + kb};
                    const double bval = w * a.divh * Nqx[ka] * Nqy[kb] / g.J;
                    put_entry(p, lv.sz, rows, ext, lvv.d[i], lvv.gid[i], dq, -bval);
                    put_entry(p, lv.sz, rows, ext, dq, gq, lvv.d[i], bval);
                  }
              }
            }
      }
    };
    std::vector<std::thread> th;
    size_t chunk = (eys.size() + nth - 1) / nth;
    for (unsigned t = 0; t < nth; ++t) {
      size_t i0 = t * chunk, i1 = std::min(eys.size(), i0 + chunk);
      if (i0 < i1) th.emplace_back(work, i0, i1);
    }
    for (auto& t : th) t.join();
  }
  // Nitsche terms on the four walls (k = 0: xi = const walls, k = 1: eta = const walls)
  const double pen_c = cpen * nu;
  LocalVel lvv;
  for (int wall = 0; wall < 4; ++wall) {
    const int k = wall / 2, side = wall % 2;
    for (int e = 0; e < n; ++e)
      for (int gi = 0; gi < G; ++gi) {
        const double t = (e + gx[gi]) / n, wt = gw[gi] / n;
        const double xi = k == 0 ? (double)side : t, eta = k == 0 ? t : (double)side;
        const int ex = k == 0 ? (side ? n - 1 : 0) : e, ey = k == 0 ? e : (side ? n - 1 : 0);
        Geo g = geo_at(ri, ro, xi, eta);
        local_velocity(lv.sz, p, ex, ey, tp, tq, xi, eta, g, lvv);
        double nv[2] = {g.inv[k][0], g.inv[k][1]};    // gradient of xi_k
        double nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1]);
        const double sgn = side ? 1.0 : -1.0;
        nv[0] *= sgn / nn; nv[1] *= sgn / nn;
        const double tl = std::sqrt(g.DF[0][1 - k] * g.DF[0][1 - k] + g.DF[1][1 - k] * g.DF[1][1 - k]);
        const double ds = wt * tl, h = g.J / (tl * n);
        for (int i = 0; i < lvv.n; ++i) {
          const Pushed& a = lvv.f[i];
          const double dna[2] = {a.g[0][0] * nv[0] + a.g[0][1] * nv[1], a.g[1][0] * nv[0] + a.g[1][1] * nv[1]};
          for (int j = 0; j < lvv.n; ++j) {
            const Pushed& b = lvv.f[j];
            const double dnb[2] = {b.g[0][0] * nv[0] + b.g[0][1] * nv[1], b.g[1][0] * nv[0] + b.g[1][1] * nv[1]};
            const double val = ds * (-nu * (dnb[0] * a.v[0] + dnb[1] * a.v[1]) - nu * (dna[0] * b.v[0] + dna[1] * b.v[1])
                                     + pen_c / h * (a.v[0] * b.v[0] + a.v[1] * b.v[1]));
            put_entry(p, lv.sz, rows, ext, lvv.d[i], lvv.gid[i], lvv.d[j], val);
          }
        }
      }
  }
  // multiplier column of the pressure rows
  for (long long g = lv.sz.n_ux + lv.sz.n_uy; g < nr; ++g) {
    Dof d = decode(lv.sz, g);
    rows[(size_t)g * RU + RU - 1] = lv.f.mq[d.x] * lv.f.mq[d.y];
  }
  // physical quadrature points and J^T for the load vector
  H.quad_xy.assign((size_t)2 * nG * nG, 0.0);
  H.jt.assign((size_t)4 * nG * nG, 0.0);
  for (int iy = 0; iy < nG; ++iy)
    for (int ix = 0; ix < nG; ++ix) {
      const double xi = (ix / G + gx[ix % G]) / n, eta = (iy / G + gx[iy % G]) / n;
      double X[2], DF[2][2], D2[2][2][2];
      annulus_map(ri, ro, xi, eta, X, DF, D2);
      const size_t o = (size_t)iy * nG + ix;
      H.quad_xy[o] = X[0];
      H.quad_xy[(size_t)nG * nG + o] = X[1];
      for (int kk = 0; kk < 2; ++kk)
        for (int i = 0; i < 2; ++i) H.jt[o * 4 + kk * 2 + i] = DF[i][kk];
    }
}

// K_c = P^T K_f P (Sec. 5.1) in per-row stencil form.  P is block diagonal with tensor
// products of the 1D knot-insertion views tp (degree p, interior indices) and tq.
int galerkin_rows(int p, const LevelHost& F, const LevelHost& C, const Transfer1D& tp, const Transfer1D& tq,
                  std::vector<double>& out, std::string& err, std::vector<double>* out_ext = nullptr) {
  const int q = p - 1, RU = (2 * p + 1) * (2 * q + 1) + 2 * p * (2 * q + 1) + 1, BX = 4 * p * p;
  const int WR = Transfer1D::WR, WP = Transfer1D::WP;
  long long nC = C.sz.n_total - 1;
  out.assign((size_t)nC * RU, 0.0);
  const bool has_ext = !F.ext.empty() && out_ext;
  if (has_ext) out_ext->assign((size_t)(C.sz.n_ux + C.sz.n_uy) * BX, 0.0);
  std::atomic<int> bad{0};
  auto work = [&](long long i0, long long i1) {
    for (long long i = i0; i < i1; ++i) {
      Dof ri = decode(C.sz, i);
      const Transfer1D& TX = ri.blk == 0 ? tp : tq;
      const Transfer1D& TY = ri.blk == 1 ? tp : tq;
      int sx = ri.blk == 0 ? 1 : 0, sy = ri.blk == 1 ? 1 : 0;   // view index = full - shift
      int cxv = ri.x - sx, cyv = ri.y - sy;
      double* orow = &out[(size_t)i * RU];
      double* oext = (has_ext && ri.blk < 2) ? &(*out_ext)[(size_t)i * BX] : nullptr;
      for (int kx = 0; kx < WR; ++kx) {
        int fxv = TX.f0[cxv] + kx;
        double wx = TX.rv[(size_t)cxv * WR + kx];
        if (wx == 0.0 || fxv >= TX.nf) continue;
        for (int ky = 0; ky < WR; ++ky) {
          int fyv = TY.f0[cyv] + ky;
          double wy = TY.rv[(size_t)cyv * WR + ky];
          if (wy == 0.0 || fyv >= TY.nf) continue;
          long long a = gid(F.sz, ri.blk, fxv + sx, fyv + sy);
          Dof ra = decode(F.sz, a);
          const double* frow = &F.rows[(size_t)a * RU];
          const double* fext = (has_ext && ra.blk < 2) ? &F.ext[(size_t)a * BX] : nullptr;
          double wa = wx * wy;
          double fscale = 0.0;
          for (int e = 0; e < RU; ++e) fscale = std::max(fscale, std::fabs(frow[e]));
          if (fext) for (int e = 0; e < BX; ++e) fscale = std::max(fscale, std::fabs(fext[e]));
          const int ne = fext ? RU + BX : RU;
          for (int e = 0; e < ne; ++e) {
            double val = e < RU ? frow[e] : fext[e - RU];
            if (val == 0.0) continue;
            Dof cb = e < RU ? box_col(F.sz, p, ra, e) : ext_col(F.sz, p, ra, e - RU);
            if (cb.blk < 0) continue;
            if (cb.blk == 3) { orow[RU - 1] += wa * val; continue; }
            const Transfer1D& JX = cb.blk == 0 ? tp : tq;
            const Transfer1D& JY = cb.blk == 1 ? tp : tq;
            int jsx = cb.blk == 0 ? 1 : 0, jsy = cb.blk == 1 ? 1 : 0;
            int bxv = cb.x - jsx, byv = cb.y - jsy;
            for (int jx = 0; jx < WP; ++jx) {
              int cjx = JX.c0[bxv] + jx;
              double wjx = JX.pv[(size_t)bxv * WP + jx];
              if (wjx == 0.0 || cjx >= JX.nc) continue;
              for (int jy = 0; jy < WP; ++jy) {
                int cjy = JY.c0[byv] + jy;
                double wjy = JY.pv[(size_t)byv * WP + jy];
                if (wjy == 0.0 || cjy >= JY.nc) continue;
                Dof cj{cb.blk, cjx + jsx, cjy + jsy};
                int idx = box_index(p, ri, cj);
                if (idx < 0 && oext) {
                  int ie = ext_index(p, ri, cj);
                  if (ie >= 0) { oext[ie] += wa * val * wjx * wjy; continue; }
                }
                if (idx < 0) {
                  // only round-off may fall outside the pattern (exact zeros in exact
                  // arithmetic can come out as tiny numbers where the compiler contracts
                  // a*b+c into one fused multiply-add, e.g. on aarch64)
                  if (std::fabs(val) > 1e-12 * fscale) bad = 1;
                  continue;
                }
                orow[idx] += wa * val * wjx * wjy;
              }
            }
          }
        }
      }
    }
  };
  unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  long long chunk = (nC + nth - 1) / nth;
  for (unsigned t = 0; t < nth; ++t) {
    long long i0 = t * chunk, i1 = std::min(nC, i0 + chunk);
    if (i0 < i1) th.emplace_back(work, i0, i1);
  }
  for (auto& t : th) t.join();
  if (bad) { err = "Galerkin product left the coarse stencil pattern"; return IGAMG_EINVAL; }
  return IGAMG_OK;
}

// 1D position class of a patch index a on n+p-2 interior positions: the first and last
// T positions are their own classes, the rest share the translation-invariant class.
int pos_class(int a, int n, int p) {
  const int T = 2 * p + 2;
  int last = n + p - 2;
  if (a < T) return a;
  if (last - a < T) return T + (last - a);
  return 2 * T;
}

template <typename Entry>
int build_patches(int p, const Level1D& L, const igamg_sizes& s, PatchTables& pt, std::string& err, Entry kent,
                  bool per_patch) {
  const int n = L.n, q = p - 1;
  auto sup = [&](int i, int d) { return std::make_pair(std::max(0, i - d), std::min(n - 1, i)); };
  auto inside = [](std::pair<int, int> a, std::pair<int, int> box) { return box.first <= a.first && a.second <= box.second; };
  struct P { int a, b, colour; std::vector<int> dofs; int nv, nq; };
  std::vector<P> all;
  int np1 = p + 1;
  for (int b = 1; b <= n + p - 2; ++b)
    for (int a = 1; a <= n + p - 2; ++a) {
      P P_; P_.a = a; P_.b = b; P_.colour = (b % np1) * np1 + (a % np1);
      auto bx = sup(a, p), by = sup(b, p);
      for (int y = std::max(0, b - p - 1); y <= std::min(n + q - 1, b + p + 1); ++y)
        for (int x = std::max(1, a - p - 1); x <= std::min(n + p - 2, a + p + 1); ++x)
          if (inside(sup(x, p), bx) && inside(sup(y, q), by)) P_.dofs.push_back((int)gid(s, 0, x, y));
      for (int y = std::max(1, b - p - 1); y <= std::min(n + p - 2, b + p + 1); ++y)
        for (int x = std::max(0, a - p - 1); x <= std::min(n + q - 1, a + p + 1); ++x)
          if (inside(sup(x, q), bx) && inside(sup(y, p), by)) P_.dofs.push_back((int)gid(s, 1, x, y));
      P_.nv = (int)P_.dofs.size();
      for (int y = std::max(0, b - p - 1); y <= std::min(n + q - 1, b + p + 1); ++y)
        for (int x = std::max(0, a - p - 1); x <= std::min(n + q - 1, a + p + 1); ++x)
          if (inside(sup(x, q), bx) && inside(sup(y, q), by)) P_.dofs.push_back((int)gid(s, 2, x, y));
      P_.nq = (int)P_.dofs.size() - P_.nv;
      all.push_back(std::move(P_));
    }
  // colour-major; inside a colour the 4+4-DOF patches first, then the larger wall
  // patches, each group lexicographic in (b, a).  The order inside a colour does not
  // change the result: same-colour patches share no DOF and are not coupled by K.
  std::stable_sort(all.begin(), all.end(), [](const P& x, const P& y) {
    if (x.colour != y.colour) return x.colour < y.colour;
    return (x.dofs.size() != 8) < (y.dofs.size() != 8); });
  int maxl = 0;
  for (auto& P_ : all) maxl = std::max(maxl, (int)P_.dofs.size());
  pt.n_patches = (int)all.size(); pt.maxl = maxl; pt.n_colours = np1 * np1;
  pt.dofs.assign((size_t)pt.n_patches * maxl, -1);
  pt.cls.assign(pt.n_patches, 0);
  pt.pos.assign(pt.n_patches, 0);
  pt.colour_off.assign(pt.n_colours + 1, 0);
  // classes: patches whose local matrices are equal share one inverse (translation
  // invariance of the constant-coefficient Stokes operator); with per_patch every patch
  // has its own.  8-DOF patches index the packed 8 x 8 table, the others the maxl table.
  std::map<std::pair<int, int>, int> cmap8, cmapg;
  std::vector<int> rep8, repg;
  for (int i = 0; i < pt.n_patches; ++i) {
    auto& P_ = all[i];
    for (size_t k = 0; k < P_.dofs.size(); ++k) pt.dofs[(size_t)i * maxl + k] = P_.dofs[k];
    pt.pos[i] = P_.a | (P_.b << 16);
    pt.colour_off[P_.colour + 1]++;
    bool is8 = P_.dofs.size() == 8;
    auto& cmap = is8 ? cmap8 : cmapg;
    auto& rep = is8 ? rep8 : repg;
    auto key = per_patch ? std::make_pair(P_.a, P_.b) : std::make_pair(pos_class(P_.a, n, p), pos_class(P_.b, n, p));
    auto it = cmap.find(key);
    if (it == cmap.end()) { int id = (int)rep.size(); cmap[key] = id; rep.push_back(i); pt.cls[i] = id; }
    else pt.cls[i] = it->second;
  }
  for (int c = 0; c < pt.n_colours; ++c) pt.colour_off[c + 1] += pt.colour_off[c];
  pt.n8.assign(pt.n_colours, 0);
  for (int c = 0; c < pt.n_colours; ++c)
    for (int k = pt.colour_off[c]; k < pt.colour_off[c + 1] && all[k].dofs.size() == 8; ++k) pt.n8[c]++;
  {
    // support of a basis function of degree d with index i on n elements: [i - d, i] clipped
    auto sup = [&](long long g, int* lo, int* hi) {
      const Dof r = decode(s, g);
      const int dx = r.blk == 0 ? p : q, dy = r.blk == 1 ? p : q;
      lo[0] = std::max(0, r.x - dx); hi[0] = std::min(n - 1, r.x);
      lo[1] = std::max(0, r.y - dy); hi[1] = std::min(n - 1, r.y);
      lo[2] = hi[2] = 0;
    };
    const int ne[3] = {n, n, 1};
    if (!validate_patch_tables(pt, s.n_total - 1, err, sup, ne)) return IGAMG_EINVAL;
  }
  // bordered local inverses, one per class (Sec. 5.2 local problems; zero-mean local
  // pressure through the border m_j = int N^q_j)
  auto local_inverse = [&](const P& P_, std::vector<double>& inv) -> bool {
    int nl = (int)P_.dofs.size(), nb = nl + 1;
    std::vector<double> Kb((size_t)nb * nb, 0.0);
    for (int r = 0; r < nl; ++r)
      for (int t = 0; t < nl; ++t) Kb[(size_t)r * nb + t] = kent(P_.dofs[r], P_.dofs[t]);
    for (int r = P_.nv; r < nl; ++r) {
      Dof d = decode(s, P_.dofs[r]);
      double m = L.mq[d.x] * L.mq[d.y];
      Kb[(size_t)r * nb + nl] = m; Kb[(size_t)nl * nb + r] = m;
    }
    return invert(Kb, nb, inv);
  };
  pt.n_cls = (int)repg.size();
  pt.n_cls8 = (int)rep8.size();
  pt.nloc.assign(std::max(pt.n_cls, 1), 0);
  pt.cinv.assign((size_t)std::max(pt.n_cls, 1) * maxl * maxl, 0.0);
  pt.cinv8.assign((size_t)std::max(pt.n_cls8, 1) * 64, 0.0);
  for (int c = 0; c < pt.n_cls; ++c) {
    auto& P_ = all[repg[c]];
    int nl = (int)P_.dofs.size(), nb = nl + 1;
    std::vector<double> inv;
    if (!local_inverse(P_, inv)) { err = "singular local patch matrix"; return IGAMG_ESINGULAR; }
    pt.nloc[c] = nl;
    for (int r = 0; r < nl; ++r)
      for (int t = 0; t < nl; ++t) pt.cinv[((size_t)c * maxl + r) * maxl + t] = inv[(size_t)r * nb + t];
  }
  for (int c = 0; c < pt.n_cls8; ++c) {
    std::vector<double> inv;
    if (!local_inverse(all[rep8[c]], inv)) { err = "singular local patch matrix"; return IGAMG_ESINGULAR; }
    for (int r = 0; r < 8; ++r)
      for (int t = 0; t < 8; ++t) pt.cinv8[(size_t)c * 64 + r * 8 + t] = inv[(size_t)r * 9 + t];
  }
  // dof -> (patch, local row) lists for the additive smoother, patch order ascending
  long long nd = s.n_total;
  pt.d2p_off.assign(nd + 1, 0);
  for (int i = 0; i < pt.n_patches; ++i)
    for (int k = 0; k < maxl; ++k) { int g = pt.dofs[(size_t)i * maxl + k]; if (g >= 0) pt.d2p_off[g + 1]++; }
  for (long long g = 0; g < nd; ++g) pt.d2p_off[g + 1] += pt.d2p_off[g];
  pt.d2p_idx.assign(pt.d2p_off[nd], 0);
  std::vector<int> fill(pt.d2p_off.begin(), pt.d2p_off.end() - 1);
  // the additive update sums corrections in the lexicographic patch order (b, then a)
  std::vector<int> lex(pt.n_patches);
  for (int i = 0; i < pt.n_patches; ++i) lex[i] = i;
  std::sort(lex.begin(), lex.end(), [&](int x, int y) {
    return all[x].b != all[y].b ? all[x].b < all[y].b : all[x].a < all[y].a; });
  for (int i : lex)
    for (int k = 0; k < maxl; ++k) { int g = pt.dofs[(size_t)i * maxl + k]; if (g >= 0) pt.d2p_idx[fill[g]++] = i * maxl + k; }
  return IGAMG_OK;
}

}  // namespace

void build_row_slots(PatchTables& pt) {
  const int maxl = pt.maxl;
  // 128-slot blocks where the patches allow (twice the blocks: a colour spreads more evenly
  // over the SMs); IGAMG_ROW_SLOTS = 256 keeps 256
  const char* env = std::getenv("IGAMG_ROW_SLOTS");
  const int smin = env && std::atoi(env) == 256 ? 256 : 128;
  pt.row_slots = maxl <= smin ? smin : (maxl <= 256 ? 256 : (maxl <= 1024 ? 1024 : 0));
  const int S = pt.row_slots;
  if (!S) return;
  // classes packed nl x nl: general classes first (their nl from nloc), then the 8-DOF ones
  pt.cinv_off.assign(pt.n_cls + pt.n_cls8 + 1, 0);
  for (int c = 0; c < pt.n_cls; ++c) pt.cinv_off[c + 1] = pt.cinv_off[c] + (long long)pt.nloc[c] * pt.nloc[c];
  for (int c = 0; c < pt.n_cls8; ++c) pt.cinv_off[pt.n_cls + c + 1] = pt.cinv_off[pt.n_cls + c] + 64;
  pt.cinv_all.assign((size_t)pt.cinv_off.back(), 0.0);
  for (int c = 0; c < pt.n_cls; ++c) {
    const int nl = pt.nloc[c];
    for (int r = 0; r < nl; ++r)
      for (int t = 0; t < nl; ++t)
        pt.cinv_all[pt.cinv_off[c] + (size_t)r * nl + t] = pt.cinv[((size_t)c * maxl + r) * maxl + t];
  }
  for (int c = 0; c < pt.n_cls8; ++c)
    std::copy(pt.cinv8.begin() + (size_t)c * 64, pt.cinv8.begin() + (size_t)(c + 1) * 64,
              pt.cinv_all.begin() + pt.cinv_off[pt.n_cls + c]);
  pt.slot_g.clear(); pt.slot_c.clear(); pt.slot_kb.clear();
  pt.colour_blk.assign(pt.n_colours + 1, 0);
  auto pad_block = [&]() {
    while (pt.slot_g.size() % S) { pt.slot_g.push_back(-1); pt.slot_c.push_back(0); pt.slot_kb.push_back(0u); }
  };
  for (int col = 0; col < pt.n_colours; ++col) {
    pt.colour_blk[col] = (int)(pt.slot_g.size() / S);
    for (int i = pt.colour_off[col]; i < pt.colour_off[col + 1]; ++i) {
      const bool is8 = i - pt.colour_off[col] < pt.n8[col];
      const int cls = is8 ? pt.n_cls + pt.cls[i] : pt.cls[i];
      const int nl = is8 ? 8 : pt.nloc[pt.cls[i]];
      if ((int)(pt.slot_g.size() % S) + nl > S) pad_block();
      const unsigned base = (unsigned)(pt.slot_g.size() % S);
      for (int k = 0; k < nl; ++k) {
        pt.slot_g.push_back(pt.dofs[(size_t)i * maxl + k]);
        pt.slot_c.push_back(cls);
        pt.slot_kb.push_back((unsigned)k | ((unsigned)nl << 10) | (base << 20));
      }
    }
    pad_block();
  }
  pt.colour_blk[pt.n_colours] = (int)(pt.slot_g.size() / S);
}

double k_entry_rows(const LevelHost& lv, int p, long long g1, long long g2) {
  const int q = p - 1, RU = (2 * p + 1) * (2 * q + 1) + 2 * p * (2 * q + 1) + 1, BX = 4 * p * p;
  Dof a = decode(lv.sz, g1), b = decode(lv.sz, g2);
  if (a.blk == 3) return b.blk == 2 ? lv.rows[(size_t)g2 * RU + RU - 1] : 0.0;
  int idx = box_index(p, a, b);
  if (idx >= 0) return lv.rows[(size_t)g1 * RU + idx];
  if (!lv.ext.empty()) {
    idx = ext_index(p, a, b);
    if (idx >= 0) return lv.ext[(size_t)g1 * BX + idx];
  }
  return 0.0;
}

bool validate_patch_tables(const PatchTables& pt, long long n_rows, std::string& err,
                           const std::function<void(long long, int*, int*)>& support, const int* n_elem) {
  std::vector<int> stamp((size_t)n_rows, -1);
  const size_t ne = (size_t)n_elem[0] * n_elem[1] * n_elem[2];
  std::vector<int> cover(support ? ne : 0, -1), cover_col(support ? ne : 0, -1);
  for (int c = 0; c < pt.n_colours; ++c)
    for (int i = pt.colour_off[c]; i < pt.colour_off[c + 1]; ++i) {
      int blo[3] = {1 << 30, 1 << 30, 1 << 30}, bhi[3] = {-1, -1, -1};
      for (int k = 0; k < pt.maxl; ++k) {
        const long long g = pt.dofs[(size_t)i * pt.maxl + k];
        if (g < 0) continue;                                    // padding
        if (g >= n_rows) { err = "patch table: DOF id out of range"; return false; }
        if (stamp[(size_t)g] == c) { err = "patch table: a DOF twice in one colour"; return false; }
        stamp[(size_t)g] = c;
        if (support) {
          int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
          support(g, lo, hi);
          for (int d = 0; d < 3; ++d) { blo[d] = std::min(blo[d], lo[d]); bhi[d] = std::max(bhi[d], hi[d]); }
        }
      }
      if (!support || bhi[0] < 0) continue;
      for (int d = 0; d < 3; ++d)
        if (blo[d] < 0 || bhi[d] >= n_elem[d]) { err = "patch table: a DOF support outside the mesh"; return false; }
      for (int z = blo[2]; z <= bhi[2]; ++z)
        for (int y = blo[1]; y <= bhi[1]; ++y)
          for (int x = blo[0]; x <= bhi[0]; ++x) {
            const size_t e = ((size_t)z * n_elem[1] + y) * n_elem[0] + x;
            if (cover_col[e] == c && cover[e] != i) {
              err = "patch table: two patches of colour " + std::to_string(c) + " share element (" +
                    std::to_string(x) + ", " + std::to_string(y) + ", " + std::to_string(z) +
                    "), so they may be coupled through K";
              return false;
            }
            cover_col[e] = c;
            cover[e] = i;
          }
    }
  return true;
}

void build_tile_tables(const PatchTables& pt, int nint, int tw, TileTables& tt) {
  tt.tw = tw;
  tt.ntx = tt.nty = (nint + tw - 1) / tw;
  const int C = pt.n_colours, nt = tt.ntx * tt.nty;
  std::vector<std::vector<int>> run((size_t)nt * C);
  tt.n8.assign((size_t)nt * C, 0);
  for (int c = 0; c < C; ++c)
    for (int i = pt.colour_off[c]; i < pt.colour_off[c + 1]; ++i) {   // table order: 8-DOF first
      const int a = pt.pos[i] & 0xffff, b = pt.pos[i] >> 16;
      const int t = ((b - 1) / tw) * tt.ntx + (a - 1) / tw;
      run[(size_t)t * C + c].push_back(i);
      if (i < pt.colour_off[c] + pt.n8[c]) tt.n8[(size_t)t * C + c]++;
    }
  tt.off.assign((size_t)nt * C + 1, 0);
  tt.list.clear();
  tt.list.reserve(pt.n_patches);
  for (size_t r = 0; r < run.size(); ++r) {
    tt.list.insert(tt.list.end(), run[r].begin(), run[r].end());
    tt.off[r + 1] = (int)tt.list.size();
  }
}

igamg_sizes level_sizes(int p, int n) {
  igamg_sizes s{};
  int q = p - 1;
  s.n = n;
  s.nx_ux = n + p - 2; s.ny_ux = n + q;
  s.nx_uy = n + q; s.ny_uy = n + p - 2;
  s.n_pdir = n + q;
  s.n_ux = (long long)s.nx_ux * s.ny_ux;
  s.n_uy = (long long)s.nx_uy * s.ny_uy;
  s.n_p = (long long)s.n_pdir * s.n_pdir;
  s.n_total = s.n_ux + s.n_uy + s.n_p + 1;
  s.n_patches = (n + p - 2) * (n + p - 2);
  s.n_colours = (p + 1) * (p + 1);
  s.n_quad = p + 2;
  s.dim = 2;
  s.n_uz = 0;
  return s;
}

void build_stencils(int p, const Level1D& L, const igamg_sizes& s, Stencils& st) {
  const int q = p - 1, n = L.n;
  st.T = 2 * p + 1;
  st.NC = 2 * st.T + 1;
  st.B0 = (2 * p + 1) * (2 * q + 1);
  st.B1 = 2 * p * (2 * q + 1);
  st.RU = st.B0 + st.B1 + 1;
  const int T = st.T, NC = st.NC, B0 = st.B0, RU = st.RU;
  const int lastp = n + p - 1, lastq = n + q - 1, nint = n + p - 2;
  st.sx.assign((size_t)NC * NC * RU, 0.0);
  st.sy.assign((size_t)NC * NC * RU, 0.0);
  st.sp.assign((size_t)NC * NC * RU, 0.0);
  std::vector<char> done(NC * NC);
  auto inq = [&](int k) { return k >= 0 && k <= lastq; };
  auto inp_free = [&](int k) { return k >= 1 && k <= nint; };
  std::fill(done.begin(), done.end(), 0);
  for (int iy = 0; iy <= lastq; ++iy)
    for (int ix = 1; ix <= nint; ++ix) {
      int c = cls1(ix, lastp, T) * NC + cls1(iy, lastq, T);
      if (done[c]) continue;
      done[c] = 1;
      double* r = &st.sx[(size_t)c * RU];
      for (int dx = -p; dx <= p; ++dx)
        for (int dy = -q; dy <= q; ++dy) {
          int jx = ix + dx, jy = iy + dy;
          if (inp_free(jx) && inq(jy))
            r[(dx + p) * (2 * q + 1) + dy + q] = L.X1.get(ix, jx) * L.Mq.get(iy, jy) + L.X2.get(ix, jx) * L.Y2.get(iy, jy);
        }
      for (int kx = -p; kx <= p - 1; ++kx)
        for (int dy = -q; dy <= q; ++dy) {
          int jx = ix + kx, jy = iy + dy;
          if (inq(jx) && inq(jy)) r[B0 + (kx + p) * (2 * q + 1) + dy + q] = -L.D.get(ix, jx) * L.Mq.get(iy, jy);
        }
    }
  std::fill(done.begin(), done.end(), 0);
  for (int iy = 1; iy <= nint; ++iy)
    for (int ix = 0; ix <= lastq; ++ix) {
      int c = cls1(ix, lastq, T) * NC + cls1(iy, lastp, T);
      if (done[c]) continue;
      done[c] = 1;
      double* r = &st.sy[(size_t)c * RU];
      for (int dx = -q; dx <= q; ++dx)
        for (int dy = -p; dy <= p; ++dy) {
          int jx = ix + dx, jy = iy + dy;
          if (inq(jx) && inp_free(jy))
            r[(dx + q) * (2 * p + 1) + dy + p] = L.Mq.get(ix, jx) * L.X1.get(iy, jy) + L.Y2.get(ix, jx) * L.X2.get(iy, jy);
        }
      for (int dx = -q; dx <= q; ++dx)
        for (int ky = -p; ky <= p - 1; ++ky) {
          int jx = ix + dx, jy = iy + ky;
          if (inq(jx) && inq(jy)) r[B0 + (dx + q) * (2 * p) + ky + p] = -L.Mq.get(ix, jx) * L.D.get(iy, jy);
        }
    }
  std::fill(done.begin(), done.end(), 0);
  for (int ky = 0; ky <= lastq; ++ky)
    for (int kx = 0; kx <= lastq; ++kx) {
      int c = cls1(kx, lastq, T) * NC + cls1(ky, lastq, T);
      if (done[c]) continue;
      done[c] = 1;
      double* r = &st.sp[(size_t)c * RU];
      for (int sI = -q; sI <= p; ++sI)
        for (int dy = -q; dy <= q; ++dy) {
          int ix = kx + sI, iy = ky + dy;
          if (inp_free(ix) && inq(iy)) r[(sI + q) * (2 * q + 1) + dy + q] = L.D.get(ix, kx) * L.Mq.get(iy, ky);
        }
      for (int dx = -q; dx <= q; ++dx)
        for (int sI = -q; sI <= p; ++sI) {
          int ix = kx + dx, iy = ky + sI;
          if (inq(ix) && inp_free(iy)) r[B0 + (dx + q) * (2 * p) + sI + q] = L.Mq.get(ix, kx) * L.D.get(iy, ky);
        }
      r[RU - 1] = L.mq[kx] * L.mq[ky];
    }
  (void)s;
}

int build_hierarchy(const igamg_problem& pr, HierarchyHost& H, std::string& err) {
  const int p = pr.p, L = pr.n_levels, nf = pr.n_fine;
  H.p = p; H.L = L; H.n_fine = nf; H.sigma = pr.sigma; H.nu = pr.nu;
  H.cpen = pr.c_penalty > 0 ? pr.c_penalty : 4.0 * (p - 1);
  const double pen_over_nu = H.cpen * nf;  // C_I / h_fine on every level
  H.lev.resize(L);
  const bool mapped = pr.geometry == IGAMG_GEOM_QUARTER_ANNULUS;
  const bool general = pr.beta_qp != nullptr || mapped;   // Oseen, mapped: per-row operators
  H.geometry = pr.geometry;
  for (int l = 0; l < L; ++l) {
    int n = nf >> (L - 1 - l);
    auto& lv = H.lev[l];
    build_level1d(p, n, pr.sigma, pr.nu, pen_over_nu, lv.f);
    lv.sz = level_sizes(p, n);
    build_stencils(p, lv.f, lv.sz, lv.st);
  }
  H.tp_free.resize(L); H.tq.resize(L);
  for (int l = 1; l < L; ++l) {
    int nc = nf >> (L - l);
    int a, b;
    auto Pp = prolong_dense(p, nc, a, b);
    if (Pp.empty() || !make_transfer(Pp, a, b, 1, H.tp_free[l])) { err = "degree-p prolongation"; return IGAMG_ESINGULAR; }
    auto Pq = prolong_dense(p - 1, nc, a, b);
    if (Pq.empty() || !make_transfer(Pq, a, b, 0, H.tq[l])) { err = "degree-(p-1) prolongation"; return IGAMG_ESINGULAR; }
  }
  if (general) {
    // fine level: the Stokes part from the class stencils plus the advection term, or the
    // operator on the mapped domain; coarse levels: Galerkin products (neither the advection
    // field nor the map is polynomial, so re-assembly would not equal R K P)
    if (mapped) {
      const double ri = pr.r_inner > 0 ? pr.r_inner : 0.075, ro = pr.r_outer > 0 ? pr.r_outer : 0.225;
      assemble_mapped(p, H.lev[L - 1], pr.sigma, pr.nu, H.cpen, ri, ro, H);
    } else {
      rows_from_classes(p, H.lev[L - 1], H.lev[L - 1].rows);
      add_advection(p, H.lev[L - 1], pr.beta_qp, H.lev[L - 1].rows);
    }
    for (int l = L - 2; l >= 0; --l) {
      int rc = galerkin_rows(p, H.lev[l + 1], H.lev[l], H.tp_free[l + 1], H.tq[l + 1], H.lev[l].rows, err,
                             mapped ? &H.lev[l].ext : nullptr);
      if (rc) return rc;
    }
  }
  for (int l = 1; l < L; ++l) {
    auto& lv = H.lev[l];
    int rc = general ? build_patches(p, lv.f, lv.sz, lv.pt, err,
                                     [&](long long a, long long b) { return k_entry_rows(lv, p, a, b); }, true)
                     : build_patches(p, lv.f, lv.sz, lv.pt, err,
                                     [&](long long a, long long b) { return k_entry(lv.f, lv.sz, a, b); }, false);
    if (rc) return rc;
  }
  // coarsest matrix, dense, and its inverse
  {
    auto& lv = H.lev[0];
    int nd = (int)lv.sz.n_total;
    std::vector<double> K((size_t)nd * nd);
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) K[(size_t)i * nd + j] = general ? k_entry_rows(lv, p, i, j) : k_entry(lv.f, lv.sz, i, j);
    if (!invert(K, nd, H.coarse_inv)) { err = "singular coarsest matrix"; return IGAMG_ESINGULAR; }
    H.ndof0 = nd;
  }
  // matrix-free advection tables of the finest level (generalized Oseen on the square)
  if (pr.beta_qp && !mapped) {
    const int G = p + 2, q = p - 1, nG = nf * G;
    std::vector<double> gx, gw;
    gauss01(G, gx, gw);
    auto tp = knots(p, nf), tq = knots(q, nf);
    H.adv_bp.assign((size_t)nf * (p + 1) * G, 0.0); H.adv_dp.assign(H.adv_bp.size(), 0.0);
    H.adv_bq.assign((size_t)nf * (q + 1) * G, 0.0); H.adv_dq.assign(H.adv_bq.size(), 0.0);
    for (int e = 0; e < nf; ++e)
      for (int g = 0; g < G; ++g) {
        const double x = (e + gx[g]) / nf;
        double N[8], dN[8];
        span_values(tp, p, e + p, x, N); span_derivs(tp, p, e + p, x, dN);
        for (int a = 0; a <= p; ++a) {
          H.adv_bp[((size_t)e * (p + 1) + a) * G + g] = N[a];
          H.adv_dp[((size_t)e * (p + 1) + a) * G + g] = dN[a];
        }
        span_values(tq, q, e + q, x, N); span_derivs(tq, q, e + q, x, dN);
        for (int a = 0; a <= q; ++a) {
          H.adv_bq[((size_t)e * (q + 1) + a) * G + g] = N[a];
          H.adv_dq[((size_t)e * (q + 1) + a) * G + g] = dN[a];
        }
      }
    H.adv_beta.assign((size_t)2 * nG * nG, 0.0);
    for (int c = 0; c < 2; ++c)
      for (int iy = 0; iy < nG; ++iy)
        for (int ix = 0; ix < nG; ++ix) {
          const size_t k = (size_t)c * nG * nG + (size_t)iy * nG + ix;
          H.adv_beta[k] = gw[ix % G] * gw[iy % G] / ((double)nf * nf) * pr.beta_qp[k];
        }
  }
  // load-vector tables on the finest level
  {
    const int G = p + 2, q = p - 1;
    H.G = G;
    std::vector<double> gx, gw;
    gauss01(G, gx, gw);
    auto tp = knots(p, nf), tq = knots(q, nf);
    H.lv_p.assign((size_t)(nf + p) * (p + 1) * G, 0.0);
    H.lv_q.assign((size_t)(nf + q) * (q + 1) * G, 0.0);
    H.quad_x.resize((size_t)nf * G);
    for (int e = 0; e < nf; ++e)
      for (int g = 0; g < G; ++g) {
        double x = (e + gx[g]) / nf, w = gw[g] / nf;
        H.quad_x[(size_t)e * G + g] = x;
        double N[8];
        span_values(tp, p, e + p, x, N);
        for (int a = 0; a <= p; ++a) { int i = e + a; int k = e - (i - p); H.lv_p[((size_t)i * (p + 1) + k) * G + g] = w * N[a]; }
        span_values(tq, q, e + q, x, N);
        for (int a = 0; a <= q; ++a) { int i = e + a; int k = e - (i - q); H.lv_q[((size_t)i * (q + 1) + k) * G + g] = w * N[a]; }
      }
  }
  return IGAMG_OK;
}

}  // namespace igamg

// ---- host-only inspection entry points -----------------------------------------------
namespace {
int host_build(const igamg_problem* prob, int level, igamg::HierarchyHost& H) {
  if (!prob || prob->dim != 2 || (prob->p != 2 && prob->p != 3)) return IGAMG_EUNSUPPORTED;
  if (!(prob->sigma > 0) || !(prob->nu > 0)) return IGAMG_EINVAL;
  if (prob->n_levels < 1 || prob->n_fine < 1 || prob->n_fine % (1 << (prob->n_levels - 1))) return IGAMG_EINVAL;
  if (level < 0 || level >= prob->n_levels) return IGAMG_EINVAL;
  if (prob->geometry < IGAMG_GEOM_SQUARE || prob->geometry > IGAMG_GEOM_QUARTER_ANNULUS) return IGAMG_EINVAL;
  if (prob->geometry == IGAMG_GEOM_QUARTER_ANNULUS && prob->beta_qp) return IGAMG_EUNSUPPORTED;
  if (igamg::level_sizes(prob->p, prob->n_fine >> (prob->n_levels - 1)).n_total > 4096) return IGAMG_EINVAL;
  std::string err;
  return igamg::build_hierarchy(*prob, H, err);
}
}  // namespace

extern "C" int igamg_host_level_matrix(const igamg_problem* prob, int level, double* K, size_t cap,
                                       long long* n_out) {
  if (prob && prob->dim == 3) return igamg::host_level_matrix3(prob, level, K, cap, n_out, false);
  igamg::HierarchyHost H;
  int rc = host_build(prob, level, H);
  if (rc) return rc;
  const auto& lv = H.lev[level];
  long long n = lv.sz.n_total;
  if (n_out) *n_out = n;
  if (!K) return IGAMG_OK;
  if (cap < (size_t)(n * n)) return IGAMG_EINVAL;
  for (long long i = 0; i < n; ++i)
    for (long long j = 0; j < n; ++j)
      K[i * n + j] = lv.rows.empty() ? igamg::k_entry(lv.f, lv.sz, i, j) : igamg::k_entry_rows(lv, prob->p, i, j);
  return IGAMG_OK;
}

extern "C" int igamg_host_prolongation(const igamg_problem* prob, int level, double* P, size_t cap,
                                       long long* n_rows, long long* n_cols) {
  if (prob && prob->dim == 3) return igamg::host_prolongation3(prob, level, P, cap, n_rows, n_cols);
  if (level < 1) return IGAMG_EINVAL;
  igamg::HierarchyHost H;
  int rc = host_build(prob, level, H);
  if (rc) return rc;
  const auto& f = H.lev[level].sz;
  const auto& c = H.lev[level - 1].sz;
  long long nr = f.n_total, nc = c.n_total;
  if (n_rows) *n_rows = nr;
  if (n_cols) *n_cols = nc;
  if (!P) return IGAMG_OK;
  if (cap < (size_t)(nr * nc)) return IGAMG_EINVAL;
  std::fill(P, P + nr * nc, 0.0);
  const auto& tp = H.tp_free[level];
  const auto& tq = H.tq[level];
  auto put = [&](long long roff, long long coff, int fnx, int cnx, const igamg::Transfer1D& TX,
                 const igamg::Transfer1D& TY) {
    for (int fy = 0; fy < TY.nf; ++fy)
      for (int fx = 0; fx < TX.nf; ++fx)
        for (int ky = 0; ky < igamg::Transfer1D::WP; ++ky)
          for (int kx = 0; kx < igamg::Transfer1D::WP; ++kx) {
            int cy = TY.c0[fy] + ky, cx = TX.c0[fx] + kx;
            if (cy >= TY.nc || cx >= TX.nc) continue;
            double w = TY.pv[(size_t)fy * igamg::Transfer1D::WP + ky] * TX.pv[(size_t)fx * igamg::Transfer1D::WP + kx];
            if (w != 0.0) P[(roff + (long long)fy * fnx + fx) * nc + coff + (long long)cy * cnx + cx] += w;
          }
  };
  put(0, 0, f.nx_ux, c.nx_ux, tp, tq);
  put(f.n_ux, c.n_ux, f.nx_uy, c.nx_uy, tq, tp);
  put(f.n_ux + f.n_uy, c.n_ux + c.n_uy, f.n_pdir, c.n_pdir, tq, tq);
  P[(nr - 1) * nc + nc - 1] = 1.0;
  return IGAMG_OK;
}

extern "C" int igamg_host_patches(const igamg_problem* prob, int level, int* colour, int* dofs,
                                  size_t cap_patches, size_t cap_dofs, int* n_patches, int* maxl) {
  if (prob && prob->dim == 3)
    return igamg::host_patches3(prob, level, colour, dofs, cap_patches, cap_dofs, n_patches, maxl);
  if (level < 1) return IGAMG_EINVAL;
  igamg::HierarchyHost H;
  int rc = host_build(prob, level, H);
  if (rc) return rc;
  const auto& pt = H.lev[level].pt;
  if (n_patches) *n_patches = pt.n_patches;
  if (maxl) *maxl = pt.maxl;
  if (colour) {
    if (cap_patches < (size_t)pt.n_patches) return IGAMG_EINVAL;
    for (int c = 0; c < pt.n_colours; ++c)
      for (int k = pt.colour_off[c]; k < pt.colour_off[c + 1]; ++k) colour[k] = c;
  }
  if (dofs) {
    if (cap_dofs < pt.dofs.size()) return IGAMG_EINVAL;
    std::copy(pt.dofs.begin(), pt.dofs.end(), dofs);
  }
  return IGAMG_OK;
}

