// Host-side set-up of the 3D (unit cube) hierarchy: Sec. 4.3 compatible spaces in 3D,
// Sec. 5.1 transfers and coarse operators, Sec. 5.2 subdomains = supports of the
// vector-potential basis functions.
//
// As in 2D every block of K is a sum of Kronecker products of the same 1D banded factors
// (Level1D), now with three factors:
//   A_cc = X1 (c) Mq (a) Mq (b) + X2 (c) Y2 (a) Mq (b) + X2 (c) Mq (a) Y2 (b),
//   B_c  = D (c) Mq (a) Mq (b),   m = mq (x) mq (x) mq,
// where c is the component's own axis (degree p) and a, b the two others (degree q).
// Coarse operators are re-assembled with the finest-mesh Nitsche penalty, which equals
// R K P for this bilinear form (the coarse space is a subspace and every integral is exact).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <map>
#include <thread>
#include <tuple>

#include "igamg_internal.h"

namespace igamg {

Sizes3 sizes3(int p, int n) {
  Sizes3 s;
  s.n = n; s.p = p; s.ni = n + p - 2; s.nq = n + p - 1;
  s.n_uc = (long long)s.ni * s.nq * s.nq;
  s.n_u = 3 * s.n_uc;
  s.n_p = (long long)s.nq * s.nq * s.nq;
  s.n_total = s.n_u + s.n_p + 1;
  return s;
}

namespace {

struct Dof3 { int blk; int i[3]; };   // blk 0..2 u_c, 3 p, 4 lambda; i = full 1D indices (x, y, z)

inline int dim_of(const Sizes3& s, int blk, int axis) { return (blk < 3 && axis == blk) ? s.ni : s.nq; }

Dof3 decode3(const Sizes3& s, long long g) {
  Dof3 d{};
  if (g < s.n_u) {
    d.blk = (int)(g / s.n_uc);
    long long r = g - d.blk * s.n_uc;
    int dx = dim_of(s, d.blk, 0), dy = dim_of(s, d.blk, 1);
    d.i[0] = (int)(r % dx); d.i[1] = (int)((r / dx) % dy); d.i[2] = (int)(r / ((long long)dx * dy));
    d.i[d.blk] += 1;
  } else if (g < s.n_u + s.n_p) {
    long long r = g - s.n_u;
    d.blk = 3;
    d.i[0] = (int)(r % s.nq); d.i[1] = (int)((r / s.nq) % s.nq); d.i[2] = (int)(r / ((long long)s.nq * s.nq));
  } else {
    d.blk = 4;
  }
  return d;
}

// global id of (blk, full indices) or -1 outside the free index range
long long gid3(const Sizes3& s, int blk, const int* i) {
  if (blk == 4) return s.n_total - 1;
  int loc[3];
  for (int a = 0; a < 3; ++a) {
    loc[a] = i[a] - ((blk < 3 && a == blk) ? 1 : 0);
    if (loc[a] < 0 || loc[a] >= dim_of(s, blk, a)) return -1;
  }
  long long base = blk < 3 ? blk * s.n_uc : s.n_u;
  return base + ((long long)loc[2] * dim_of(s, blk, 1) + loc[1]) * dim_of(s, blk, 0) + loc[0];
}

}  // namespace

double k_entry3(const Level1D& L, const Sizes3& s, long long g1, long long g2) {
  Dof3 a = decode3(s, g1), b = decode3(s, g2);
  if (a.blk < 3 && b.blk == a.blk) {
    int c = a.blk, o1 = (c + 1) % 3, o2 = (c + 2) % 3;
    double m1 = L.Mq.get(a.i[o1], b.i[o1]), m2 = L.Mq.get(a.i[o2], b.i[o2]);
    return L.X1.get(a.i[c], b.i[c]) * m1 * m2 +
           L.X2.get(a.i[c], b.i[c]) * (L.Y2.get(a.i[o1], b.i[o1]) * m2 + m1 * L.Y2.get(a.i[o2], b.i[o2]));
  }
  if (a.blk < 3 && b.blk == 3) {
    int c = a.blk, o1 = (c + 1) % 3, o2 = (c + 2) % 3;
    return -L.D.get(a.i[c], b.i[c]) * L.Mq.get(a.i[o1], b.i[o1]) * L.Mq.get(a.i[o2], b.i[o2]);
  }
  if (a.blk == 3 && b.blk < 3) {
    int c = b.blk, o1 = (c + 1) % 3, o2 = (c + 2) % 3;
    return L.D.get(b.i[c], a.i[c]) * L.Mq.get(b.i[o1], a.i[o1]) * L.Mq.get(b.i[o2], a.i[o2]);
  }
  if (a.blk == 3 && b.blk == 4) return L.mq[a.i[0]] * L.mq[a.i[1]] * L.mq[a.i[2]];
  if (a.blk == 4 && b.blk == 3) return L.mq[b.i[0]] * L.mq[b.i[1]] * L.mq[b.i[2]];
  return 0.0;
}

namespace {

// Description of box k of a row of kind `kind` (see Stencils3): column block, long axis,
// long-axis origin offset and length.
struct Box3 { int blk, axis, org, len; };
Box3 box_of(int p, int kind, int k) {
  const int q = p - 1;
  if (kind < 3) {
    if (k == 0) return {kind, kind, -p, 2 * p + 1};
    return {3, kind, -p, 2 * p};           // k = 2 is a zero box over p
  }
  return {k, k, -q, 2 * p};
}

int box_start(int p, int k) {
  const int q = p - 1, W = 2 * q + 1;
  return k == 0 ? 0 : (2 * p + 1) * W * W + (k - 1) * 2 * p * W * W;
}

// record of the row at full indices i of kind `kind`
void fill_record(int p, const Level1D& L, const Sizes3& s, int kind, const int* i, double* r, int RU) {
  const int q = p - 1, W = 2 * q + 1;
  std::fill(r, r + RU, 0.0);
  long long g = gid3(s, kind, i);
  const int nbox = kind < 3 ? 2 : 3;
  for (int k = 0; k < nbox; ++k) {
    Box3 b = box_of(p, kind, k);
    int c = b.axis, o1 = (c + 1) % 3, o2 = (c + 2) % 3;
    int st = box_start(p, k);
    for (int a = 0; a < b.len; ++a)
      for (int e1 = 0; e1 < W; ++e1)
        for (int e2 = 0; e2 < W; ++e2) {
          int j[3];
          j[c] = i[c] + b.org + a; j[o1] = i[o1] - q + e1; j[o2] = i[o2] - q + e2;
          long long h = gid3(s, b.blk, j);
          if (h >= 0) r[st + (a * W + e1) * W + e2] = k_entry3(L, s, g, h);
        }
  }
  if (kind == 3) r[RU - 1] = L.mq[i[0]] * L.mq[i[1]] * L.mq[i[2]];
}

void build_stencils3(int p, const Level1D& L, const Sizes3& s, Stencils3& st) {
  const int q = p - 1, W = 2 * q + 1;
  st.T = 2 * p + 1;
  st.NC = 2 * st.T + 1;
  st.B0 = (2 * p + 1) * W * W;
  st.B1 = 2 * p * W * W;
  st.RU = st.B0 + 2 * st.B1 + 1;
  const int T = st.T, NC = st.NC, RU = st.RU;
  const int lastp = s.n + p - 1, lastq = s.n + q - 1;
  for (int kind = 0; kind < 4; ++kind) {
    auto& cmap = st.cmap[kind];
    auto& rec = st.rec[kind];
    cmap.assign((size_t)NC * NC * NC, -1);
    rec.clear();
    int lo[3], hi[3], last[3];
    for (int a = 0; a < 3; ++a) {
      bool pa = kind < 3 && a == kind;
      lo[a] = pa ? 1 : 0; hi[a] = pa ? s.ni : s.nq - 1; last[a] = pa ? lastp : lastq;
    }
    // only indices within T of an end, or the first interior one, give distinct classes
    auto cand = [&](int a) {
      std::vector<int> v;
      for (int x = lo[a]; x <= hi[a]; ++x)
        if (x < T + 1 || last[a] - x < T + 1) v.push_back(x);
      return v;
    };
    auto cx = cand(0), cy = cand(1), cz = cand(2);
    for (int z : cz)
      for (int y : cy)
        for (int x : cx) {
          int i[3] = {x, y, z};
          int cl = (cls1(z, last[2], T) * NC + cls1(y, last[1], T)) * NC + cls1(x, last[0], T);
          if (cmap[cl] >= 0) continue;
          cmap[cl] = (int)(rec.size() / RU);
          rec.resize(rec.size() + RU);
          fill_record(p, L, s, kind, i, &rec[rec.size() - RU], RU);
        }
  }
}

// 1D position class of a patch index a in [lo, hi] (T = 2p+2 from each end).
int pos_class3(int a, int lo, int hi, int p) {
  const int T = 2 * p + 2;
  if (a - lo < T) return a - lo;
  if (hi - a < T) return T + (hi - a);
  return 2 * T;
}

template <typename Entry>
int build_patches3(int p, const Level1D& L, const Sizes3& s, PatchTables& pt, std::string& err, Entry kent,
                   bool per_patch) {
  const int n = s.n, q = p - 1;
  auto sup = [&](int i, int d) { return std::make_pair(std::max(0, i - d), std::min(n - 1, i)); };
  auto inside = [](std::pair<int, int> a, std::pair<int, int> box) { return box.first <= a.first && a.second <= box.second; };
  struct P { int fam, i[3], colour; std::vector<int> dofs; int nv; std::tuple<int, int, int, int> key; };
  std::vector<P> all;
  const int ncol_fam = p * (p + 1) * (p + 1);
  for (int fam = 0; fam < 3; ++fam) {
    int lo[3], hi[3], dg[3], stride[3];
    for (int a = 0; a < 3; ++a) {
      bool qa = a == fam;                    // vector-potential family fam is degree q along fam
      dg[a] = qa ? q : p;
      lo[a] = qa ? 0 : 1; hi[a] = qa ? s.nq - 1 : s.ni;
      stride[a] = qa ? p : p + 1;            // support width in elements along a
    }
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          P P_;
          P_.fam = fam; P_.i[0] = i; P_.i[1] = j; P_.i[2] = k;
          P_.colour = fam * ncol_fam + ((k % stride[2]) * stride[1] + (j % stride[1])) * stride[0] + (i % stride[0]);
          std::pair<int, int> box[3] = {sup(i, dg[0]), sup(j, dg[1]), sup(k, dg[2])};
          const int idx[3] = {i, j, k};
          auto collect = [&](int blk) {
            int d3[3];
            for (int a = 0; a < 3; ++a) d3[a] = (blk < 3 && a == blk) ? p : q;
            int r0[3], r1[3];
            for (int a = 0; a < 3; ++a) { r0[a] = std::max(0, idx[a] - p - 1); r1[a] = std::min(n + d3[a] - 1, idx[a] + p + 1); }
            int jj[3];
            for (jj[2] = r0[2]; jj[2] <= r1[2]; ++jj[2])
              for (jj[1] = r0[1]; jj[1] <= r1[1]; ++jj[1])
                for (jj[0] = r0[0]; jj[0] <= r1[0]; ++jj[0]) {
                  long long g = gid3(s, blk, jj);
                  if (g < 0) continue;
                  bool in = true;
                  for (int a = 0; a < 3 && in; ++a) in = inside(sup(jj[a], d3[a]), box[a]);
                  if (in) P_.dofs.push_back((int)g);
                }
          };
          collect(0); collect(1); collect(2);
          P_.nv = (int)P_.dofs.size();
          collect(3);
          P_.key = per_patch ? std::make_tuple(fam, i, j, k)
                             : std::make_tuple(fam, pos_class3(i, lo[0], hi[0], p), pos_class3(j, lo[1], hi[1], p),
                                               pos_class3(k, lo[2], hi[2], p));
          all.push_back(std::move(P_));
        }
  }
  // colour-major (families x, y, z); inside a colour the 4+4-DOF patches first
  std::stable_sort(all.begin(), all.end(), [](const P& x, const P& y) {
    if (x.colour != y.colour) return x.colour < y.colour;
    return (x.dofs.size() != 8) < (y.dofs.size() != 8); });
  int maxl = 0;
  for (auto& P_ : all) maxl = std::max(maxl, (int)P_.dofs.size());
  pt.n_patches = (int)all.size(); pt.maxl = maxl; pt.n_colours = 3 * ncol_fam;
  pt.dofs.assign((size_t)pt.n_patches * maxl, -1);
  pt.cls.assign(pt.n_patches, 0);
  pt.colour_off.assign(pt.n_colours + 1, 0);
  std::map<std::tuple<int, int, int, int>, int> cmap8, cmapg;
  std::vector<int> rep8, repg;
  for (int i = 0; i < pt.n_patches; ++i) {
    auto& P_ = all[i];
    for (size_t k = 0; k < P_.dofs.size(); ++k) pt.dofs[(size_t)i * maxl + k] = P_.dofs[k];
    pt.colour_off[P_.colour + 1]++;
    bool is8 = P_.dofs.size() == 8;
    auto& cmap = is8 ? cmap8 : cmapg;
    auto& rep = is8 ? rep8 : repg;
    auto it = cmap.find(P_.key);
    if (it == cmap.end()) { int id = (int)rep.size(); cmap[P_.key] = id; rep.push_back(i); pt.cls[i] = id; }
    else pt.cls[i] = it->second;
  }
  for (int c = 0; c < pt.n_colours; ++c) pt.colour_off[c + 1] += pt.colour_off[c];
  pt.n8.assign(pt.n_colours, 0);
  for (int c = 0; c < pt.n_colours; ++c)
    for (int k = pt.colour_off[c]; k < pt.colour_off[c + 1] && all[k].dofs.size() == 8; ++k) pt.n8[c]++;
  {
    // support of a basis function of degree d with index i on n elements: [i - d, i] clipped;
    // velocity component c has degree p along axis c and q across
    auto sup = [&](long long g, int* lo, int* hi) {
      const Dof3 r = decode3(s, g);
      for (int a = 0; a < 3; ++a) {
        const int d = (r.blk < 3 && r.blk == a) ? p : q;
        lo[a] = std::max(0, r.i[a] - d);
        hi[a] = std::min(n - 1, r.i[a]);
      }
    };
    const int ne[3] = {n, n, n};
    if (!validate_patch_tables(pt, s.n_total - 1, err, sup, ne)) return IGAMG_EINVAL;
  }
  // bordered local inverses (zero-mean local pressure through m_j = int N^q_j), one per class
  auto local_inverse = [&](const P& P_, std::vector<double>& inv) -> bool {
    int nl = (int)P_.dofs.size(), nb = nl + 1;
    std::vector<double> Kb((size_t)nb * nb, 0.0);
    for (int r = 0; r < nl; ++r)
      for (int t = 0; t < nl; ++t) Kb[(size_t)r * nb + t] = kent(P_.dofs[r], P_.dofs[t]);
    for (int r = P_.nv; r < nl; ++r) {
      Dof3 d = decode3(s, P_.dofs[r]);
      double m = L.mq[d.i[0]] * L.mq[d.i[1]] * L.mq[d.i[2]];
      Kb[(size_t)r * nb + nl] = m; Kb[(size_t)nl * nb + r] = m;
    }
    return invert(Kb, nb, inv);
  };
  pt.n_cls = (int)repg.size();
  pt.n_cls8 = (int)rep8.size();
  pt.nloc.assign(std::max(pt.n_cls, 1), 0);
  pt.cinv.assign((size_t)std::max(pt.n_cls, 1) * maxl * maxl, 0.0);
  pt.cinv8.assign((size_t)std::max(pt.n_cls8, 1) * 64, 0.0);
  // the wall classes are independent dense inversions: spread them over host threads
  std::atomic<int> next{0}, bad{0};
  auto work = [&]() {
    for (;;) {
      int c = next.fetch_add(1);
      if (c >= pt.n_cls) break;
      auto& P_ = all[repg[c]];
      int nl = (int)P_.dofs.size(), nb = nl + 1;
      std::vector<double> inv;
      if (!local_inverse(P_, inv)) { bad = 1; continue; }
      pt.nloc[c] = nl;
      for (int r = 0; r < nl; ++r)
        for (int t = 0; t < nl; ++t) pt.cinv[((size_t)c * maxl + r) * maxl + t] = inv[(size_t)r * nb + t];
    }
  };
  int nth = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) th.emplace_back(work);
  for (auto& t : th) t.join();
  if (bad) { err = "singular local patch matrix"; return IGAMG_ESINGULAR; }
  std::atomic<int> next8{0};
  auto work8 = [&]() {
    for (;;) {
      int c = next8.fetch_add(1);
      if (c >= pt.n_cls8) break;
      std::vector<double> inv;
      if (!local_inverse(all[rep8[c]], inv)) { bad = 1; continue; }
      for (int r = 0; r < 8; ++r)
        for (int t = 0; t < 8; ++t) pt.cinv8[(size_t)c * 64 + r * 8 + t] = inv[(size_t)r * 9 + t];
    }
  };
  th.clear();
  for (int t = 0; t < nth; ++t) th.emplace_back(work8);
  for (auto& t : th) t.join();
  if (bad) { err = "singular local patch matrix"; return IGAMG_ESINGULAR; }
  build_row_slots(pt);
  if (per_patch) { std::vector<double>().swap(pt.cinv); std::vector<double>().swap(pt.cinv8); }
  return IGAMG_OK;
}

// ---- generalized Oseen (Sec. 3.1): the advection block (beta . grad u, v), componentwise ----
// Stored per velocity row as box 0 of the row record (B0 entries: long axis = the component's
// own axis, offsets -p..p; -q..q across).  Position of column j in the box of row i:
int adv_pos(int p, int c, const int* i, const int* j) {
  const int q = p - 1, W = 2 * q + 1;
  const int o1 = (c + 1) % 3, o2 = (c + 2) % 3;
  int a = j[c] - i[c] + p, e1 = j[o1] - i[o1] + q, e2 = j[o2] - i[o2] + q;
  if (a < 0 || a > 2 * p || e1 < 0 || e1 >= W || e2 < 0 || e2 >= W) return -1;
  return (a * W + e1) * W + e2;
}

// Fine level: element-by-element Gauss quadrature ((p+2)^3 points) of int v (beta . grad u)
// for every component, beta sampled at the quadrature points (3, nG, nG, nG).  Elements are
// processed in z-slabs coloured by ez mod (p+1), so slabs of one colour touch disjoint rows.
void add_advection3(int p, const Sizes3& s, const double* beta, std::vector<double>& adv) {
  const int q = p - 1, n = s.n, G = p + 2, nG = n * G;
  const int W = 2 * q + 1, B0 = (2 * p + 1) * W * W;
  adv.assign((size_t)s.n_u * B0, 0.0);
  auto tp = knots(p, n), tq = knots(q, n);
  std::vector<double> gx, gw;
  gauss01(G, gx, gw);
  // per element and degree: values and derivatives at the G points, (d+1) x G
  auto table = [&](int d, std::vector<double>& V, std::vector<double>& D) {
    const auto& t = d == p ? tp : tq;
    V.assign((size_t)n * (d + 1) * G, 0.0);
    D.assign((size_t)n * (d + 1) * G, 0.0);
    for (int e = 0; e < n; ++e)
      for (int g = 0; g < G; ++g) {
        double x = (e + gx[g]) / n, N[8], dN[8];
        span_values(t, d, e + d, x, N);
        span_derivs(t, d, e + d, x, dN);
        for (int k = 0; k <= d; ++k) {
          V[((size_t)e * (d + 1) + k) * G + g] = N[k];
          D[((size_t)e * (d + 1) + k) * G + g] = dN[k];
        }
      }
  };
  std::vector<double> Vp, Dp, Vq, Dq;
  table(p, Vp, Dp);
  table(q, Vq, Dq);
  const int nth = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
  for (int colour = 0; colour <= p; ++colour) {
    std::atomic<int> next{0};
    auto work = [&]() {
      std::vector<double> A, Bm, M;
      for (;;) {
        int slab = colour + (p + 1) * next.fetch_add(1);
        if (slab >= n) break;
        const int ez = slab;
        for (int ey = 0; ey < n; ++ey)
          for (int ex = 0; ex < n; ++ex) {
            const int e[3] = {ex, ey, ez};
            for (int c = 0; c < 3; ++c) {
              int d[3];
              const double *V[3], *D[3];
              for (int ax = 0; ax < 3; ++ax) {
                d[ax] = ax == c ? p : q;
                V[ax] = (ax == c ? Vp.data() : Vq.data()) + (size_t)e[ax] * (d[ax] + 1) * G;
                D[ax] = (ax == c ? Dp.data() : Dq.data()) + (size_t)e[ax] * (d[ax] + 1) * G;
              }
              const int nl = (d[0] + 1) * (d[1] + 1) * (d[2] + 1), ng = G * G * G;
              A.assign((size_t)nl * ng, 0.0);
              Bm.assign((size_t)nl * ng, 0.0);
              for (int kz = 0; kz <= d[2]; ++kz)
                for (int ky = 0; ky <= d[1]; ++ky)
                  for (int kx = 0; kx <= d[0]; ++kx) {
                    const int a = (kz * (d[1] + 1) + ky) * (d[0] + 1) + kx;
                    for (int gz = 0; gz < G; ++gz)
                      for (int gy = 0; gy < G; ++gy)
                        for (int gxx = 0; gxx < G; ++gxx) {
                          const int g = (gz * G + gy) * G + gxx;
                          const double w = gw[gz] * gw[gy] * gw[gxx] / ((double)n * n * n);
                          const double vx = V[0][kx * G + gxx], vy = V[1][ky * G + gy], vz = V[2][kz * G + gz];
                          const size_t qi = ((size_t)(ez * G + gz) * nG + (ey * G + gy)) * nG + (ex * G + gxx);
                          const double b0 = beta[qi], b1 = beta[(size_t)nG * nG * nG + qi],
                                       b2 = beta[(size_t)2 * nG * nG * nG + qi];
                          A[(size_t)a * ng + g] = w * vx * vy * vz;
                          Bm[(size_t)a * ng + g] = b0 * D[0][kx * G + gxx] * vy * vz + b1 * vx * D[1][ky * G + gy] * vz +
                                                   b2 * vx * vy * D[2][kz * G + gz];
                        }
                  }
              for (int a = 0; a < nl; ++a) {
                int ia[3] = {e[0] + a % (d[0] + 1), e[1] + (a / (d[0] + 1)) % (d[1] + 1), e[2] + a / ((d[0] + 1) * (d[1] + 1))};
                long long gi = gid3(s, c, ia);
                if (gi < 0) continue;
                for (int b = 0; b < nl; ++b) {
                  int ib[3] = {e[0] + b % (d[0] + 1), e[1] + (b / (d[0] + 1)) % (d[1] + 1), e[2] + b / ((d[0] + 1) * (d[1] + 1))};
                  if (gid3(s, c, ib) < 0) continue;
                  double v = 0.0;
                  for (int g = 0; g < ng; ++g) v += A[(size_t)a * ng + g] * Bm[(size_t)b * ng + g];
                  int pos = adv_pos(p, c, ia, ib);
                  if (pos >= 0) adv[(size_t)gi * B0 + pos] += v;
                }
              }
            }
          }
      }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(work);
    for (auto& t : th) t.join();
  }
}

// Coarse level: the advection block of R K P (Sec. 5.1), C_c = P_c^T A_c P_c per component,
// with P_c the tensor product of the 1D knot-insertion bands (degree p along c, p-1 across).
// Rows of the coarse level are independent: spread over host threads.
void galerkin_adv3(int p, const Sizes3& sf, const Sizes3& sc, const std::vector<double>& advf,
                   const Transfer1D& tp, const Transfer1D& tq, std::vector<double>& advc) {
  const int q = p - 1, W = 2 * q + 1, B0 = (2 * p + 1) * W * W;
  constexpr int WP = Transfer1D::WP, WR = Transfer1D::WR;
  advc.assign((size_t)sc.n_u * B0, 0.0);
  const int nth = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
  std::atomic<long long> next{0};
  auto work = [&]() {
    for (;;) {
      long long i0 = next.fetch_add(256);
      if (i0 >= sc.n_u) break;
      for (long long gi = i0; gi < std::min(sc.n_u, i0 + 256); ++gi) {
        Dof3 ci = decode3(sc, gi);
        const int c = ci.blk;
        const Transfer1D* T[3];
        for (int ax = 0; ax < 3; ++ax) T[ax] = ax == c ? &tp : &tq;
        // local (view) index of coarse row along each axis: the p-axis view drops index 0
        int li[3];
        for (int ax = 0; ax < 3; ++ax) li[ax] = ci.i[ax] - (ax == c ? 1 : 0);
        double* out = &advc[(size_t)gi * B0];
        for (int rz = 0; rz < WR; ++rz)
          for (int ry = 0; ry < WR; ++ry)
            for (int rx = 0; rx < WR; ++rx) {
              const int r[3] = {rx, ry, rz};
              int fa[3];
              double wa = 1.0;
              bool ok = true;
              for (int ax = 0; ax < 3 && ok; ++ax) {
                int f = T[ax]->f0[li[ax]] + r[ax];
                if (f >= T[ax]->nf) { ok = false; break; }
                double w = T[ax]->rv[(size_t)li[ax] * WR + r[ax]];
                if (w == 0.0) { ok = false; break; }
                wa *= w;
                fa[ax] = f + (ax == c ? 1 : 0);                 // full fine index
              }
              if (!ok) continue;
              long long ga = gid3(sf, c, fa);
              if (ga < 0) continue;
              const double* arow = &advf[(size_t)ga * B0];
              for (int a = 0; a <= 2 * p; ++a)
                for (int e1 = 0; e1 < W; ++e1)
                  for (int e2 = 0; e2 < W; ++e2) {
                    const double v = arow[(a * W + e1) * W + e2];
                    if (v == 0.0) continue;
                    const int o1 = (c + 1) % 3, o2 = (c + 2) % 3;
                    int fb[3];
                    fb[c] = fa[c] - p + a; fb[o1] = fa[o1] - q + e1; fb[o2] = fa[o2] - q + e2;
                    int lb[3];
                    bool okb = true;
                    for (int ax = 0; ax < 3; ++ax) {
                      lb[ax] = fb[ax] - (ax == c ? 1 : 0);
                      if (lb[ax] < 0 || lb[ax] >= T[ax]->nf) okb = false;
                    }
                    if (!okb) continue;
                    for (int kz = 0; kz < WP; ++kz)
                      for (int ky = 0; ky < WP; ++ky)
                        for (int kx = 0; kx < WP; ++kx) {
                          const int k[3] = {kx, ky, kz};
                          int cj[3];
                          double wb = v * wa;
                          bool okj = true;
                          for (int ax = 0; ax < 3 && okj; ++ax) {
                            int cc = T[ax]->c0[lb[ax]] + k[ax];
                            double w = T[ax]->pv[(size_t)lb[ax] * WP + k[ax]];
                            if (cc >= T[ax]->nc || w == 0.0) { okj = false; break; }
                            wb *= w;
                            cj[ax] = cc + (ax == c ? 1 : 0);
                          }
                          if (!okj) continue;
                          int pos = adv_pos(p, c, ci.i, cj);
                          if (pos >= 0) out[pos] += wb;
                        }
                  }
            }
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) th.emplace_back(work);
  for (auto& t : th) t.join();
}

// Per-row records of a level: class record of the row plus the advection box (velocity rows).
void rows_with_advection3(int p, const LevelHost3& lv, std::vector<double>& rows) {
  const auto& s = lv.sz;
  const auto& st = lv.st;
  const int q = p - 1, RU = st.RU, W = 2 * q + 1, B0 = (2 * p + 1) * W * W;
  rows.assign((size_t)(s.n_total - 1) * RU, 0.0);
  const int lastp = s.n + p - 1, lastq = s.n + q - 1;
  for (long long g = 0; g < s.n_total - 1; ++g) {
    Dof3 d = decode3(s, g);
    int last[3];
    for (int x = 0; x < 3; ++x) last[x] = (d.blk < 3 && x == d.blk) ? lastp : lastq;
    int cl = (cls1(d.i[2], last[2], st.T) * st.NC + cls1(d.i[1], last[1], st.T)) * st.NC + cls1(d.i[0], last[0], st.T);
    const double* r = &st.rec[d.blk][(size_t)st.cmap[d.blk][cl] * RU];
    double* o = &rows[(size_t)g * RU];
    std::copy(r, r + RU, o);
    if (d.blk < 3)
      for (int k = 0; k < B0; ++k) o[k] += lv.adv[(size_t)g * B0 + k];
  }
}

// ---- mapped domains (Sec. 4.3 push-forwards; Sec. 6.4's hollow cylinder section) ----------
// Position of column b in the record of row a (boxes 0..2), or -1.
int rec_pos3(int p, const Dof3& a, const Dof3& b) {
  const int q = p - 1, W = 2 * q + 1;
  const int nbox = a.blk < 3 ? 2 : 3;
  for (int k = 0; k < nbox; ++k) {
    Box3 bx = box_of(p, a.blk, k);
    if (bx.blk != b.blk) continue;
    const int c = bx.axis, o1 = (c + 1) % 3, o2 = (c + 2) % 3;
    const int da = b.i[c] - a.i[c] - bx.org, e1 = b.i[o1] - a.i[o1] + q, e2 = b.i[o2] - a.i[o2] + q;
    if (da < 0 || da >= bx.len || e1 < 0 || e1 >= W || e2 < 0 || e2 >= W) return -1;
    return box_start(p, k) + (da * W + e1) * W + e2;
  }
  return -1;
}

// Column of record entry e of row a (blk = -1 outside the free ranges; 4 = lambda).
Dof3 rec_col3(const Sizes3& s, int p, const Dof3& a, int e) {
  const int q = p - 1, W = 2 * q + 1, RU = (2 * p + 1) * W * W + 2 * 2 * p * W * W + 1;
  Dof3 c{-1, {0, 0, 0}};
  if (e == RU - 1) { if (a.blk == 3) c.blk = 4; return c; }
  const int nbox = a.blk < 3 ? 2 : 3;
  for (int k = nbox - 1; k >= 0; --k) {
    const int st = box_start(p, k);
    if (e < st) continue;
    Box3 bx = box_of(p, a.blk, k);
    const int f = e - st, da = f / (W * W), e1 = (f / W) % W, e2 = f % W;
    if (da >= bx.len) return c;
    const int ax = bx.axis, o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
    c.blk = bx.blk;
    c.i[ax] = a.i[ax] + bx.org + da; c.i[o1] = a.i[o1] - q + e1; c.i[o2] = a.i[o2] - q + e2;
    if (gid3(s, c.blk, c.i) < 0) c.blk = -1;
    return c;
  }
  return c;
}

// Extra box of a u_x or u_y row (mapped domains): its coupling to the other of the two,
// 2p x 2p x (2q+1) entries [x][y][z]; u_x row -> u_y columns x - p .. x + q, y - q .. y + p;
// u_y row -> u_x columns x - q .. x + p, y - p .. y + q; z - q .. z + q for both.
int ext_pos3(int p, const Dof3& a, const Dof3& b) {
  const int q = p - 1, W = 2 * q + 1, L2 = 2 * p;
  if (!((a.blk == 0 && b.blk == 1) || (a.blk == 1 && b.blk == 0))) return -1;
  const int ox = a.blk == 0 ? -p : -q, oy = a.blk == 0 ? -q : -p;
  const int ix = b.i[0] - a.i[0] - ox, iy = b.i[1] - a.i[1] - oy, iz = b.i[2] - a.i[2] + q;
  if (ix < 0 || ix >= L2 || iy < 0 || iy >= L2 || iz < 0 || iz >= W) return -1;
  return (ix * L2 + iy) * W + iz;
}

Dof3 ext_col3(const Sizes3& s, int p, const Dof3& a, int e) {
  const int q = p - 1, W = 2 * q + 1, L2 = 2 * p;
  Dof3 c{-1, {0, 0, 0}};
  if (a.blk != 0 && a.blk != 1) return c;
  const int ox = a.blk == 0 ? -p : -q, oy = a.blk == 0 ? -q : -p;
  c.blk = 1 - a.blk;
  c.i[0] = a.i[0] + ox + e / (L2 * W);
  c.i[1] = a.i[1] + oy + (e / W) % L2;
  c.i[2] = a.i[2] - q + e % W;
  if (gid3(s, c.blk, c.i) < 0) c.blk = -1;
  return c;
}

// F(xi, eta, zeta) = (r(xi) C(eta), d zeta): the quarter annulus (rational quadratic
// Bezier quarter circle C, radius r = ri + (ro - ri) xi) extruded by the depth d.
void cylinder_map(double ri, double ro, double d, const double xi3[3], double X[3], double DF[3][3],
                  double D2[3][3][3]) {
  const double xi = xi3[0], eta = xi3[1], zeta = xi3[2];
  const double w = std::sqrt(0.5), t = eta, u = 1.0 - eta;
  const double Nx = u * u + w * 2 * t * u, Ny = w * 2 * t * u + t * t;
  const double dNx = -2 * u + w * (2 - 4 * t), dNy = w * (2 - 4 * t) + 2 * t;
  const double ddNx = 2 - 4 * w, ddNy = -4 * w + 2;
  const double Wt = u * u + w * 2 * t * u + t * t, dW = -2 * u + w * (2 - 4 * t) + 2 * t, ddW = 4 - 4 * w;
  const double C[2] = {Nx / Wt, Ny / Wt};
  const double A[2] = {dNx * Wt - Nx * dW, dNy * Wt - Ny * dW};
  const double dA[2] = {ddNx * Wt - Nx * ddW, ddNy * Wt - Ny * ddW};
  const double dr = ro - ri, r = ri + dr * xi;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      DF[i][k] = 0.0;
      for (int l = 0; l < 3; ++l) D2[i][k][l] = 0.0;
    }
  for (int i = 0; i < 2; ++i) {
    const double dC = A[i] / (Wt * Wt), ddC = dA[i] / (Wt * Wt) - 2 * A[i] * dW / (Wt * Wt * Wt);
    X[i] = r * C[i];
    DF[i][0] = dr * C[i];
    DF[i][1] = r * dC;
    D2[i][0][1] = D2[i][1][0] = dr * dC;
    D2[i][1][1] = r * ddC;
  }
  X[2] = d * zeta;
  DF[2][2] = d;
}

struct Geo3 { double X[3], DF[3][3], D2[3][3][3], J, dJ[3], inv[3][3]; };

Geo3 geo3_at(double ri, double ro, double d, const double xi3[3]) {
  Geo3 g;
  cylinder_map(ri, ro, d, xi3, g.X, g.DF, g.D2);
  const auto& M = g.DF;
  g.inv[0][0] = M[1][1] * M[2][2] - M[1][2] * M[2][1];
  g.inv[0][1] = M[0][2] * M[2][1] - M[0][1] * M[2][2];
  g.inv[0][2] = M[0][1] * M[1][2] - M[0][2] * M[1][1];
  g.inv[1][0] = M[1][2] * M[2][0] - M[1][0] * M[2][2];
  g.inv[1][1] = M[0][0] * M[2][2] - M[0][2] * M[2][0];
  g.inv[1][2] = M[0][2] * M[1][0] - M[0][0] * M[1][2];
  g.inv[2][0] = M[1][0] * M[2][1] - M[1][1] * M[2][0];
  g.inv[2][1] = M[0][1] * M[2][0] - M[0][0] * M[2][1];
  g.inv[2][2] = M[0][0] * M[1][1] - M[0][1] * M[1][0];
  g.J = M[0][0] * g.inv[0][0] + M[0][1] * g.inv[1][0] + M[0][2] * g.inv[2][0];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) g.inv[i][j] /= g.J;
  // d det J / dxi_k = det J tr(J^-1 dJ/dxi_k) (Jacobi's formula)
  for (int k = 0; k < 3; ++k) {
    double tr = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) tr += g.inv[i][j] * g.D2[j][i][k];
    g.dJ[k] = g.J * tr;
  }
  return g;
}

struct Pushed3 { double v[3], g[3][3], divh; };

// v = N a_c / det J (contravariant Piola, a_c = column c of DF) with its physical gradient
Pushed3 push3(double N, const double dN[3], int c, const Geo3& G) {
  Pushed3 o;
  double Gk[3][3];
  for (int i = 0; i < 3; ++i) {
    const double a = G.DF[i][c];
    o.v[i] = N * a / G.J;
    for (int k = 0; k < 3; ++k) Gk[i][k] = dN[k] * a / G.J + N * G.D2[i][c][k] / G.J - N * a * G.dJ[k] / (G.J * G.J);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o.g[i][j] = Gk[i][0] * G.inv[0][j] + Gk[i][1] * G.inv[1][j] + Gk[i][2] * G.inv[2][j];
  o.divh = dN[c];
  return o;
}

struct LocalVel3 { int n = 0; long long gid[128]; Dof3 d[128]; Pushed3 f[128]; };

// free velocity functions of element e at parametric point xi3
void local_velocity3(const Sizes3& s, int p, const int e[3], const std::vector<double>& tp,
                     const std::vector<double>& tq, const double xi3[3], const Geo3& G, LocalVel3& out) {
  const int q = p - 1;
  double Np[3][8], dNp[3][8], Nq[3][8], dNq[3][8];
  for (int ax = 0; ax < 3; ++ax) {
    span_values(tp, p, e[ax] + p, xi3[ax], Np[ax]); span_derivs(tp, p, e[ax] + p, xi3[ax], dNp[ax]);
    span_values(tq, q, e[ax] + q, xi3[ax], Nq[ax]); span_derivs(tq, q, e[ax] + q, xi3[ax], dNq[ax]);
  }
  out.n = 0;
  for (int c = 0; c < 3; ++c) {
    int deg[3] = {q, q, q};
    deg[c] = p;
    for (int kz = 0; kz <= deg[2]; ++kz)
      for (int ky = 0; ky <= deg[1]; ++ky)
        for (int kx = 0; kx <= deg[0]; ++kx) {
          const int k[3] = {kx, ky, kz};
          Dof3 d{c, {e[0] + kx, e[1] + ky, e[2] + kz}};
          const long long g = gid3(s, c, d.i);
          if (g < 0) continue;
          double val[3], der[3];
          for (int ax = 0; ax < 3; ++ax) {
            val[ax] = ax == c ? Np[ax][k[ax]] : Nq[ax][k[ax]];
            der[ax] = ax == c ? dNp[ax][k[ax]] : dNq[ax][k[ax]];
          }
          const double N = val[0] * val[1] * val[2];
          const double dN[3] = {der[0] * val[1] * val[2], val[0] * der[1] * val[2], val[0] * val[1] * der[2]};
          out.gid[out.n] = g; out.d[out.n] = d;
          out.f[out.n++] = push3(N, dN, c, G);
        }
  }
}

// K(row a, column b) += val into the level's records; returns |val| when (a, b) lies outside
// the record pattern (then nothing is stored).
double put3(int p, std::vector<double>& rows, std::vector<double>& ext, const Dof3& a, long long ga, const Dof3& b,
            double val) {
  const int q = p - 1, W = 2 * q + 1, RU = (2 * p + 1) * W * W + 4 * p * W * W + 1, BX = 4 * p * p * W;
  int pos = rec_pos3(p, a, b);
  if (pos >= 0) { rows[(size_t)ga * RU + pos] += val; return 0.0; }
  pos = ext_pos3(p, a, b);
  if (pos >= 0) { ext[(size_t)ga * BX + pos] += val; return 0.0; }
  return std::fabs(val);
}

// Fine-level operator of generalized Stokes on the hollow cylinder section, in record form:
// sigma (u, v) + nu (grad u, grad v) - (div v, p) + (div u, q) on the physical domain with
// (p+2)-point Gauss rules per direction; Nitsche terms on the six faces, h = det J /
// (|t1 x t2| n); the multiplier column m_j = int q_hat_j dxi.  Also fills the physical
// quadrature points and J^T for the load vector.
int assemble_mapped3(int p, LevelHost3& lv, double sigma, double nu, double cpen, double ri, double ro, double depth,
                     HierarchyHost3& H, std::string& err) {
  const int q = p - 1, W = 2 * q + 1, n = lv.sz.n, G = p + 2, nG = n * G;
  const int RU = (2 * p + 1) * W * W + 4 * p * W * W + 1, BX = 4 * p * p * W;
  const auto& sz = lv.sz;
  lv.rows.assign((size_t)(sz.n_total - 1) * RU, 0.0);
  lv.ext.assign((size_t)2 * sz.n_uc * BX, 0.0);
  std::vector<double> gx, gw;
  gauss01(G, gx, gw);
  auto tp = knots(p, n), tq = knots(q, n);
  double outside = 0.0, scale = 0.0;
  // an element slab ez writes only the records of functions with z index in [ez, ez + p],
  // so slabs p + 2 apart never share a record: p + 2 sequential phases
  const unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<double> out_max(nth, 0.0), sc_max(nth, 0.0);
  for (int ph = 0; ph < p + 2; ++ph) {
    std::vector<int> ezs;
    for (int ez = ph; ez < n; ez += p + 2) ezs.push_back(ez);
    auto work = [&](unsigned t, size_t i0, size_t i1) {
      LocalVel3 lvv;
      const int nq3 = (q + 1) * (q + 1) * (q + 1);
      std::vector<double> M, B;                      // element matrices, summed over its points
      for (size_t ii = i0; ii < i1; ++ii) {
        const int ez = ezs[ii];
        for (int ey = 0; ey < n; ++ey)
          for (int ex = 0; ex < n; ++ex) {
            const int e[3] = {ex, ey, ez};
            int nv = -1;
            for (int gzi = 0; gzi < G; ++gzi)
              for (int gyi = 0; gyi < G; ++gyi)
                for (int gxi = 0; gxi < G; ++gxi) {
                  const double xi3[3] = {(ex + gx[gxi]) / n, (ey + gx[gyi]) / n, (ez + gx[gzi]) / n};
                  const double w = gw[gxi] * gw[gyi] * gw[gzi] / ((double)n * n * n);
                  Geo3 g = geo3_at(ri, ro, depth, xi3);
                  local_velocity3(sz, p, e, tp, tq, xi3, g, lvv);   // same functions, same order at every point
                  if (nv < 0) {
                    nv = lvv.n;
                    M.assign((size_t)nv * nv, 0.0);
                    B.assign((size_t)nv * nq3, 0.0);
                  }
                  double Nq[3][8];
                  for (int ax = 0; ax < 3; ++ax) span_values(tq, q, e[ax] + q, xi3[ax], Nq[ax]);
                  const double wJ = w * g.J;
                  for (int i = 0; i < nv; ++i) {
                    const Pushed3& a = lvv.f[i];
                    for (int j = 0; j < nv; ++j) {
                      const Pushed3& b = lvv.f[j];
                      const double m = a.v[0] * b.v[0] + a.v[1] * b.v[1] + a.v[2] * b.v[2];
                      double k = 0.0;
                      for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c) k += a.g[r][c] * b.g[r][c];
                      M[(size_t)i * nv + j] += wJ * (sigma * m + nu * k);
                    }
                    // b(v, q) = int divhat vhat qhat / det J dxi
                    int kq = 0;
                    for (int kz = 0; kz <= q; ++kz)
                      for (int ky = 0; ky <= q; ++ky)
                        for (int kx = 0; kx <= q; ++kx)
                          B[(size_t)i * nq3 + kq++] += w * a.divh * Nq[0][kx] * Nq[1][ky] * Nq[2][kz] / g.J;
                  }
                }
            // scatter the element's matrices into the records
            for (int i = 0; i < nv; ++i) {
              for (int j = 0; j < nv; ++j) {
                const double val = M[(size_t)i * nv + j];
                sc_max[t] = std::max(sc_max[t], std::fabs(val));
                out_max[t] = std::max(out_max[t], put3(p, lv.rows, lv.ext, lvv.d[i], lvv.gid[i], lvv.d[j], val));
              }
              int kq = 0;
              for (int kz = 0; kz <= q; ++kz)
                for (int ky = 0; ky <= q; ++ky)
                  for (int kx = 0; kx <= q; ++kx) {
                    const Dof3 dq{3, {ex + kx, ey + ky, ez + kz}};
                    const long long gq = gid3(sz, 3, dq.i);
                    const double bval = B[(size_t)i * nq3 + kq++];
                    put3(p, lv.rows, lv.ext, lvv.d[i], lvv.gid[i], dq, -bval);
                    put3(p, lv.rows, lv.ext, dq, gq, lvv.d[i], bval);
                  }
            }
          }
      }
    };
    std::vector<std::thread> th;
    const size_t chunk = (ezs.size() + nth - 1) / nth;
    for (unsigned t = 0; t < nth; ++t) {
      const size_t i0 = t * chunk, i1 = std::min(ezs.size(), i0 + chunk);
      if (i0 < i1) th.emplace_back(work, t, i0, i1);
    }
    for (auto& t : th) t.join();
  }
  for (unsigned t = 0; t < nth; ++t) { outside = std::max(outside, out_max[t]); scale = std::max(scale, sc_max[t]); }
  // Nitsche terms on the six faces
  const double pen_c = cpen * nu;
  LocalVel3 lvv;
  for (int k = 0; k < 3; ++k) {
    const int a1 = (k + 1) % 3, a2 = (k + 2) % 3;
    for (int side = 0; side < 2; ++side)
      for (int e1 = 0; e1 < n; ++e1)
        for (int e2 = 0; e2 < n; ++e2)
          for (int g1 = 0; g1 < G; ++g1)
            for (int g2 = 0; g2 < G; ++g2) {
              int e[3];
              double xi3[3];
              e[k] = side ? n - 1 : 0; xi3[k] = side;
              e[a1] = e1; xi3[a1] = (e1 + gx[g1]) / n;
              e[a2] = e2; xi3[a2] = (e2 + gx[g2]) / n;
              const double wt = gw[g1] * gw[g2] / ((double)n * n);
              Geo3 g = geo3_at(ri, ro, depth, xi3);
              local_velocity3(sz, p, e, tp, tq, xi3, g, lvv);
              double nv[3] = {g.inv[k][0], g.inv[k][1], g.inv[k][2]};     // gradient of xi_k
              const double nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
              for (int c = 0; c < 3; ++c) nv[c] *= (side ? 1.0 : -1.0) / nn;
              const double t1[3] = {g.DF[0][a1], g.DF[1][a1], g.DF[2][a1]};
              const double t2[3] = {g.DF[0][a2], g.DF[1][a2], g.DF[2][a2]};
              const double cr[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2], t1[0] * t2[1] - t1[1] * t2[0]};
              const double area = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
              const double ds = wt * area, h = g.J / (area * n);
              for (int i = 0; i < lvv.n; ++i) {
                const Pushed3& a = lvv.f[i];
                double dna[3];
                for (int r = 0; r < 3; ++r) dna[r] = a.g[r][0] * nv[0] + a.g[r][1] * nv[1] + a.g[r][2] * nv[2];
                for (int j = 0; j < lvv.n; ++j) {
                  const Pushed3& b = lvv.f[j];
                  double dnb[3];
                  for (int r = 0; r < 3; ++r) dnb[r] = b.g[r][0] * nv[0] + b.g[r][1] * nv[1] + b.g[r][2] * nv[2];
                  double t_ab = 0.0, t_ba = 0.0, uv = 0.0;
                  for (int r = 0; r < 3; ++r) { t_ab += dnb[r] * a.v[r]; t_ba += dna[r] * b.v[r]; uv += a.v[r] * b.v[r]; }
                  const double val = ds * (-nu * t_ab - nu * t_ba + pen_c / h * uv);
                  outside = std::max(outside, put3(p, lv.rows, lv.ext, lvv.d[i], lvv.gid[i], lvv.d[j], val));
                }
              }
            }
  }
  if (outside > 1e-12 * scale) { err = "mapped operator left the record pattern"; return IGAMG_EINVAL; }
  // multiplier column of the pressure rows
  for (long long g = sz.n_u; g < sz.n_total - 1; ++g) {
    Dof3 d = decode3(sz, g);
    lv.rows[(size_t)g * RU + RU - 1] = lv.f.mq[d.i[0]] * lv.f.mq[d.i[1]] * lv.f.mq[d.i[2]];
  }
  // physical quadrature points and J^T for the load vector
  H.quad_xyz.assign((size_t)3 * nG * nG * nG, 0.0);
  H.jt.assign((size_t)9 * nG * nG * nG, 0.0);
  const size_t np3 = (size_t)nG * nG * nG;
  for (int iz = 0; iz < nG; ++iz)
    for (int iy = 0; iy < nG; ++iy)
      for (int ix = 0; ix < nG; ++ix) {
        const double xi3[3] = {(ix / G + gx[ix % G]) / n, (iy / G + gx[iy % G]) / n, (iz / G + gx[iz % G]) / n};
        double X[3], DF[3][3], D2[3][3][3];
        cylinder_map(ri, ro, depth, xi3, X, DF, D2);
        const size_t o = ((size_t)iz * nG + iy) * nG + ix;
        for (int c = 0; c < 3; ++c) H.quad_xyz[c * np3 + o] = X[c];
        for (int kk = 0; kk < 3; ++kk)
          for (int i = 0; i < 3; ++i) H.jt[o * 9 + kk * 3 + i] = DF[i][kk];
      }
  return IGAMG_OK;
}

// K_c = P^T K_f P (Sec. 5.1) for whole per-row records (all boxes and the extra box): the
// operator on a mapped domain has no re-assembly formula on coarse levels.
int galerkin_rows3(int p, const LevelHost3& F, LevelHost3& C, const Transfer1D& tp, const Transfer1D& tq,
                   std::string& err) {
  const int q = p - 1, W = 2 * q + 1, RU = (2 * p + 1) * W * W + 4 * p * W * W + 1, BX = 4 * p * p * W;
  constexpr int WP = Transfer1D::WP, WR = Transfer1D::WR;
  const Sizes3 &sf = F.sz, &sc = C.sz;
  C.rows.assign((size_t)(sc.n_total - 1) * RU, 0.0);
  const bool has_ext = !F.ext.empty();
  if (has_ext) C.ext.assign((size_t)2 * sc.n_uc * BX, 0.0);
  std::atomic<long long> next{0};
  std::atomic<int> bad{0};
  auto view = [&](int blk, int ax) -> const Transfer1D& { return (blk < 3 && ax == blk) ? tp : tq; };
  auto work = [&]() {
    for (;;) {
      const long long i0 = next.fetch_add(128);
      if (i0 >= sc.n_total - 1) break;
      for (long long gi = i0; gi < std::min(sc.n_total - 1, i0 + 128); ++gi) {
        const Dof3 ci = decode3(sc, gi);
        int li[3];
        for (int ax = 0; ax < 3; ++ax) li[ax] = ci.i[ax] - ((ci.blk < 3 && ax == ci.blk) ? 1 : 0);
        double* orow = &C.rows[(size_t)gi * RU];
        double* oext = (has_ext && ci.blk < 2) ? &C.ext[(size_t)gi * BX] : nullptr;
        for (int rz = 0; rz < WR; ++rz)
          for (int ry = 0; ry < WR; ++ry)
            for (int rx = 0; rx < WR; ++rx) {
              const int r[3] = {rx, ry, rz};
              int fa[3];
              double wa = 1.0;
              bool ok = true;
              for (int ax = 0; ax < 3 && ok; ++ax) {
                const Transfer1D& T = view(ci.blk, ax);
                const int f = T.f0[li[ax]] + r[ax];
                const double w = f < T.nf ? T.rv[(size_t)li[ax] * WR + r[ax]] : 0.0;
                if (w == 0.0) { ok = false; break; }
                wa *= w;
                fa[ax] = f + ((ci.blk < 3 && ax == ci.blk) ? 1 : 0);
              }
              if (!ok) continue;
              const long long ga = gid3(sf, ci.blk, fa);
              if (ga < 0) continue;
              const Dof3 da{ci.blk, {fa[0], fa[1], fa[2]}};
              const double* frow = &F.rows[(size_t)ga * RU];
              const double* fext = (has_ext && ci.blk < 2) ? &F.ext[(size_t)ga * BX] : nullptr;
              double fscale = 0.0;
              for (int e = 0; e < RU; ++e) fscale = std::max(fscale, std::fabs(frow[e]));
              if (fext) for (int e = 0; e < BX; ++e) fscale = std::max(fscale, std::fabs(fext[e]));
              const int ne = fext ? RU + BX : RU;
              for (int e = 0; e < ne; ++e) {
                const double v = e < RU ? frow[e] : fext[e - RU];
                if (v == 0.0) continue;
                const Dof3 cb = e < RU ? rec_col3(sf, p, da, e) : ext_col3(sf, p, da, e - RU);
                if (cb.blk < 0) continue;
                if (cb.blk == 4) { orow[RU - 1] += wa * v; continue; }
                int lb[3];
                for (int ax = 0; ax < 3; ++ax) lb[ax] = cb.i[ax] - ((cb.blk < 3 && ax == cb.blk) ? 1 : 0);
                for (int kz = 0; kz < WP; ++kz)
                  for (int ky = 0; ky < WP; ++ky)
                    for (int kx = 0; kx < WP; ++kx) {
                      const int k[3] = {kx, ky, kz};
                      Dof3 cj{cb.blk, {0, 0, 0}};
                      double wb = wa * v;
                      bool okj = true;
                      for (int ax = 0; ax < 3 && okj; ++ax) {
                        const Transfer1D& T = view(cb.blk, ax);
                        const int cc = T.c0[lb[ax]] + k[ax];
                        const double w = cc < T.nc ? T.pv[(size_t)lb[ax] * WP + k[ax]] : 0.0;
                        if (w == 0.0) { okj = false; break; }
                        wb *= w;
                        cj.i[ax] = cc + ((cb.blk < 3 && ax == cb.blk) ? 1 : 0);
                      }
                      if (!okj) continue;
                      int pos = rec_pos3(p, ci, cj);
                      if (pos >= 0) { orow[pos] += wb; continue; }
                      pos = oext ? ext_pos3(p, ci, cj) : -1;
                      if (pos >= 0) { oext[pos] += wb; continue; }
                      // only round-off may fall outside the pattern
                      if (std::fabs(v) > 1e-12 * fscale) bad = 1;
                    }
              }
            }
      }
    }
  };
  const int nth = std::max(1, std::min(32, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) th.emplace_back(work);
  for (auto& t : th) t.join();
  if (bad) { err = "Galerkin product left the coarse record pattern"; return IGAMG_EINVAL; }
  return IGAMG_OK;
}

}  // namespace

// entry (g1, g2) from the per-row records (generalized Oseen)
double k_entry3_rows(const LevelHost3& lv, int p, long long g1, long long g2) {
  const auto& s = lv.sz;
  const int q = p - 1, W = 2 * q + 1, RU = lv.st.RU;
  Dof3 a = decode3(s, g1), b = decode3(s, g2);
  if (a.blk == 4) {
    if (b.blk != 3) return 0.0;
    return lv.rows[(size_t)g2 * RU + RU - 1];
  }
  const double* r = &lv.rows[(size_t)g1 * RU];
  if (b.blk == 4) return a.blk == 3 ? r[RU - 1] : 0.0;
  if (!lv.ext.empty() && a.blk < 2 && b.blk < 2 && a.blk != b.blk) {
    const int pos = ext_pos3(p, a, b);
    return pos < 0 ? 0.0 : lv.ext[(size_t)g1 * (4 * p * p * W) + pos];
  }
  const int nbox = a.blk < 3 ? 2 : 3;
  for (int k = 0; k < nbox; ++k) {
    Box3 bx = box_of(p, a.blk, k);
    if (bx.blk != b.blk) continue;
    int c = bx.axis, o1 = (c + 1) % 3, o2 = (c + 2) % 3;
    int da = b.i[c] - a.i[c] - bx.org, e1 = b.i[o1] - a.i[o1] + q, e2 = b.i[o2] - a.i[o2] + q;
    if (da < 0 || da >= bx.len || e1 < 0 || e1 >= W || e2 < 0 || e2 >= W) return 0.0;
    return r[box_start(p, k) + (da * W + e1) * W + e2];
  }
  return 0.0;
}

double k_entry3_records(const LevelHost3& lv, int p, long long g1, long long g2) {
  const auto& s = lv.sz;
  const auto& st = lv.st;
  const int q = p - 1, W = 2 * q + 1;
  Dof3 a = decode3(s, g1), b = decode3(s, g2);
  if (a.blk == 4) {
    if (b.blk != 3) return 0.0;
    std::swap(a, b);   // lambda row = m^T: read the p row's lambda coefficient
  }
  int kind = a.blk;
  const int lastp = s.n + p - 1, lastq = s.n + q - 1;
  int last[3];
  for (int x = 0; x < 3; ++x) last[x] = (kind < 3 && x == kind) ? lastp : lastq;
  int cl = (cls1(a.i[2], last[2], st.T) * st.NC + cls1(a.i[1], last[1], st.T)) * st.NC + cls1(a.i[0], last[0], st.T);
  const double* r = &st.rec[kind][(size_t)st.cmap[kind][cl] * st.RU];
  if (b.blk == 4) return kind == 3 ? r[st.RU - 1] : 0.0;
  const int nbox = kind < 3 ? 2 : 3;
  for (int k = 0; k < nbox; ++k) {
    Box3 bx = box_of(p, kind, k);
    if (bx.blk != b.blk) continue;
    int c = bx.axis, o1 = (c + 1) % 3, o2 = (c + 2) % 3;
    int da = b.i[c] - a.i[c] - bx.org, e1 = b.i[o1] - a.i[o1] + q, e2 = b.i[o2] - a.i[o2] + q;
    if (da < 0 || da >= bx.len || e1 < 0 || e1 >= W || e2 < 0 || e2 >= W) return 0.0;
    return r[box_start(p, k) + (da * W + e1) * W + e2];
  }
  return 0.0;
}

int build_level_only3(const igamg_problem& pr, HierarchyHost3& H, std::string& err) {
  const int p = pr.p, nf = pr.n_fine;
  H.p = p; H.L = 1; H.n_fine = nf; H.sigma = pr.sigma; H.nu = pr.nu;
  H.cpen = pr.c_penalty > 0 ? pr.c_penalty : 4.0 * (p - 1);
  H.lev.resize(1);
  auto& lv = H.lev[0];
  build_level1d(p, nf, pr.sigma, pr.nu, H.cpen * nf, lv.f);
  lv.sz = sizes3(p, nf);
  build_stencils3(p, lv.f, lv.sz, lv.st);
  (void)err;
  return IGAMG_OK;
}

namespace {
int build3(const igamg_problem& pr, HierarchyHost3& H, std::string& err, bool full);
}

int build_hierarchy3(const igamg_problem& pr, HierarchyHost3& H, std::string& err) { return build3(pr, H, err, true); }
int build_operators3(const igamg_problem& pr, HierarchyHost3& H, std::string& err) { return build3(pr, H, err, false); }

namespace {
int build3(const igamg_problem& pr, HierarchyHost3& H, std::string& err, bool full) {
  const int p = pr.p, L = pr.n_levels, nf = pr.n_fine;
  H.p = p; H.L = L; H.n_fine = nf; H.sigma = pr.sigma; H.nu = pr.nu;
  H.cpen = pr.c_penalty > 0 ? pr.c_penalty : 4.0 * (p - 1);
  const double pen_over_nu = H.cpen * nf;
  H.lev.resize(L);
  for (int l = 0; l < L; ++l) {
    int n = nf >> (L - 1 - l);
    auto& lv = H.lev[l];
    build_level1d(p, n, pr.sigma, pr.nu, pen_over_nu, lv.f);
    lv.sz = sizes3(p, n);
    build_stencils3(p, lv.f, lv.sz, lv.st);
    igamg_sizes& o = lv.pub;
    o.n = n;
    o.nx_ux = lv.sz.ni; o.ny_ux = lv.sz.nq;
    o.nx_uy = lv.sz.nq; o.ny_uy = lv.sz.ni;
    o.n_pdir = lv.sz.nq;
    o.n_ux = o.n_uy = lv.sz.n_uc;
    o.n_p = lv.sz.n_p; o.n_total = lv.sz.n_total;
    o.n_patches = 3 * lv.sz.nq * lv.sz.ni * lv.sz.ni;
    o.n_colours = 3 * p * (p + 1) * (p + 1);
    o.n_quad = p + 2;
    o.dim = 3; o.n_uz = lv.sz.n_uc;
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
  const bool mapped = pr.geometry == IGAMG_GEOM_HOLLOW_CYLINDER;
  const bool general = pr.beta_qp != nullptr || mapped;   // Oseen, mapped: per-row records
  H.geometry = pr.geometry;
  if (mapped) {
    // fine level assembled on the mapped domain; coarse levels whole-row Galerkin products
    const double ri = pr.r_inner > 0 ? pr.r_inner : 0.075, ro = pr.r_outer > 0 ? pr.r_outer : 0.225;
    int rc = assemble_mapped3(p, H.lev[L - 1], pr.sigma, pr.nu, H.cpen, ri, ro, 0.1, H, err);
    if (rc) return rc;
    for (int l = L - 2; l >= 0; --l)
      if ((rc = galerkin_rows3(p, H.lev[l + 1], H.lev[l], H.tp_free[l + 1], H.tq[l + 1], err))) return rc;
  } else if (general) {
    add_advection3(p, H.lev[L - 1].sz, pr.beta_qp, H.lev[L - 1].adv);
    for (int l = L - 2; l >= 0; --l)
      galerkin_adv3(p, H.lev[l + 1].sz, H.lev[l].sz, H.lev[l + 1].adv, H.tp_free[l + 1], H.tq[l + 1], H.lev[l].adv);
    for (int l = 0; l < L; ++l) rows_with_advection3(p, H.lev[l], H.lev[l].rows);
  }
  if (!full) return IGAMG_OK;
  for (int l = 1; l < L; ++l) {
    auto& lv = H.lev[l];
    int rc = general ? build_patches3(p, lv.f, lv.sz, lv.pt, err,
                                      [&](long long a, long long b) { return k_entry3_rows(lv, p, a, b); }, true)
                     : build_patches3(p, lv.f, lv.sz, lv.pt, err,
                                      [&](long long a, long long b) { return k_entry3(lv.f, lv.sz, a, b); }, false);
    if (rc) return rc;
  }
  {
    auto& lv = H.lev[0];
    int nd = (int)lv.sz.n_total;
    std::vector<double> K((size_t)nd * nd);
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j)
        K[(size_t)i * nd + j] = general ? k_entry3_rows(lv, p, i, j) : k_entry3(lv.f, lv.sz, i, j);
    if (!invert(K, nd, H.coarse_inv)) { err = "singular coarsest matrix"; return IGAMG_ESINGULAR; }
    H.ndof0 = nd;
  }
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
}  // namespace

}  // namespace igamg

// ---- host-only inspection (3D): the same entry points dispatch here for dim = 3 --------
namespace {
int host_build3(const igamg_problem* prob, int level, igamg::HierarchyHost3& H, bool full = true) {
  if (!(prob->sigma > 0) || !(prob->nu > 0)) return IGAMG_EINVAL;
  if (prob->n_levels < 1 || prob->n_fine < 1 || prob->n_fine % (1 << (prob->n_levels - 1))) return IGAMG_EINVAL;
  if (level < 0 || level >= prob->n_levels) return IGAMG_EINVAL;
  if (igamg::sizes3(prob->p, prob->n_fine >> (prob->n_levels - 1)).n_total > 4096) return IGAMG_EINVAL;
  std::string err;
  return full ? igamg::build_hierarchy3(*prob, H, err) : igamg::build_operators3(*prob, H, err);
}
}  // namespace

namespace igamg {

int host_level_matrix3(const igamg_problem* prob, int level, double* K, size_t cap, long long* n_out, bool records) {
  HierarchyHost3 H;
  int rc = host_build3(prob, level, H, false);
  if (rc) return rc;
  const auto& lv = H.lev[level];
  long long n = lv.sz.n_total;
  if (n_out) *n_out = n;
  if (!K) return IGAMG_OK;
  if (cap < (size_t)(n * n)) return IGAMG_EINVAL;
  for (long long i = 0; i < n; ++i)
    for (long long j = 0; j < n; ++j)
      K[i * n + j] = !lv.rows.empty() ? k_entry3_rows(lv, prob->p, i, j)
                     : (records ? k_entry3_records(lv, prob->p, i, j) : k_entry3(lv.f, lv.sz, i, j));
  return IGAMG_OK;
}

int host_prolongation3(const igamg_problem* prob, int level, double* P, size_t cap, long long* n_rows,
                       long long* n_cols) {
  if (level < 1) return IGAMG_EINVAL;
  HierarchyHost3 H;
  int rc = host_build3(prob, level, H);
  if (rc) return rc;
  const auto& f = H.lev[level].sz;
  const auto& c = H.lev[level - 1].sz;
  long long nr = f.n_total, nc = c.n_total;
  if (n_rows) *n_rows = nr;
  if (n_cols) *n_cols = nc;
  if (!P) return IGAMG_OK;
  if (cap < (size_t)(nr * nc)) return IGAMG_EINVAL;
  std::fill(P, P + nr * nc, 0.0);
  constexpr int WP = Transfer1D::WP;
  for (int blk = 0; blk < 4; ++blk) {
    const Transfer1D* T[3];
    for (int a = 0; a < 3; ++a) T[a] = (blk < 3 && a == blk) ? &H.tp_free[level] : &H.tq[level];
    long long rbase = blk < 3 ? blk * f.n_uc : f.n_u, cbase = blk < 3 ? blk * c.n_uc : c.n_u;
    for (int fz = 0; fz < T[2]->nf; ++fz)
      for (int fy = 0; fy < T[1]->nf; ++fy)
        for (int fx = 0; fx < T[0]->nf; ++fx)
          for (int kz = 0; kz < WP; ++kz)
            for (int ky = 0; ky < WP; ++ky)
              for (int kx = 0; kx < WP; ++kx) {
                int cz = T[2]->c0[fz] + kz, cy = T[1]->c0[fy] + ky, cx = T[0]->c0[fx] + kx;
                if (cz >= T[2]->nc || cy >= T[1]->nc || cx >= T[0]->nc) continue;
                double w = T[2]->pv[(size_t)fz * WP + kz] * T[1]->pv[(size_t)fy * WP + ky] * T[0]->pv[(size_t)fx * WP + kx];
                if (w == 0.0) continue;
                long long r = rbase + ((long long)fz * T[1]->nf + fy) * T[0]->nf + fx;
                long long col = cbase + ((long long)cz * T[1]->nc + cy) * T[0]->nc + cx;
                P[r * nc + col] += w;
              }
  }
  P[(nr - 1) * nc + nc - 1] = 1.0;
  return IGAMG_OK;
}

int host_patches3(const igamg_problem* prob, int level, int* colour, int* dofs, size_t cap_patches,
                  size_t cap_dofs, int* n_patches, int* maxl) {
  if (level < 1) return IGAMG_EINVAL;
  HierarchyHost3 H;
  int rc = host_build3(prob, level, H);
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

}  // namespace igamg
