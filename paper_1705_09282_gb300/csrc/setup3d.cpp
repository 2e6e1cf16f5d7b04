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

int build_patches3(int p, const Level1D& L, const Sizes3& s, PatchTables& pt, std::string& err) {
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
          P_.key = std::make_tuple(fam, pos_class3(i, lo[0], hi[0], p), pos_class3(j, lo[1], hi[1], p),
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
  // bordered local inverses (zero-mean local pressure through m_j = int N^q_j), one per class
  auto local_inverse = [&](const P& P_, std::vector<double>& inv) -> bool {
    int nl = (int)P_.dofs.size(), nb = nl + 1;
    std::vector<double> Kb((size_t)nb * nb, 0.0);
    for (int r = 0; r < nl; ++r)
      for (int t = 0; t < nl; ++t) Kb[(size_t)r * nb + t] = k_entry3(L, s, P_.dofs[r], P_.dofs[t]);
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
  for (int c = 0; c < pt.n_cls8; ++c) {
    std::vector<double> inv;
    if (!local_inverse(all[rep8[c]], inv)) { err = "singular local patch matrix"; return IGAMG_ESINGULAR; }
    for (int r = 0; r < 8; ++r)
      for (int t = 0; t < 8; ++t) pt.cinv8[(size_t)c * 64 + r * 8 + t] = inv[(size_t)r * 9 + t];
  }
  build_row_slots(pt);
  return IGAMG_OK;
}

}  // namespace

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

int build_hierarchy3(const igamg_problem& pr, HierarchyHost3& H, std::string& err) {
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
  for (int l = 1; l < L; ++l) {
    auto& lv = H.lev[l];
    int rc = build_patches3(p, lv.f, lv.sz, lv.pt, err);
    if (rc) return rc;
  }
  {
    auto& lv = H.lev[0];
    int nd = (int)lv.sz.n_total;
    std::vector<double> K((size_t)nd * nd);
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) K[(size_t)i * nd + j] = k_entry3(lv.f, lv.sz, i, j);
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

}  // namespace igamg

// ---- host-only inspection (3D): the same entry points dispatch here for dim = 3 --------
namespace {
int host_build3(const igamg_problem* prob, int level, igamg::HierarchyHost3& H) {
  if (!(prob->sigma > 0) || !(prob->nu > 0)) return IGAMG_EINVAL;
  if (prob->n_levels < 1 || prob->n_fine < 1 || prob->n_fine % (1 << (prob->n_levels - 1))) return IGAMG_EINVAL;
  if (level < 0 || level >= prob->n_levels) return IGAMG_EINVAL;
  if (igamg::sizes3(prob->p, prob->n_fine >> (prob->n_levels - 1)).n_total > 4096) return IGAMG_EINVAL;
  std::string err;
  return igamg::build_hierarchy3(*prob, H, err);
}
}  // namespace

namespace igamg {

int host_level_matrix3(const igamg_problem* prob, int level, double* K, size_t cap, long long* n_out, bool records) {
  HierarchyHost3 H;
  int rc = host_build3(prob, level, H);
  if (rc) return rc;
  const auto& lv = H.lev[level];
  long long n = lv.sz.n_total;
  if (n_out) *n_out = n;
  if (!K) return IGAMG_OK;
  if (cap < (size_t)(n * n)) return IGAMG_EINVAL;
  for (long long i = 0; i < n; ++i)
    for (long long j = 0; j < n; ++j)
      K[i * n + j] = records ? k_entry3_records(lv, prob->p, i, j) : k_entry3(lv.f, lv.sz, i, j);
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
