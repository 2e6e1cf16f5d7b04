// Residual of the finest generalized-Oseen level with the advection term applied matrix-free:
// the (beta . grad u, v) integrals of Sec. 3.1 evaluated element by element at the (p+2)^2
// Gauss points, sum-factorised per direction, instead of read from per-row stencil records.
#pragma once
#include "kernels.cuh"

namespace igamg {
namespace dev {

// Tables of the matrix-free advection apply (device copies of HierarchyHost::adv_*).  On
// elements P .. n-1-P every local basis function is a uniform B-spline, so their tables are
// the same for all of them; those, and the class-stencil records of the rows in the interior
// class, also travel by value (kernel parameters: the multiply-adds take them as constant
// operands, with no load instruction).
constexpr int kAdvMaxPG = 4 * 5, kAdvMaxQG = 3 * 5, kAdvMaxRU = 7 * 5 + 6 * 5 + 1;   // p <= 3
template <typename T>
struct AdvTab {
  int n = 0;                                  // elements per direction (finest level)
  const T *bp = nullptr, *dp = nullptr;       // degree p: [(e*(p+1)+a)*G + g] values, derivatives
  const T *bq = nullptr, *dq = nullptr;       // degree p-1: [(e*p+a)*G + g]
  const T* beta = nullptr;                    // Gauss weight * beta, (2, nG, nG)
  int inner = 0;                              // 1: the interior copies below are valid
  T ibp[kAdvMaxPG], idp[kAdvMaxPG];           // interior element: [a*G + g]
  T ibq[kAdvMaxQG], idq[kAdvMaxQG];
  T rx[kAdvMaxRU], ry[kAdvMaxRU], rp[kAdvMaxRU];   // interior class records of u_x, u_y, p rows
};

constexpr int kAdvThreads = 256;              // one element per thread: (TE + P)^2 = 256

template <int P>
struct AdvShape {
  static constexpr int Q = P - 1, G = P + 2;
  static constexpr int E = 16;                // elements per tile side (one per thread)
  static constexpr int TE = E - P;            // owned index positions per tile side
  static constexpr int CW = E + P;            // coefficient positions per tile side
  static constexpr int W = CW + 1;            // row length of the staged tiles: one more column
                                              // for the zero-padded end of the pressure rows' box
  static constexpr int NXP = (P + 1) * G * E, NXQ = (Q + 1) * G * E;   // one table, one side
  static constexpr int NC = (P + 1) * (Q + 1);                        // local functions per component
  static constexpr int ELEMS = 3 * W * CW + 4 * (NXP + NXQ) + 2 * NC * kAdvThreads;
  template <typename T>
  static constexpr size_t smem() { return (size_t)ELEMS * sizeof(T); }
};

// One velocity component on one element: u = sum_{a,b} c[a][b] X_a(x) Y_b(y) with X of degree
// DX, Y of degree DY; out[a][b] = sum_q s(q) X_a Y_b (q), s = (w beta) . grad u at the Gauss
// points q, in four 1D contractions: (c, X) -> tv, td; (tv, td, Y) -> grad u per Gauss row;
// (s, X) -> z; (z, Y) -> out.  xb(a, g), xd(a, g), yb(b, g), yd(b, g) give the element's 1D
// basis values and derivatives at its Gauss points.
// bwx, bwy: the element's w * beta at its first Gauss point, rows nG apart.
template <int G, int DX, int DY, typename T, typename XB, typename XD, typename YB, typename YD>
__device__ __forceinline__ void adv_element(const T* __restrict__ sU, int cw, XB xb, XD xd, YB yb, YD yd,
                                            const T* __restrict__ bwx, const T* __restrict__ bwy, int nG,
                                            int lx, int ly, T* out) {
  T tv[DY + 1][G], td[DY + 1][G];
#pragma unroll
  for (int b = 0; b <= DY; ++b) {
    T c[DX + 1];
#pragma unroll
    for (int a = 0; a <= DX; ++a) c[a] = sU[(ly + b) * cw + lx + a];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      T v = T(0), d = T(0);
#pragma unroll
      for (int a = 0; a <= DX; ++a) {
        v = fma(c[a], xb(a, g), v);
        d = fma(c[a], xd(a, g), d);
      }
      tv[b][g] = v;
      td[b][g] = d;
    }
  }
  T r[DX + 1][DY + 1];
#pragma unroll
  for (int a = 0; a <= DX; ++a)
#pragma unroll
    for (int b = 0; b <= DY; ++b) r[a][b] = T(0);
#pragma unroll
  for (int gy = 0; gy < G; ++gy) {
    T yv[DY + 1], ydv[DY + 1];
#pragma unroll
    for (int b = 0; b <= DY; ++b) {
      yv[b] = yb(b, gy);
      ydv[b] = yd(b, gy);
    }
    T s[G];
#pragma unroll
    for (int gx = 0; gx < G; ++gx) {
      T ux = T(0), uy = T(0);
#pragma unroll
      for (int b = 0; b <= DY; ++b) {
        ux = fma(td[b][gx], yv[b], ux);
        uy = fma(tv[b][gx], ydv[b], uy);
      }
      s[gx] = fma(bwx[gy * nG + gx], ux, bwy[gy * nG + gx] * uy);
    }
#pragma unroll
    for (int a = 0; a <= DX; ++a) {
      T z = T(0);
#pragma unroll
      for (int gx = 0; gx < G; ++gx) z = fma(s[gx], xb(a, gx), z);
#pragma unroll
      for (int b = 0; b <= DY; ++b) r[a][b] = fma(z, yv[b], r[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a <= DX; ++a)
#pragma unroll
    for (int b = 0; b <= DY; ++b) out[(a * (DY + 1) + b) * kAdvThreads] = r[a][b];
}

// The Stokes part of one row (the class-stencil record st(j), Sec. 3.4's blocks as in row_KU)
// applied to the staged tiles: sA holds the first box's unknowns, sB the second's, both with
// row length W; (ax0, ay0) and (bx0, by0) are the tile positions of the boxes' first entries,
// WY0 and WY1 their extents in y.  The same terms in the same order and chains as row_KU with
// four chains on the class stencils, so the result equals that row's to the last bit.
template <int B0, int B1, int WY0, int WY1, typename T, typename ST>
__device__ __forceinline__ T stokes_row_tile(ST st, const T* sA, int ax0, int ay0, const T* sB, int bx0, int by0,
                                             int W, T lam) {
  T acc = T(0), acc1 = T(0), acc2 = T(0), acc3 = T(0);
#pragma unroll
  for (int j = 0; j < B0; ++j) {
    const int dx = j / WY0, dy = j - dx * WY0;
    const T v = sA[(ay0 + dy) * W + ax0 + dx];
    if (j & 1) acc1 = fma(st(j), v, acc1);
    else acc = fma(st(j), v, acc);
  }
#pragma unroll
  for (int j = 0; j < B1; ++j) {
    const int dx = j / WY1, dy = j - dx * WY1;
    const T v = sB[(by0 + dy) * W + bx0 + dx];
    if (j & 1) acc3 = fma(st(B0 + j), v, acc3);
    else acc2 = fma(st(B0 + j), v, acc2);
  }
  acc3 = fma(st(B0 + B1), lam, acc3);
  return (acc + acc1) + (acc2 + acc3);
}

// R = F - K U on the finest Oseen level for every row but lambda, with K = (Stokes part from
// the class stencils in L; L.srow must be null) + (advection, matrix-free from A).  One block
// per tile of TE x TE index positions (rows u_x(X, Y), u_y(X, Y), p(X, Y) with X, Y in the tile):
//  1. the u_x, u_y and p coefficients of the positions around the tile (X0 - P .. X0 + TE + P
//     in each direction) and the 1D tables of its E x E elements (X0 - P .. X0 + TE - 1) are
//     staged in shared memory;
//  2. each thread evaluates one element's advection integrals for both components into
//     shared memory (zero for positions outside the mesh);
//  3. each owned row sums the contributions of the elements in its support in a fixed order
//     (deterministic), subtracts the Stokes part (its class-stencil record applied to the
//     staged tiles of u_x, u_y and p), and writes R; per-block partial sums of R^2 and m.p go
//     to part[2 * block], as in k_residual.
// Blocks per SM: FP64 one (the registers of the FP64 element evaluation), FP32 three (p = 2)
// or two (p = 3), the most that fit without register spills.
template <int P, typename T>
__global__ void __launch_bounds__(kAdvThreads, sizeof(T) == 8 ? 1 : (P == 2 ? 3 : 2))
    k_residual_adv(LevelTab<T> L, AdvTab<T> A, const T* __restrict__ U, const T* __restrict__ F, T* __restrict__ R,
                   double* __restrict__ part, int tiles_x) {
  using S = AdvShape<P>;
  constexpr int Q = S::Q, G = S::G, E = S::E, TE = S::TE, CW = S::CW;
  extern __shared__ __align__(16) unsigned char adv_smem[];
  __shared__ double sh[64];
  constexpr int W = S::W;
  T* sUx = reinterpret_cast<T*>(adv_smem);
  T* sUy = sUx + W * CW;
  T* sP = sUy + W * CW;
  T* xbp = sP + W * CW;                     // x side: degree p values, derivatives, then p-1
  T* xdp = xbp + S::NXP;
  T* xbq = xdp + S::NXP;
  T* xdq = xbq + S::NXQ;
  T* ybp = xdq + S::NXQ;                    // y side
  T* ydp = ybp + S::NXP;
  T* ybq = ydp + S::NXP;
  T* ydq = ybq + S::NXQ;
  T* cx = ydq + S::NXQ;                     // element contributions, u_x then u_y
  T* cy = cx + S::NC * kAdvThreads;
  const int t = threadIdx.x, n = A.n, nG = n * G;
  const int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
  const int X0 = bx * TE, Y0 = by * TE;
  const int lx = t % E, ly = t / E, ex = X0 - P + lx, ey = Y0 - P + ly;
  const bool elem = ex >= 0 && ex < n && ey >= 0 && ey < n;

  // 1. coefficients (zero outside the index ranges: the eliminated normal components too)
  const int nu = L.n_ux + L.n_uy;
  for (int i = t; i < W * CW; i += kAdvThreads) {
    const int ix = X0 - P + i % W, iy = Y0 - P + i / W;
    const bool okq = ix >= 0 && ix <= L.lastq;
    sUx[i] = (ix >= 1 && ix <= L.nint && iy >= 0 && iy <= L.lastq) ? U[iy * L.nxu + ix - 1] : T(0);
    sUy[i] = (okq && iy >= 1 && iy <= L.nint) ? U[L.n_ux + (iy - 1) * L.npd + ix] : T(0);
    sP[i] = (okq && iy >= 0 && iy <= L.lastq) ? U[nu + iy * L.npd + ix] : T(0);
  }
  for (int i = t; i < S::NXP; i += kAdvThreads) {
    const int l = i % E, ag = i / E, ex = X0 - P + l, ey = Y0 - P + l;
    const bool okx = ex >= 0 && ex < n, oky = ey >= 0 && ey < n;
    xbp[i] = okx ? A.bp[(size_t)ex * (P + 1) * G + ag] : T(0);
    xdp[i] = okx ? A.dp[(size_t)ex * (P + 1) * G + ag] : T(0);
    ybp[i] = oky ? A.bp[(size_t)ey * (P + 1) * G + ag] : T(0);
    ydp[i] = oky ? A.dp[(size_t)ey * (P + 1) * G + ag] : T(0);
  }
  for (int i = t; i < S::NXQ; i += kAdvThreads) {
    const int l = i % E, ag = i / E, ex = X0 - P + l, ey = Y0 - P + l;
    const bool okx = ex >= 0 && ex < n, oky = ey >= 0 && ey < n;
    xbq[i] = okx ? A.bq[(size_t)ex * (Q + 1) * G + ag] : T(0);
    xdq[i] = okx ? A.dq[(size_t)ex * (Q + 1) * G + ag] : T(0);
    ybq[i] = oky ? A.bq[(size_t)ey * (Q + 1) * G + ag] : T(0);
    ydq[i] = oky ? A.dq[(size_t)ey * (Q + 1) * G + ag] : T(0);
  }
  __syncthreads();
  // 2. one element per thread
  {
    if (elem) {
      const T* bwx = A.beta + (size_t)(ey * G) * nG + ex * G;
      const T* bwy = bwx + (size_t)nG * nG;
      if (A.inner && ex >= P && ex < n - P && ey >= P && ey < n - P) {
        auto ibp = [&](int a, int g) { return A.ibp[a * G + g]; };
        auto idp = [&](int a, int g) { return A.idp[a * G + g]; };
        auto ibq = [&](int a, int g) { return A.ibq[a * G + g]; };
        auto idq = [&](int a, int g) { return A.idq[a * G + g]; };
        adv_element<G, P, Q>(sUx, W, ibp, idp, ibq, idq, bwx, bwy, nG, lx, ly, cx + t);
        adv_element<G, Q, P>(sUy, W, ibq, idq, ibp, idp, bwx, bwy, nG, lx, ly, cy + t);
      } else {
        auto sx = [&](const T* tab) { return [=](int a, int g) { return tab[(a * G + g) * E + lx]; }; };
        auto sy = [&](const T* tab) { return [=](int b, int g) { return tab[(b * G + g) * E + ly]; }; };
        adv_element<G, P, Q>(sUx, W, sx(xbp), sx(xdp), sy(ybq), sy(ydq), bwx, bwy, nG, lx, ly, cx + t);
        adv_element<G, Q, P>(sUy, W, sx(xbq), sx(xdq), sy(ybp), sy(ydp), bwx, bwy, nG, lx, ly, cy + t);
      }
    } else {
#pragma unroll
      for (int k = 0; k < S::NC; ++k) { cx[k * kAdvThreads + t] = T(0); cy[k * kAdvThreads + t] = T(0); }
    }
  }
  __syncthreads();
  // 3. owned rows
  constexpr int WQ = 2 * Q + 1, WPP = 2 * P + 1, B0 = WPP * WQ, B1 = 2 * P * WQ, RU = B0 + B1 + 1;
  constexpr int TCL = 2 * P + 1, NCL = 2 * TCL + 1;   // interior 1D position class, classes
  const T lam = U[L.n_total - 1];
  T r2 = T(0), mp = T(0);
  if (t < TE * TE) {
    const int ox = t % TE, oy = t / TE, X = X0 + ox, Y = Y0 + oy;
    if (X >= 1 && X <= L.nint && Y <= L.lastq) {           // u_x row: x-degree p, y-degree p-1
      const int g = Y * L.nxu + X - 1;
      T adv = T(0);
#pragma unroll
      for (int a = 0; a <= P; ++a)
#pragma unroll
        for (int b = 0; b <= Q; ++b) adv += cx[(a * (Q + 1) + b) * kAdvThreads + (oy + P - b) * E + ox + P - a];
      // box 0: u_x at (X - P .. X + P, Y - Q .. Y + Q); box 1: p at (X - P .. X + P - 1, Y - Q .. Y + Q)
      const int ccx = cls1d<P>(X, L.lastp), ccy = cls1d<P>(Y, L.lastq);
      T ku;
      if (A.inner && ccx == TCL && ccy == TCL) {
        ku = stokes_row_tile<B0, B1, WQ, WQ>([&](int j) { return A.rx[j]; }, sUx, ox, oy + P - Q, sP, ox, oy + P - Q, W, lam);
      } else {
        const T* st = L.sx + (ccx * NCL + ccy) * RU;
        ku = stokes_row_tile<B0, B1, WQ, WQ>([=](int j) { return st[j]; }, sUx, ox, oy + P - Q, sP, ox, oy + P - Q, W, lam);
      }
      const T r = F[g] - ku - adv;
      R[g] = r;
      r2 = fma(r, r, r2);
    }
    if (X <= L.lastq && Y >= 1 && Y <= L.nint) {           // u_y row: x-degree p-1, y-degree p
      const int g = L.n_ux + (Y - 1) * L.npd + X;
      T adv = T(0);
#pragma unroll
      for (int a = 0; a <= Q; ++a)
#pragma unroll
        for (int b = 0; b <= P; ++b) adv += cy[(a * (P + 1) + b) * kAdvThreads + (oy + P - b) * E + ox + P - a];
      // box 0: u_y at (X - Q .. X + Q, Y - P .. Y + P); box 1: p at (X - Q .. X + Q, Y - P .. Y + P - 1)
      const int ccx = cls1d<P>(X, L.lastq), ccy = cls1d<P>(Y, L.lastp);
      T ku;
      if (A.inner && ccx == TCL && ccy == TCL) {
        ku = stokes_row_tile<B0, B1, WPP, 2 * P>([&](int j) { return A.ry[j]; }, sUy, ox + P - Q, oy, sP, ox + P - Q, oy, W, lam);
      } else {
        const T* st = L.sy + (ccx * NCL + ccy) * RU;
        ku = stokes_row_tile<B0, B1, WPP, 2 * P>([=](int j) { return st[j]; }, sUy, ox + P - Q, oy, sP, ox + P - Q, oy, W, lam);
      }
      const T r = F[g] - ku - adv;
      R[g] = r;
      r2 = fma(r, r, r2);
    }
    if (X <= L.lastq && Y <= L.lastq) {                    // pressure row: Stokes part only
      const int k = Y * L.npd + X, g = nu + k;
      // box 0: u_x at (X - Q .. X + P + 1, Y - Q .. Y + Q), its last column zero-padded;
      // box 1: u_y at (X - Q .. X + Q, Y - Q .. Y + P)
      const int ccx = cls1d<P>(X, L.lastq), ccy = cls1d<P>(Y, L.lastq);
      T ku;
      if (A.inner && ccx == TCL && ccy == TCL) {
        ku = stokes_row_tile<B0, B1, WQ, 2 * P>([&](int j) { return A.rp[j]; }, sUx, ox + P - Q, oy + P - Q, sUy,
                                                ox + P - Q, oy + P - Q, W, lam);
      } else {
        const T* st = L.sp + (ccx * NCL + ccy) * RU;
        ku = stokes_row_tile<B0, B1, WQ, 2 * P>([=](int j) { return st[j]; }, sUx, ox + P - Q, oy + P - Q, sUy,
                                                ox + P - Q, oy + P - Q, W, lam);
      }
      const T r = F[g] - ku;
      R[g] = r;
      r2 = fma(r, r, r2);
      mp = mean_coef<P>(L, k) * U[g];
    }
  }
  block_partials<T>(r2, mp, sh, part);
}

}  // namespace dev
}  // namespace igamg
