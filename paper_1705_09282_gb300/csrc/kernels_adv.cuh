// Residual of the finest generalized-Oseen level with the advection term applied matrix-free:
// the (beta . grad u, v) integrals of Sec. 3.1 evaluated element by element at the (p+2)^2
// Gauss points, sum-factorised per direction, instead of read from per-row stencil records.
#pragma once
#include "kernels.cuh"

namespace igamg {
namespace dev {

// Tables of the matrix-free advection apply (device copies of HierarchyHost::adv_*).
template <typename T>
struct AdvTab {
  int n = 0;                                  // elements per direction (finest level)
  const T *bp = nullptr, *dp = nullptr;       // degree p: [(e*(p+1)+a)*G + g] values, derivatives
  const T *bq = nullptr, *dq = nullptr;       // degree p-1: [(e*p+a)*G + g]
  const T* beta = nullptr;                    // Gauss weight * beta, (2, nG, nG)
};

constexpr int kAdvThreads = 256;              // one element per thread: (TE + P)^2 = 256

template <int P>
struct AdvShape {
  static constexpr int Q = P - 1, G = P + 2;
  static constexpr int E = 16;                // elements per tile side (one per thread)
  static constexpr int TE = E - P;            // owned index positions per tile side
  static constexpr int CW = E + P;            // coefficient positions per tile side
  static constexpr int NXP = (P + 1) * G * E, NXQ = (Q + 1) * G * E;   // one table, one side
  static constexpr int NC = (P + 1) * (Q + 1);                        // local functions per component
  static constexpr int ELEMS = 2 * CW * CW + 4 * (NXP + NXQ) + 2 * NC * kAdvThreads;
  template <typename T>
  static constexpr size_t smem() { return (size_t)ELEMS * sizeof(T); }
};

// One velocity component on one element: u = sum_{a,b} c[a][b] X_a(x) Y_b(y) with X of degree
// DX, Y of degree DY; out[a][b] = sum_q s(q) X_a Y_b (q), s = (w beta) . grad u at the Gauss
// points q, in four 1D contractions: (c, X) -> tv, td; (tv, td, Y) -> grad u per Gauss row;
// (s, X) -> z; (z, Y) -> out.  X tables are [(a*G+g)*E + lx], Y tables [(b*G+g)*E + ly].
template <int G, int E, int DX, int DY, typename T>
__device__ __forceinline__ void adv_element(const T* __restrict__ sU, int cw, const T* __restrict__ xb,
                                            const T* __restrict__ xd, const T* __restrict__ yb,
                                            const T* __restrict__ yd, const T* __restrict__ bwx,
                                            const T* __restrict__ bwy, int nG, int lx, int ly, T* out) {
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
        v = fma(c[a], xb[(a * G + g) * E + lx], v);
        d = fma(c[a], xd[(a * G + g) * E + lx], d);
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
      yv[b] = yb[(b * G + gy) * E + ly];
      ydv[b] = yd[(b * G + gy) * E + ly];
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
      for (int gx = 0; gx < G; ++gx) z = fma(s[gx], xb[(a * G + gx) * E + lx], z);
#pragma unroll
      for (int b = 0; b <= DY; ++b) r[a][b] = fma(z, yv[b], r[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a <= DX; ++a)
#pragma unroll
    for (int b = 0; b <= DY; ++b) out[(a * (DY + 1) + b) * kAdvThreads] = r[a][b];
}

// R = F - K U on the finest Oseen level for every row but lambda, with K = (Stokes part from
// the class stencils in L; L.srow must be null) + (advection, matrix-free from A).  One block
// per tile of TE x TE index positions (rows u_x(X, Y), u_y(X, Y), p(X, Y) with X, Y in the tile):
//  1. the U coefficients of the CW x CW positions around the tile and the 1D tables of its
//     E x E elements (positions X - P .. X + TE - 1) are staged in shared memory;
//  2. each thread evaluates one element's advection integrals for both components into
//     shared memory (zero for positions outside the mesh);
//  3. each owned row sums the contributions of the elements in its support in a fixed order
//     (deterministic), subtracts the Stokes part, and writes R; per-block partial sums of R^2
//     and m.p go to part[2 * block], as in k_residual.
template <int P, typename T>
__global__ void __launch_bounds__(kAdvThreads, sizeof(T) == 8 ? 1 : (P == 2 ? 4 : 2)) k_residual_adv(LevelTab<T> L, AdvTab<T> A, const T* __restrict__ U,
                                                              const T* __restrict__ F, T* __restrict__ R,
                                                              double* __restrict__ part, int tiles_x) {
  using S = AdvShape<P>;
  constexpr int Q = S::Q, G = S::G, E = S::E, TE = S::TE, CW = S::CW;
  extern __shared__ __align__(16) unsigned char adv_smem[];
  __shared__ double sh[64];
  T* sUx = reinterpret_cast<T*>(adv_smem);
  T* sUy = sUx + CW * CW;
  T* xbp = sUy + CW * CW;                   // x side: degree p values, derivatives, then p-1
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
  // 1. coefficients (zero outside the index ranges: the eliminated normal components too)
  for (int i = t; i < CW * CW; i += kAdvThreads) {
    const int ix = X0 - P + i % CW, iy = Y0 - P + i / CW;
    sUx[i] = (ix >= 1 && ix <= L.nint && iy >= 0 && iy <= L.lastq) ? U[iy * L.nxu + ix - 1] : T(0);
    sUy[i] = (ix >= 0 && ix <= L.lastq && iy >= 1 && iy <= L.nint) ? U[L.n_ux + (iy - 1) * L.npd + ix] : T(0);
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
    const int lx = t % E, ly = t / E, ex = X0 - P + lx, ey = Y0 - P + ly;
    if (ex >= 0 && ex < n && ey >= 0 && ey < n) {
      const T* bwx = A.beta + (size_t)(ey * G) * nG + ex * G;
      const T* bwy = bwx + (size_t)nG * nG;
      adv_element<G, E, P, Q>(sUx, CW, xbp, xdp, ybq, ydq, bwx, bwy, nG, lx, ly, cx + t);
      adv_element<G, E, Q, P>(sUy, CW, xbq, xdq, ybp, ydp, bwx, bwy, nG, lx, ly, cy + t);
    } else {
#pragma unroll
      for (int k = 0; k < S::NC; ++k) { cx[k * kAdvThreads + t] = T(0); cy[k * kAdvThreads + t] = T(0); }
    }
  }
  __syncthreads();
  // 3. owned rows
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
      const T r = F[g] - row_KU<P>(L, U, g) - adv;
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
      const T r = F[g] - row_KU<P>(L, U, g) - adv;
      R[g] = r;
      r2 = fma(r, r, r2);
    }
    if (X <= L.lastq && Y <= L.lastq) {                    // pressure row: Stokes part only
      const int k = Y * L.npd + X, g = L.n_ux + L.n_uy + k;
      const T r = F[g] - row_KU<P>(L, U, g);
      R[g] = r;
      r2 = fma(r, r, r2);
      mp = mean_coef<P>(L, k) * U[g];
    }
  }
  block_partials<T>(r2, mp, sh, part);
}

}  // namespace dev
}  // namespace igamg
