// Device kernels of the V-cycle (Algorithm 1 with the Schwarz smoothers of Sec. 5.2),
// templated on the streamfunction degree P and on the value type T (double or float).
//
// GB300 note: FP64 issue rate is a small fraction of FP32, so every kernel spends as few
// FP64 instructions as it can: rows use precomputed class stencils (one FMA per
// neighbour), all index arithmetic is 32-bit integer, and the smoother keeps all 32
// lanes of a warp busy (four 8-DOF patches per warp).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace igamg {
namespace dev {

template <typename T>
struct LevelTab {
  int n, nxu, npd, nint, lastp, lastq;   // nxu = n+p-2 = nint, npd = n+p-1, lastp = n+p-1, lastq = n+p-2
  int n_ux, n_uy, n_p, n_total;
  const T *sx, *sy, *sp;                 // class stencils (see Stencils in igamg_internal.h)
};

template <typename T>
struct Xfer {                            // 1D prolongation, two banded views
  int nf, nc;
  const int *c0, *f0;
  const T *pv, *rv;
};

constexpr int kWP = 3, kWR = 5;          // Transfer1D::WP / WR

// largest local system of a patch for even n >= 2 (the corner / whole-domain patches):
// 12 + 9 DOFs for P = 2, 24 + 16 for P = 3
template <int P>
struct MaxLocal { static constexpr int value = P == 2 ? 21 : 40; };

// acc = sum_s a[s] r[s] for s < nl <= ML, unrolled so that all loads issue together.
template <int ML, typename T>
__device__ __forceinline__ T dot_bounded(const T* __restrict__ a, const T* r, int nl) {
  T s0 = T(0), s1 = T(0);
#pragma unroll
  for (int s = 0; s < ML; s += 2) {
    if (s < nl) s0 = fma(a[s], r[s], s0);
    if (s + 1 < ML && s + 1 < nl) s1 = fma(a[s + 1], r[s + 1], s1);
  }
  return s0 + s1;
}

template <int P>
__host__ __device__ __forceinline__ int cls1d(int i, int last) {
  constexpr int TC = 2 * P + 1;
  return i < TC ? i : (last - i < TC ? 2 * TC - (last - i) : TC);
}

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// (K U)_g for one row g (not the lambda row): Sec. 3.4 blocks [A -B; B^T 0] plus m lambda.
template <int P, typename T>
__host__ __device__ __forceinline__ T row_KU(const LevelTab<T>& L, const T* __restrict__ U, int g) {
  constexpr int Q = P - 1, TC = 2 * P + 1, NC = 2 * TC + 1;
  constexpr int WQ = 2 * Q + 1, WPP = 2 * P + 1, RX = (4 * P + 1) * WQ, RP = 4 * P * WQ + 1;
  const T* ux = U;
  const T* uy = U + L.n_ux;
  const T* pr = U + L.n_ux + L.n_uy;
  T acc = T(0), acc2 = T(0);   // two chains: shorter FP64 dependency
  if (g < L.n_ux) {
    int iy = g / L.nxu, ix = g - iy * L.nxu + 1;
    const T* st = L.sx + (cls1d<P>(ix, L.lastp) * NC + cls1d<P>(iy, L.lastq)) * RX;
#pragma unroll
    for (int dx = -P; dx <= P; ++dx) {
      int jx = clampi(ix + dx, 1, L.nint) - 1;
#pragma unroll
      for (int dy = -Q; dy <= Q; ++dy) {
        int jy = clampi(iy + dy, 0, L.lastq);
        acc = fma(st[(dx + P) * WQ + dy + Q], ux[jy * L.nxu + jx], acc);
      }
    }
#pragma unroll
    for (int kx = -P; kx <= P - 1; ++kx) {
      int jx = clampi(ix + kx, 0, L.lastq);
#pragma unroll
      for (int dy = -Q; dy <= Q; ++dy) {
        int jy = clampi(iy + dy, 0, L.lastq);
        acc2 = fma(st[WPP * WQ + (kx + P) * WQ + dy + Q], pr[jy * L.npd + jx], acc2);
      }
    }
  } else if (g < L.n_ux + L.n_uy) {
    int r = g - L.n_ux;
    int iy = r / L.npd + 1, ix = r - (iy - 1) * L.npd;
    const T* st = L.sy + (cls1d<P>(ix, L.lastq) * NC + cls1d<P>(iy, L.lastp)) * RX;
#pragma unroll
    for (int dx = -Q; dx <= Q; ++dx) {
      int jx = clampi(ix + dx, 0, L.lastq);
#pragma unroll
      for (int dy = -P; dy <= P; ++dy) {
        int jy = clampi(iy + dy, 1, L.nint) - 1;
        acc = fma(st[(dx + Q) * WPP + dy + P], uy[jy * L.npd + jx], acc);
      }
    }
#pragma unroll
    for (int dx = -Q; dx <= Q; ++dx) {
      int jx = clampi(ix + dx, 0, L.lastq);
#pragma unroll
      for (int ky = -P; ky <= P - 1; ++ky) {
        int jy = clampi(iy + ky, 0, L.lastq);
        acc2 = fma(st[WQ * WPP + (dx + Q) * (2 * P) + ky + P], pr[jy * L.npd + jx], acc2);
      }
    }
  } else {
    int r = g - L.n_ux - L.n_uy;
    int ky = r / L.npd, kx = r - ky * L.npd;
    const T* st = L.sp + (cls1d<P>(kx, L.lastq) * NC + cls1d<P>(ky, L.lastq)) * RP;
#pragma unroll
    for (int s = -Q; s <= P; ++s) {
      int ix = clampi(kx + s, 1, L.nint) - 1;
#pragma unroll
      for (int dy = -Q; dy <= Q; ++dy) {
        int iy = clampi(ky + dy, 0, L.lastq);
        acc = fma(st[(s + Q) * WQ + dy + Q], ux[iy * L.nxu + ix], acc);
      }
    }
#pragma unroll
    for (int dx = -Q; dx <= Q; ++dx) {
      int ix = clampi(kx + dx, 0, L.lastq);
#pragma unroll
      for (int s = -Q; s <= P; ++s) {
        int iy = clampi(ky + s, 1, L.nint) - 1;
        acc2 = fma(st[2 * P * WQ + (dx + Q) * (2 * P) + s + Q], uy[iy * L.npd + ix], acc2);
      }
    }
    acc = fma(st[RP - 1], U[L.n_total - 1], acc);
  }
  return acc + acc2;
}

// m_k for a pressure row (the last stencil entry).
template <int P, typename T>
__device__ __forceinline__ T mean_coef(const LevelTab<T>& L, int r) {
  constexpr int Q = P - 1, TC = 2 * P + 1, NC = 2 * TC + 1, RP = 4 * P * (2 * Q + 1) + 1;
  int ky = r / L.npd, kx = r - ky * L.npd;
  return L.sp[(cls1d<P>(kx, L.lastq) * NC + cls1d<P>(ky, L.lastq)) * RP + RP - 1];
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// R = F - K U for every row but lambda; per-block partial sums of R^2 and of m.p (double).
template <int P, typename T>
__global__ void __launch_bounds__(256) k_residual(LevelTab<T> L, const T* __restrict__ U, const T* __restrict__ F,
                                                  T* __restrict__ R, double* __restrict__ part) {
  __shared__ double sh[32];
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, mp = 0.0;
  if (g < L.n_total - 1) {
    T r = F[g] - row_KU<P>(L, U, g);
    R[g] = r;
    r2 = (double)r * (double)r;
    int off = g - L.n_ux - L.n_uy;
    if (off >= 0) mp = (double)mean_coef<P>(L, off) * (double)U[g];
  }
  double s1 = block_sum(r2, sh);
  double s2 = block_sum(mp, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1; part[2 * blockIdx.x + 1] = s2; }
}

// lambda row and ||R||^2 from the partials (one block, fixed order).
template <typename T>
__global__ void k_residual_finish(int n_total, const T* __restrict__ F, T* __restrict__ R,
                                  const double* __restrict__ part, int nparts, double* __restrict__ norm2) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) { a += part[2 * i]; b += part[2 * i + 1]; }
  double s1 = block_sum(a, sh);
  double s2 = block_sum(b, sh);
  if (threadIdx.x == 0) {
    double rl = (double)F[n_total - 1] - s2;
    R[n_total - 1] = (T)rl;
    if (norm2) *norm2 = s1 + rl * rl;
  }
}

// One colour of the multiplicative Schwarz sweep (eq. MSM).  Blocks [0, nb8): four
// 8-DOF patches per warp, lane = (patch, local row); the local residual row, then the
// bordered local inverse applied through shuffles.  Blocks [nb8, ...): one warp per
// larger (wall) patch.  Same-colour patches share no DOF and are not coupled by K.
template <int P, typename T>
__global__ void __launch_bounds__(256) k_mult_colour(LevelTab<T> L, T* __restrict__ U, const T* __restrict__ F,
                                                     const int* __restrict__ dofs, const int* __restrict__ cls,
                                                     const T* __restrict__ cinv, const int* __restrict__ nloc,
                                                     int maxl, int first, int n8, int ngen, int nb8) {
  int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if ((int)blockIdx.x < nb8) {
    int grp = (blockIdx.x * 8 + wib) * 4 + (lane >> 3);
    int row = lane & 7;
    bool active = grp < n8;
    int patch = first + (active ? grp : 0);
    int g = dofs[patch * maxl + row];
    T r = active ? F[g] - row_KU<P>(L, U, g) : T(0);
    const T* A = cinv + ((size_t)cls[patch] * maxl + row) * maxl;
    T d = T(0);
#pragma unroll
    for (int s = 0; s < 8; ++s) d = fma(A[s], __shfl_sync(0xffffffffu, r, (lane & ~7) + s), d);
    if (active) U[g] += d;
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  int w = ((int)blockIdx.x - nb8) * 8 + wib;
  if (w >= ngen) return;
  int patch = first + n8 + w;
  int c = cls[patch], nl = nloc[c];
  T* r = sh + wib * maxl;
  const int* pd = dofs + (size_t)patch * maxl;
  for (int k = lane; k < nl; k += 32) { int g = pd[k]; r[k] = F[g] - row_KU<P>(L, U, g); }
  __syncwarp();
  const T* A = cinv + (size_t)c * maxl * maxl;
  for (int k = lane; k < nl; k += 32) U[pd[k]] += dot_bounded<MaxLocal<P>::value>(A + (size_t)k * maxl, r, nl);
}

// Additive sweep (eq. ASM), part 1: local corrections from one common residual, kept per patch.
template <int P, typename T>
__global__ void __launch_bounds__(256) k_add_local(const T* __restrict__ R, const int* __restrict__ dofs,
                                                   const int* __restrict__ cls, const T* __restrict__ cinv,
                                                   const int* __restrict__ nloc, int maxl, int count,
                                                   T* __restrict__ delta) {
  extern __shared__ unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= count) return;
  int c = cls[warp], nl = nloc[c];
  T* r = sh + (threadIdx.x >> 5) * maxl;
  const int* pd = dofs + (size_t)warp * maxl;
  for (int k = lane; k < nl; k += 32) r[k] = R[pd[k]];
  __syncwarp();
  const T* A = cinv + (size_t)c * maxl * maxl;
  for (int k = lane; k < nl; k += 32)
    delta[(size_t)warp * maxl + k] = dot_bounded<MaxLocal<P>::value>(A + (size_t)k * maxl, r, nl);
}

// Additive sweep, part 2: U_g += eta * (sum of the corrections of the patches holding g).
template <typename T>
__global__ void k_add_gather(int n, T* __restrict__ U, const T* __restrict__ delta, const int* __restrict__ off,
                             const int* __restrict__ idx, T eta) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  T s = T(0);
  for (int j = off[g]; j < off[g + 1]; ++j) s += delta[idx[j]];
  if (off[g + 1] > off[g]) U[g] += eta * s;
}

// block of a coarse/fine vector: (x count, first entry, which 1D views in x and y)
template <typename T>
struct BlockView { int x, y, nx; const T* base; };

// g_c = P^T r_f (lambda copied); one thread per coarse entry.
template <typename T>
__global__ void k_restrict(LevelTab<T> Lf, LevelTab<T> Lc, Xfer<T> tp, Xfer<T> tq, const T* __restrict__ rf,
                           T* __restrict__ gc) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lc.n_total) return;
  if (g == Lc.n_total - 1) { gc[g] = rf[Lf.n_total - 1]; return; }
  int cx, cy, fnx;
  const T* src;
  bool bx_p, by_p;
  if (g < Lc.n_ux) { cy = g / Lc.nxu; cx = g - cy * Lc.nxu; bx_p = true; by_p = false; src = rf; fnx = Lf.nxu; }
  else if (g < Lc.n_ux + Lc.n_uy) { int r = g - Lc.n_ux; cy = r / Lc.npd; cx = r - cy * Lc.npd; bx_p = false; by_p = true; src = rf + Lf.n_ux; fnx = Lf.npd; }
  else { int r = g - Lc.n_ux - Lc.n_uy; cy = r / Lc.npd; cx = r - cy * Lc.npd; bx_p = false; by_p = false; src = rf + Lf.n_ux + Lf.n_uy; fnx = Lf.npd; }
  const int* fx0p = bx_p ? tp.f0 : tq.f0; const T* rx = bx_p ? tp.rv : tq.rv; int nfx = bx_p ? tp.nf : tq.nf;
  const int* fy0p = by_p ? tp.f0 : tq.f0; const T* ry = by_p ? tp.rv : tq.rv; int nfy = by_p ? tp.nf : tq.nf;
  int fx0 = fx0p[cx], fy0 = fy0p[cy];
  T acc = T(0);
#pragma unroll
  for (int ky = 0; ky < kWR; ++ky) {
    int fy = fy0 + ky;
    T wy = ry[cy * kWR + ky];
    if (fy >= nfy) continue;
    T s = T(0);
#pragma unroll
    for (int kx = 0; kx < kWR; ++kx) {
      int fx = fx0 + kx;
      if (fx >= nfx) continue;
      s = fma(rx[cx * kWR + kx], src[fy * fnx + fx], s);
    }
    acc = fma(wy, s, acc);
  }
  gc[g] = acc;
}

// u_f += P u_c (lambda added); one thread per fine entry.
template <typename T>
__global__ void k_prolong_add(LevelTab<T> Lf, LevelTab<T> Lc, Xfer<T> tp, Xfer<T> tq, const T* __restrict__ uc,
                              T* __restrict__ uf) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lf.n_total) return;
  if (g == Lf.n_total - 1) { uf[g] += uc[Lc.n_total - 1]; return; }
  int fx, fy, cnx;
  const T* src;
  bool bx_p, by_p;
  if (g < Lf.n_ux) { fy = g / Lf.nxu; fx = g - fy * Lf.nxu; bx_p = true; by_p = false; src = uc; cnx = Lc.nxu; }
  else if (g < Lf.n_ux + Lf.n_uy) { int r = g - Lf.n_ux; fy = r / Lf.npd; fx = r - fy * Lf.npd; bx_p = false; by_p = true; src = uc + Lc.n_ux; cnx = Lc.npd; }
  else { int r = g - Lf.n_ux - Lf.n_uy; fy = r / Lf.npd; fx = r - fy * Lf.npd; bx_p = false; by_p = false; src = uc + Lc.n_ux + Lc.n_uy; cnx = Lc.npd; }
  const int* cx0p = bx_p ? tp.c0 : tq.c0; const T* px = bx_p ? tp.pv : tq.pv; int ncx = bx_p ? tp.nc : tq.nc;
  const int* cy0p = by_p ? tp.c0 : tq.c0; const T* py = by_p ? tp.pv : tq.pv; int ncy = by_p ? tp.nc : tq.nc;
  int cx0 = cx0p[fx], cy0 = cy0p[fy];
  T acc = T(0);
#pragma unroll
  for (int ky = 0; ky < kWP; ++ky) {
    int cy = cy0 + ky;
    if (cy >= ncy) continue;
    T s = T(0);
#pragma unroll
    for (int kx = 0; kx < kWP; ++kx) {
      int cx = cx0 + kx;
      if (cx >= ncx) continue;
      s = fma(px[fx * kWP + kx], src[cy * cnx + cx], s);
    }
    acc = fma(py[fy * kWP + ky], s, acc);
  }
  uf[g] += acc;
}

// U = K_0^{-1} G (dense inverse, one block).
template <typename T>
__global__ void k_coarse(int n, const T* __restrict__ Kinv, const T* __restrict__ G, T* __restrict__ U) {
  extern __shared__ unsigned char smem_raw[];
  T* g = reinterpret_cast<T*>(smem_raw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = G[i];
  __syncthreads();
  int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x >> 5; i < n; i += nw) {
    const T* row = Kinv + (size_t)i * n;
    T acc = T(0);
    for (int j = lane; j < n; j += 32) acc = fma(row[j], g[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) U[i] = acc;
  }
}

// ---- mixed precision helpers ---------------------------------------------------------
__global__ void k_to_float(int n, const double* __restrict__ a, float* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// Discrete streamfunction of a velocity correction by integration along y of its u_x
// block: psi(ix, k+1) = psi(ix, k) + e_x(ix, k) / dcoef_k, psi = 0 on the bottom wall.
// One thread per interior column; psi stored on the (n+p-2)^2 interior, FP64.
__global__ void k_integrate_psi(int nint, int nxu, const double* __restrict__ inv_dcoef,
                                const float* __restrict__ e, double* __restrict__ psi) {
  int ix = blockIdx.x * blockDim.x + threadIdx.x;  // interior column 0..nint-1
  if (ix >= nint) return;
  double acc = 0.0;
  for (int k = 0; k < nint; ++k) {
    acc = fma((double)e[k * nxu + ix], inv_dcoef[k], acc);
    psi[k * nint + ix] = acc;
  }
}

// U += (curl psi, e_p, e_lambda) in FP64 (exact discrete curl: divergence-free to round-off).
template <typename LT>
__global__ void k_curl_update(LT L, const double* __restrict__ dcoef, const double* __restrict__ psi,
                              const float* __restrict__ e, double* __restrict__ U) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_total) return;
  int ni = L.nint;
  auto PS = [&](int ix, int iy) { return (ix < 1 || ix > ni || iy < 1 || iy > ni) ? 0.0 : psi[(iy - 1) * ni + ix - 1]; };
  if (g < L.n_ux) {
    int ky = g / L.nxu, ix = g - ky * L.nxu + 1;
    U[g] += dcoef[ky] * (PS(ix, ky + 1) - PS(ix, ky));
  } else if (g < L.n_ux + L.n_uy) {
    int r = g - L.n_ux;
    int iy = r / L.npd + 1, kx = r - (iy - 1) * L.npd;
    U[g] -= dcoef[kx] * (PS(kx + 1, iy) - PS(kx, iy));
  } else {
    U[g] += (double)e[g];
  }
}

}  // namespace dev
}  // namespace igamg
