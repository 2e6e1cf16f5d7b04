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
  const T* srow;                         // per-row records (general operators), or null
  const T* sext;                         // mapped domains: per velocity row, the 2p x 2p
                                         // coefficients on the other velocity component, or null
};

template <typename T>
struct Xfer {                            // 1D prolongation, two banded views
  int nf, nc;
  const int *c0, *f0;
  const T *pv, *rv;
};

constexpr int kWP = 3, kWR = 5;          // Transfer1D::WP / WR

// acc = sum_{s < nl} a[s] r[s] with four independent chains (loads issue together).
template <typename T>
__device__ __forceinline__ T dot_n(const T* __restrict__ a, const T* r, int nl) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int s = 0;
  for (; s + 4 <= nl; s += 4) {
    s0 = fma(a[s], r[s], s0);
    s1 = fma(a[s + 1], r[s + 1], s1);
    s2 = fma(a[s + 2], r[s + 2], s2);
    s3 = fma(a[s + 3], r[s + 3], s3);
  }
  for (; s < nl; ++s) s0 = fma(a[s], r[s], s0);
  return (s0 + s1) + (s2 + s3);
}

template <int P>
__host__ __device__ __forceinline__ int cls1d(int i, int last) {
  constexpr int TC = 2 * P + 1;
  return i < TC ? i : (last - i < TC ? 2 * TC - (last - i) : TC);
}

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// (K U)_g for one row g (not the lambda row): Sec. 3.4 blocks [A -B; B^T 0] plus m lambda.
//
// Every row is two boxes of neighbours (velocity part, then pressure or second velocity
// part) plus the m lambda term.  All three row kinds run the same unconditional loops
// over fixed-size, zero-padded stencil records with clamped (always valid) neighbour
// indices: no lane diverges on the row kind (each FP64 instruction already costs 64 issue
// cycles per warp on GB300) and every load can be issued ahead of the FMAs.
// PART = 2: the whole row; PART = 0: box 0 only; PART = 1: box 1 and the lambda term (the
// split form lets two warps share one row's multiply-adds, see k_mult_colour_split).
// CH = 4: four independent multiply-add chains (latency-bound launches); CH = 2: one chain per
// box and two fewer FP64 adds per row (throughput-bound lockstep batches).
template <int P, typename T, int PART = 2, int CH = 4>
__host__ __device__ __forceinline__ T row_KU(const LevelTab<T>& L, const T* __restrict__ U, int g) {
  constexpr int Q = P - 1, TC = 2 * P + 1, NC = 2 * TC + 1;
  constexpr int WQ = 2 * Q + 1, WPP = 2 * P + 1;
  constexpr int B0 = WPP * WQ, B1 = 2 * P * WQ, RU = B0 + B1 + 1;
  const int nu = L.n_ux + L.n_uy;
  const bool is_x = g < L.n_ux, is_p = g >= nu, is_y = !is_x && !is_p;
  const int off = is_x ? 0 : (is_p ? nu : L.n_ux);
  const int rs = is_x ? L.nxu : L.npd;
  const int r = g - off;
  const int q_ = r / rs;
  const int iy = q_ + (is_y ? 1 : 0);
  const int ix = r - q_ * rs + (is_x ? 1 : 0);
  const int cx = cls1d<P>(ix, is_x ? L.lastp : L.lastq);
  const int cy = cls1d<P>(iy, is_y ? L.lastp : L.lastq);
  const T* st = L.srow ? L.srow + (size_t)g * RU : (is_x ? L.sx : (is_p ? L.sp : L.sy)) + (cx * NC + cy) * RU;
  // box 0: own velocity block (u rows) or u_x (p rows)
  const int b0_base = is_y ? L.n_ux : 0;
  const int b0_stride = is_y ? L.npd : L.nxu;
  const int b0_x0 = is_x ? -P : -Q, b0_y0 = is_y ? -P : -Q, b0_wy = is_y ? WPP : WQ;
  const int b0_xlo = is_y ? 0 : 1, b0_xhi = is_y ? L.lastq : L.nint, b0_xsh = is_y ? 0 : 1;
  const int b0_ylo = is_y ? 1 : 0, b0_yhi = is_y ? L.nint : L.lastq, b0_ysh = is_y ? 1 : 0;
  // box 1: pressure (u rows) or u_y (p rows)
  const int b1_base = is_p ? L.n_ux : nu;
  const int b1_x0 = is_x ? -P : -Q, b1_y0 = is_x ? -Q : (is_p ? -Q : -P), b1_wy = is_x ? WQ : 2 * P;
  const int b1_ylo = is_p ? 1 : 0, b1_yhi = is_p ? L.nint : L.lastq, b1_ysh = is_p ? 1 : 0;
  // with CH = 4, the even and odd terms of each box in separate chains: FP64 latency on this
  // GPU is long, so a row's critical path is its longest chain
  T acc = T(0), acc1 = T(0), acc2 = T(0), acc3 = T(0);
  constexpr bool kSplit = CH == 4;
  if (PART != 1) {
#pragma unroll
    for (int j = 0; j < B0; ++j) {
      int dx = j / b0_wy, dy = j - dx * b0_wy;
      int x = clampi(ix + b0_x0 + dx, b0_xlo, b0_xhi) - b0_xsh;
      int y = clampi(iy + b0_y0 + dy, b0_ylo, b0_yhi) - b0_ysh;
      if (kSplit && (j & 1)) acc1 = fma(st[j], U[b0_base + y * b0_stride + x], acc1);
      else acc = fma(st[j], U[b0_base + y * b0_stride + x], acc);
    }
  }
  if (PART != 0) {
#pragma unroll
    for (int j = 0; j < B1; ++j) {
      int dx = j / b1_wy, dy = j - dx * b1_wy;
      int x = clampi(ix + b1_x0 + dx, 0, L.lastq);
      int y = clampi(iy + b1_y0 + dy, b1_ylo, b1_yhi) - b1_ysh;
      if (kSplit && (j & 1)) acc3 = fma(st[B0 + j], U[b1_base + y * L.npd + x], acc3);
      else acc2 = fma(st[B0 + j], U[b1_base + y * L.npd + x], acc2);
    }
    if (kSplit) acc3 = fma(st[RU - 1], U[L.n_total - 1], acc3);
    else acc = fma(st[RU - 1], U[L.n_total - 1], acc);
    if (L.sext && !is_p) {
      // third box (mapped domains): u_x row -> u_y columns (x - P .. x + Q, y - Q .. y + P),
      // u_y row -> u_x columns (x - Q .. x + P, y - P .. y + Q); clamped positions carry 0
      constexpr int W2 = 2 * P;
      const T* se = L.sext + (size_t)g * (W2 * W2);
      const int ox = is_x ? -P : -Q, oy = is_x ? -Q : -P;
#pragma unroll
      for (int j = 0; j < W2 * W2; ++j) {
        int dx = j / W2, dy = j - dx * W2;
        int cx = ix + ox + dx, cy = iy + oy + dy;
        int idx = is_x ? L.n_ux + (clampi(cy, 1, L.nint) - 1) * L.npd + clampi(cx, 0, L.lastq)
                       : clampi(cy, 0, L.lastq) * L.nxu + clampi(cx, 1, L.nint) - 1;
        if (kSplit && (j & 1)) acc3 = fma(se[j], U[idx], acc3);
        else acc2 = fma(se[j], U[idx], acc2);
      }
    }
  }
  return kSplit ? (acc + acc1) + (acc2 + acc3) : acc + acc2;
}

// m_k for a pressure row (the last stencil entry).
template <int P, typename T>
__device__ __forceinline__ T mean_coef(const LevelTab<T>& L, int r) {
  constexpr int Q = P - 1, TC = 2 * P + 1, NC = 2 * TC + 1;
  constexpr int RU = (2 * P + 1) * (2 * Q + 1) + 2 * P * (2 * Q + 1) + 1;
  if (L.srow) return L.srow[(size_t)(L.n_ux + L.n_uy + r) * RU + RU - 1];
  int ky = r / L.npd, kx = r - ky * L.npd;
  return L.sp[(cls1d<P>(kx, L.lastq) * NC + cls1d<P>(ky, L.lastq)) * RU + RU - 1];
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

// Per-block sums of a thread's R^2 and m.p terms into part[2 * block], part[2 * block + 1].
// FP64 values: two FP64 block reductions.  FP32 values: summed in FP32 within each warp (at
// most 32 terms) and in FP64 across warps -- every FP64 instruction costs a warp 32 cycles of
// the SM's FP64 pipe on GB300, and one FP64 reduction per row made the FP32 kernels FP64-bound.
template <typename T>
__device__ __forceinline__ void block_partials(T r2, T mp, double* sh, double* __restrict__ part) {
  if constexpr (sizeof(T) == 8) {
    const double s1 = block_sum((double)r2, sh);
    const double s2 = block_sum((double)mp, sh);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1; part[2 * blockIdx.x + 1] = s2; }
  } else {
    for (int o = 16; o > 0; o >>= 1) {
      r2 += __shfl_xor_sync(0xffffffffu, r2, o);
      mp += __shfl_xor_sync(0xffffffffu, mp, o);
    }
    const int w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { sh[w] = (double)r2; sh[32 + w] = (double)mp; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s1 = 0.0, s2 = 0.0;
      for (int i = 0; i < nw; ++i) { s1 += sh[i]; s2 += sh[32 + i]; }
      part[2 * blockIdx.x] = s1;
      part[2 * blockIdx.x + 1] = s2;
    }
  }
}

// R = F - K U for every row but lambda; per-block partial sums of R^2 and of m.p.
template <int P, typename T>
__global__ void __launch_bounds__(256) k_residual(LevelTab<T> L, const T* __restrict__ U, const T* __restrict__ F,
                                                  T* __restrict__ R, double* __restrict__ part) {
  __shared__ double sh[64];
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  T r2 = T(0), mp = T(0);
  if (g < L.n_total - 1) {
    T r = F[g] - row_KU<P>(L, U, g);
    R[g] = r;
    r2 = r * r;
    int off = g - L.n_ux - L.n_uy;
    if (off >= 0) mp = mean_coef<P>(L, off) * U[g];
  }
  block_partials<T>(r2, mp, sh, part);
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

// ---- building blocks shared by the per-level kernels and the fused coarse-level kernel --

// One lane of an 8-DOF patch (four patches per warp, lane = (patch, local row)): the local
// residual row, then the bordered local inverse through shuffles, then the update.  All
// 32 lanes of the warp must call it together (the shuffles span the warp).
template <int P, typename T, int CH = 4>
__device__ __forceinline__ void fast_patch_lane(const LevelTab<T>& L, T* U, const T* F, const int* __restrict__ dofs,
                                                const int* __restrict__ cls, const T* __restrict__ cinv8, int maxl,
                                                int first, int n8, int grp, int lane) {
  int row = lane & 7;
  bool active = grp < n8;
  int patch = first + (active ? grp : 0);
  int g = dofs[patch * maxl + row];
  T r = F[g] - row_KU<P, T, 2, CH>(L, U, g);
  const T* A = cinv8 + (size_t)cls[patch] * 64 + row * 8;
  T d[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int s = 0; s < 8; ++s) d[s & (CH - 1)] = fma(A[s], __shfl_sync(0xffffffffu, r, (lane & ~7) + s), d[s & (CH - 1)]);
  if (active) U[g] += CH == 4 ? (d[0] + d[1]) + (d[2] + d[3]) : d[0] + d[1];
}

// Half of row g of K U for the two-lanes-per-row patch form: half 0 sums box 0, half 1 box 1
// and the lambda term.  Both halves run the same instruction stream (no divergence between
// the two lanes of a row): a loop of B0 terms over their own box, half 1's past its B1 + 1
// terms padded with zero coefficients at a valid (clamped) index.  Not for mapped domains
// (their third box is not split).
template <int P, typename T>
__device__ __forceinline__ T row_half(const LevelTab<T>& L, const T* __restrict__ U, int g, int half) {
  constexpr int Q = P - 1, TC = 2 * P + 1, NC = 2 * TC + 1;
  constexpr int WQ = 2 * Q + 1, WPP = 2 * P + 1;
  constexpr int B0 = WPP * WQ, B1 = 2 * P * WQ, RU = B0 + B1 + 1;
  static_assert(B0 >= B1 + 1, "box 0 must cover box 1 and the lambda term");
  const int nu = L.n_ux + L.n_uy;
  const bool is_x = g < L.n_ux, is_p = g >= nu, is_y = !is_x && !is_p;
  const int off = is_x ? 0 : (is_p ? nu : L.n_ux);
  const int rs = is_x ? L.nxu : L.npd;
  const int r = g - off;
  const int q_ = r / rs;
  const int iy = q_ + (is_y ? 1 : 0);
  const int ix = r - q_ * rs + (is_x ? 1 : 0);
  const int cx = cls1d<P>(ix, is_x ? L.lastp : L.lastq);
  const int cy = cls1d<P>(iy, is_y ? L.lastp : L.lastq);
  const T* st = L.srow ? L.srow + (size_t)g * RU : (is_x ? L.sx : (is_p ? L.sp : L.sy)) + (cx * NC + cy) * RU;
  // box 0: own velocity block (u rows) or u_x (p rows); box 1: pressure (u rows) or u_y (p rows)
  const int base = half ? (is_p ? L.n_ux : nu) : (is_y ? L.n_ux : 0);
  const int stride = half ? L.npd : (is_y ? L.npd : L.nxu);
  const int x0 = (is_x ? -P : -Q);
  const int y0 = half ? (is_x ? -Q : (is_p ? -Q : -P)) : (is_y ? -P : -Q);
  const int wy = half ? (is_x ? WQ : 2 * P) : (is_y ? WPP : WQ);
  const int xlo = half ? 0 : (is_y ? 0 : 1), xhi = half ? L.lastq : (is_y ? L.lastq : L.nint);
  const int xsh = half ? 0 : (is_y ? 0 : 1);
  const int ylo = half ? (is_p ? 1 : 0) : (is_y ? 1 : 0), yhi = half ? (is_p ? L.nint : L.lastq) : (is_y ? L.nint : L.lastq);
  const int ysh = half ? (is_p ? 1 : 0) : (is_y ? 1 : 0);
  const int cnt = half ? B1 : B0, coff = half ? B0 : 0;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  int dx = 0, dy = 0;
#pragma unroll
  for (int j = 0; j < B0; ++j) {
    const int x = clampi(ix + x0 + dx, xlo, xhi) - xsh;
    const int y = clampi(iy + y0 + dy, ylo, yhi) - ysh;
    const bool lam = half && j == B1;
    const T c = j < cnt ? st[coff + j] : (lam ? st[RU - 1] : T(0));
    const int idx = lam ? L.n_total - 1 : base + y * stride + x;
    acc[j & 3] = fma(c, U[idx], acc[j & 3]);
    if (j + 1 < cnt) { ++dy; if (dy == wy) { dy = 0; ++dx; } }   // stays on the last entry past cnt
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// One lane of an 8-DOF patch in the two-lanes-per-row form: two patches per warp, lane =
// (patch, local row, half).  The row's two halves meet by one shuffle; each half then
// applies four of the eight columns of the bordered local inverse and the halves meet
// again.  Compared with fast_patch_lane: half the dependent multiply-adds per lane and
// twice the warps per colour, for about 16 % more FP64 instructions per patch.
template <int P, typename T>
__device__ __forceinline__ void fast_patch_lane2(const LevelTab<T>& L, T* U, const T* F, const int* __restrict__ dofs,
                                                 const int* __restrict__ cls, const T* __restrict__ cinv8, int maxl,
                                                 int first, int n8, int grp, int lane) {
  const int half = lane & 1, row = (lane >> 1) & 7, lane0 = lane & 16;
  const bool active = grp < n8;
  const int patch = first + (active ? grp : 0);
  const int g = dofs[patch * maxl + row];
  const T fv = F[g];
  const T v = (half ? T(0) : fv) - row_half<P>(L, U, g, half);
  const T r = v + __shfl_xor_sync(0xffffffffu, v, 1);
  const T* A = cinv8 + (size_t)cls[patch] * 64 + row * 8 + half * 4;
  T d0 = T(0), d1 = T(0);
#pragma unroll
  for (int k = 0; k < 4; k += 2) {
    d0 = fma(A[k], __shfl_sync(0xffffffffu, r, lane0 + (half * 4 + k) * 2), d0);
    d1 = fma(A[k + 1], __shfl_sync(0xffffffffu, r, lane0 + (half * 4 + k + 1) * 2), d1);
  }
  T d = d0 + d1;
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  if (active && half == 0) U[g] += d;
}

// A larger (wall) patch solved by one warp; r is warp-private scratch of maxl entries.
template <int P, typename T, int CH = 4>
__device__ __forceinline__ void general_patch_warp(const LevelTab<T>& L, T* U, const T* F, const int* __restrict__ dofs,
                                                   const int* __restrict__ cls, const T* __restrict__ cinv,
                                                   const int* __restrict__ nloc, int maxl, int patch, int lane, T* r) {
  int c = cls[patch], nl = nloc[c];
  const int* pd = dofs + (size_t)patch * maxl;
  for (int k = lane; k < nl; k += 32) { int g = pd[k]; r[k] = F[g] - row_KU<P, T, 2, CH>(L, U, g); }
  __syncwarp();
  const T* A = cinv + (size_t)c * maxl * maxl;
  for (int k = lane; k < nl; k += 32) U[pd[k]] += dot_n(A + (size_t)k * maxl, r, nl);
  __syncwarp();
}

// g_c = P^T r_f at coarse entry g (not lambda).
template <typename T>
__device__ __forceinline__ T restrict_elem(const LevelTab<T>& Lf, const LevelTab<T>& Lc, const Xfer<T>& tp,
                                           const Xfer<T>& tq, const T* rf, int g) {
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
    int fy = min(fy0 + ky, nfy - 1);            // weights past the end are zero
    T wy = ry[cy * kWR + ky];
    T s = T(0);
#pragma unroll
    for (int kx = 0; kx < kWR; ++kx) {
      int fx = min(fx0 + kx, nfx - 1);
      s = fma(rx[cx * kWR + kx], src[fy * fnx + fx], s);
    }
    acc = fma(wy, s, acc);
  }
  return acc;
}

// (P u_c) at fine entry g (not lambda).
template <typename T>
__device__ __forceinline__ T prolong_elem(const LevelTab<T>& Lf, const LevelTab<T>& Lc, const Xfer<T>& tp,
                                          const Xfer<T>& tq, const T* uc, int g) {
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
    int cy = min(cy0 + ky, ncy - 1);            // weights past the end are zero
    T s = T(0);
#pragma unroll
    for (int kx = 0; kx < kWP; ++kx) {
      int cx = min(cx0 + kx, ncx - 1);
      s = fma(px[fx * kWP + kx], src[cy * cnx + cx], s);
    }
    acc = fma(py[fy * kWP + ky], s, acc);
  }
  return acc;
}

// One colour of the multiplicative Schwarz sweep (eq. MSM).  Blocks [0, nb8): four 8-DOF
// patches per warp.  Blocks [nb8, ...): one warp per larger (wall) patch.  Any block size
// that is a multiple of 32 (the launch picks 128 threads so that a colour's blocks spread
// evenly over the SMs).  Same-colour
// patches share no DOF and are not coupled by K, so they may be solved in any order.
template <int P, typename T, int LPR = 1, int CH = 4>
__device__ __forceinline__ void mult_colour_block(const LevelTab<T>& L, T* __restrict__ U, const T* __restrict__ F,
                                                  const int* __restrict__ dofs, const int* __restrict__ cls,
                                                  const T* __restrict__ cinv, const T* __restrict__ cinv8,
                                                  const int* __restrict__ nloc, int maxl, int first, int n8,
                                                  int ngen, int nb8, int blk) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  if (blk < nb8) {
    if (LPR == 2)
      fast_patch_lane2<P>(L, U, F, dofs, cls, cinv8, maxl, first, n8, (blk * wpb + wib) * 2 + (lane >> 4), lane);
    else
      fast_patch_lane<P, T, CH>(L, U, F, dofs, cls, cinv8, maxl, first, n8, (blk * wpb + wib) * 4 + (lane >> 3), lane);
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  int w = (blk - nb8) * wpb + wib;
  if (w >= ngen) return;
  general_patch_warp<P, T, CH>(L, U, F, dofs, cls, cinv, nloc, maxl, first + n8 + w, lane, sh + wib * maxl);
}

// CH: multiply-add chains per row and per local inverse (4: shorter dependent chains; 2: four
// fewer FP64 adds per lane, for launches that keep the FP64 pipe busy).
template <int P, typename T, int LPR = 1, int CH = 4>
__global__ void __launch_bounds__(256) k_mult_colour(LevelTab<T> L, T* __restrict__ U, const T* __restrict__ F,
                                                     const int* __restrict__ dofs, const int* __restrict__ cls,
                                                     const T* __restrict__ cinv, const T* __restrict__ cinv8,
                                                     const int* __restrict__ nloc,
                                                     int maxl, int first, int n8, int ngen, int nb8) {
  mult_colour_block<P, T, LPR, CH>(L, U, F, dofs, cls, cinv, cinv8, nloc, maxl, first, n8, ngen, nb8, (int)blockIdx.x);
}

// The same colour step with each 8-DOF patch row split over two warps: warps 0-7 of the
// block sum box 0 of their rows (minus F), warps 8-15 box 1 and the lambda term of the same
// rows; the halves meet in shared memory, then warps 0-7 apply the local inverses.  Each
// warp issues about half the FP64 instructions of k_mult_colour's, which shortens the
// critical path on GB300 (one FP64 instruction per warp every 64 cycles).  Blocks [nb8, ...)
// hold the larger (wall) patches, one warp each.
template <int P, typename T>
__global__ void __launch_bounds__(512) k_mult_colour_split(LevelTab<T> L, T* __restrict__ U, const T* __restrict__ F,
                                                           const int* __restrict__ dofs, const int* __restrict__ cls,
                                                           const T* __restrict__ cinv, const T* __restrict__ cinv8,
                                                           const int* __restrict__ nloc,
                                                           int maxl, int first, int n8, int ngen, int nb8) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if ((int)blockIdx.x < nb8) {
    __shared__ T part[2][256];
    const int half = wib >> 3, w8 = wib & 7;
    const int slot = w8 * 32 + lane;                    // (patch in block, row)
    const int grp = (blockIdx.x * 8 + w8) * 4 + (lane >> 3), row = lane & 7;
    const bool active = grp < n8;
    const int patch = first + (active ? grp : 0);
    const int g = dofs[(size_t)patch * maxl + row];
    T v = half == 0 ? F[g] - row_KU<P, T, 0>(L, U, g) : -row_KU<P, T, 1>(L, U, g);
    part[half][slot] = v;
    __syncthreads();
    if (half) return;
    const T r = v + part[1][slot];
    part[0][slot] = r;
    __syncwarp();
    const T* A = cinv8 + (size_t)cls[patch] * 64 + row * 8;
    const T* rp = &part[0][slot - row];
    T d0 = T(0), d1 = T(0);
#pragma unroll
    for (int s = 0; s < 8; s += 2) {
      d0 = fma(A[s], rp[s], d0);
      d1 = fma(A[s + 1], rp[s + 1], d1);
    }
    if (active) U[g] += d0 + d1;
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  int w = ((int)blockIdx.x - nb8) * 16 + wib;
  if (w >= ngen) return;
  general_patch_warp<P>(L, U, F, dofs, cls, cinv, nloc, maxl, first + n8 + w, lane, sh + wib * maxl);
}

// ---- pipelined multiplicative sweep: all colours of nu sweeps in one persistent launch ----
//
// The patches are cut into square tiles of patch positions (tw x tw, tw >= p); one block
// owns one tile and runs its patches colour by colour.  A patch at position (a, b) reads
// and writes only DOFs whose supports lie in, or overlap, the elements [a-p, a] x [b-p, b],
// so it depends on patches within p positions, i.e. on the eight neighbouring tiles.  Each
// tile publishes how many colour steps it has finished (prog, monotone across launches);
// a tile starts step k once every neighbour has finished step k-1.  Neighbours are then
// never more than one step apart, which gives every patch exactly the values it would see
// in the sequential colour-major sweep (eq. MSM): the earlier colours' updates near it are
// done (read after write) and no later colour near it has started (write after read).
// The launch is cooperative (all blocks resident), and every wait is bounded: a block that
// gives up sets *err and returns, the others notice *err and return too, and the host
// resets prog and err before it reports the timeout.
struct TileSched {
  int ntx, nty, n_colours;
  const int* list;      // patch indices (colour-major tables) by (tile, colour), 8-DOF first
  const int* off;       // ntx * nty * n_colours + 1 offsets into list
  const int* n8;        // per (tile, colour): 8-DOF patches at the front of its run
  unsigned* prog;       // per tile: colour steps finished
  int* err;             // 1 once a wait has given up
  int stall;            // failure-path test only: this tile never publishes (-1: none)
};

constexpr long kSpinLimit = 1L << 21;   // polls (about 0.5-1 us each) before giving up

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// With a relaxed load before it (acquire pattern) or a relaxed store after it (release
// pattern), this fence orders the block's U updates against the step counters.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(const volatile int*)p; }

// What one lane needs of its first 8-DOF patch of a colour step, loaded before the wait for
// the neighbouring tiles (none of it depends on U): the row, its forcing entry and the
// patch's inverse row.
template <typename T>
struct LanePatch {
  int g;
  T f;
  const T* A;
  bool active, any;
};

template <typename T>
__device__ __forceinline__ LanePatch<T> lane_patch_load(const TileSched& ts, const T* __restrict__ F,
                                                        const int* __restrict__ dofs, const int* __restrict__ cls,
                                                        const T* __restrict__ cinv8, int maxl, int run, int grp,
                                                        int lane) {
  LanePatch<T> lp;
  const int o0 = ts.off[run], n8 = ts.n8[run];
  lp.any = n8 > 0;
  lp.active = grp < n8;
  lp.g = 0; lp.f = T(0); lp.A = cinv8;
  if (lp.any) {
    const int patch = ts.list[o0 + (lp.active ? grp : 0)];
    lp.g = dofs[patch * maxl + (lane & 7)];
    lp.f = F[lp.g];
    lp.A = cinv8 + (size_t)cls[patch] * 64 + (lane & 7) * 8;
  }
  return lp;
}

// The rest of list_patch_lane for a prefetched lane: residual row, local inverse, update.
template <int P, typename T>
__device__ __forceinline__ void lane_patch_solve(const LevelTab<T>& L, T* U, const LanePatch<T>& lp, int lane) {
  T r = lp.f - row_KU<P>(L, U, lp.g);
  T d[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int s = 0; s < 8; ++s) d[s & 3] = fma(lp.A[s], __shfl_sync(0xffffffffu, r, (lane & ~7) + s), d[s & 3]);
  if (lp.active) U[lp.g] += (d[0] + d[1]) + (d[2] + d[3]);
}

// fast_patch_lane for a patch taken from an index list (four patches per warp).
template <int P, typename T>
__device__ __forceinline__ void list_patch_lane(const LevelTab<T>& L, T* U, const T* F, const int* __restrict__ dofs,
                                                const int* __restrict__ cls, const T* __restrict__ cinv8, int maxl,
                                                const int* __restrict__ list, int n8, int grp, int lane) {
  int row = lane & 7;
  bool active = grp < n8;
  int patch = list[active ? grp : (grp & ~3)];
  int g = dofs[patch * maxl + row];
  T r = F[g] - row_KU<P>(L, U, g);
  const T* A = cinv8 + (size_t)cls[patch] * 64 + row * 8;
  T d[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int s = 0; s < 8; ++s) d[s & 3] = fma(A[s], __shfl_sync(0xffffffffu, r, (lane & ~7) + s), d[s & 3]);
  if (active) U[g] += (d[0] + d[1]) + (d[2] + d[3]);
}

// NT: threads per block (128 for tiled levels, 6 blocks per SM; 512 for a level that is
// one tile).  With one tile there is nobody to wait for: the steps are separated by the
// block barrier alone, without counters or fences.
template <int P, typename T, int NT>
__global__ void __launch_bounds__(NT, NT <= 128 ? 6 : 1) k_sweep_tiles(LevelTab<T> L, T* __restrict__ U, const T* __restrict__ F,
                                                     const int* __restrict__ dofs, const int* __restrict__ cls,
                                                     const T* __restrict__ cinv, const T* __restrict__ cinv8,
                                                     const int* __restrict__ nloc, int maxl, TileSched ts, int steps) {
  extern __shared__ unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  __shared__ int s_go;
  const int t = blockIdx.x, tx = t % ts.ntx, ty = t / ts.ntx;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const bool solo = gridDim.x == 1;
  if (threadIdx.x == 0) s_go = ld_volatile_i32(ts.err) == 0;
  __syncthreads();
  if (!s_go) return;
  const unsigned base = ts.prog[t];     // every tile ended the previous launch at the same count
  // the neighbour that lane j < 8 of warp 0 watches
  const unsigned* watch = nullptr;
  if (wib == 0 && lane < 8) {
    const int j = lane < 4 ? lane : lane + 1;     // 3 x 3 stencil without its centre
    const int x = tx + j % 3 - 1, y = ty + j / 3 - 1;
    if (x >= 0 && y >= 0 && x < ts.ntx && y < ts.nty) watch = ts.prog + y * ts.ntx + x;
  }
  const int grp0 = wib * 4 + (lane >> 3);
  LanePatch<T> lp = lane_patch_load(ts, F, dofs, cls, cinv8, maxl, t * ts.n_colours, grp0, lane);
  for (int k = 0; k < steps; ++k) {
    if (k > 0 && solo) __syncthreads();
    if (k > 0 && !solo) {
      if (wib == 0) {
        const unsigned need = base + (unsigned)k;
        bool ok = false;
        for (long it = 0; it < kSpinLimit; ++it) {
          const bool mine = watch == nullptr || (int)(ld_relaxed_u32(watch) - need) >= 0;
          ok = __all_sync(0xffffffffu, mine);
          if (ok) break;
          int stop = lane == 0 ? ld_volatile_i32(ts.err) : 0;
          if (__shfl_sync(0xffffffffu, stop, 0)) break;
          __nanosleep(20);
        }
        fence_acq_rel_gpu();
        if (lane == 0) {
          if (!ok) atomicExch(ts.err, 1);
          s_go = ok;
        }
      }
      __syncthreads();
      if (!s_go) return;
    }
    const int run = t * ts.n_colours + k % ts.n_colours;
    const int o0 = ts.off[run], n8 = ts.n8[run], ngen = ts.off[run + 1] - o0 - n8;
    if (lp.any && wib * 4 < n8) lane_patch_solve<P>(L, U, lp, lane);
    for (int g0 = wib * 4 + wpb * 4; g0 < n8; g0 += wpb * 4)
      list_patch_lane<P>(L, U, F, dofs, cls, cinv8, maxl, ts.list + o0, n8, g0 + (lane >> 3), lane);
    for (int w = wib; w < ngen; w += wpb)
      general_patch_warp<P>(L, U, F, dofs, cls, cinv, nloc, maxl, ts.list[o0 + n8 + w], lane, sh + wib * maxl);
    if (!solo) {
      __syncthreads();
      if (threadIdx.x == 0 && t != ts.stall) {
        fence_acq_rel_gpu();
        st_relaxed_u32(ts.prog + t, base + (unsigned)k + 1u);
      }
    }
    if (k + 1 < steps)                  // the next step's rows, while the neighbours finish
      lp = lane_patch_load(ts, F, dofs, cls, cinv8, maxl, t * ts.n_colours + (k + 1) % ts.n_colours, grp0, lane);
  }
}

// Additive sweep (eq. ASM), part 1: local corrections from one common residual, kept per patch.
template <int P, typename T>
__global__ void __launch_bounds__(256) k_add_local(const T* __restrict__ R, const int* __restrict__ dofs,
                                                   const int* __restrict__ cls, const T* __restrict__ cinv,
                                                   const T* __restrict__ cinv8, const int* __restrict__ nloc,
                                                   int maxl, int count, T* __restrict__ delta) {
  extern __shared__ unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= count) return;
  const int* pd = dofs + (size_t)warp * maxl;
  // 8-DOF patches use the packed 8 x 8 table (their ninth DOF slot is padding)
  bool is8 = maxl == 8 || pd[8] < 0;
  int c = cls[warp], nl = is8 ? 8 : nloc[c];
  const T* A = is8 ? cinv8 + (size_t)c * 64 : cinv + (size_t)c * maxl * maxl;
  int ld = is8 ? 8 : maxl;
  T* r = sh + (threadIdx.x >> 5) * maxl;
  for (int k = lane; k < nl; k += 32) r[k] = R[pd[k]];
  __syncwarp();
  for (int k = lane; k < nl; k += 32)
    delta[(size_t)warp * maxl + k] = dot_n(A + (size_t)k * ld, r, nl);
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

// g_c = P^T r_f (lambda copied); one thread per coarse entry.
template <typename T>
__global__ void k_restrict(LevelTab<T> Lf, LevelTab<T> Lc, Xfer<T> tp, Xfer<T> tq, const T* __restrict__ rf,
                           T* __restrict__ gc) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lc.n_total) return;
  gc[g] = (g == Lc.n_total - 1) ? rf[Lf.n_total - 1] : restrict_elem(Lf, Lc, tp, tq, rf, g);
}

// u_f += P u_c (lambda added); one thread per fine entry.
template <typename T>
__global__ void k_prolong_add(LevelTab<T> Lf, LevelTab<T> Lc, Xfer<T> tp, Xfer<T> tq, const T* __restrict__ uc,
                              T* __restrict__ uf) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lf.n_total) return;
  uf[g] += (g == Lf.n_total - 1) ? uc[Lc.n_total - 1] : prolong_elem(Lf, Lc, tp, tq, uc, g);
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
#pragma unroll 4
    for (int j = lane; j < n; j += 32) acc = fma(row[j], g[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) U[i] = acc;
  }
}

// ---- the coarse end of the V-cycle in one thread block ------------------------------------
constexpr int kMaxFused = 8;        // levels handled by one fused launch
constexpr int kMaxColours = 16;     // (p+1)^2 for p <= 3

template <typename T>
struct FusedLevel {
  LevelTab<T> L;
  Xfer<T> tp, tq;                   // transfer from the level below into this one (l >= 1)
  const T *cinv, *cinv8;
  const int *dofs, *cls, *nloc;
  int maxl, n_colours;
  int colour_off[kMaxColours + 1], n8[kMaxColours];
  int offU, offF, offR;             // offsets of this level's vectors in shared memory
};

template <typename T>
struct FusedDesc {
  int nlev;                         // levels 0 .. nlev-1 of the hierarchy
  int nu1, nu2, ndof0, scratch_off; // scratch: one maxl-vector per warp for wall patches
  const T* coarse_inv;
  FusedLevel<T> lev[kMaxFused];
};

// MGV(l_c, U, F) of Algorithm 1 for the coarsest levels 0 .. l_c = nlev-1, entirely inside
// one block: every level vector lives in shared memory and the phases (colours, residual,
// transfers, coarse solve) are separated by __syncthreads instead of kernel launches.
// F_{l_c} is read from Fin; U_{l_c} starts from Uio (load_u) or zero and is written back.
template <int P, typename T>
__global__ void __launch_bounds__(1024) k_fused_coarse(FusedDesc<T> D, const T* __restrict__ Fin, T* __restrict__ Uio,
                                                       int load_u) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  const int lc = D.nlev - 1;
  {
    const FusedLevel<T>& V = D.lev[lc];
    T* U = sm + V.offU; T* F = sm + V.offF;
    for (int i = tid; i < V.L.n_total; i += nt) { F[i] = Fin[i]; U[i] = load_u ? Uio[i] : T(0); }
  }
  __syncthreads();
  auto smooth = [&](int l) {
    const FusedLevel<T>& V = D.lev[l];
    T* U = sm + V.offU; const T* F = sm + V.offF;
    T* scratch = sm + D.scratch_off + warp * V.maxl;
    for (int c = 0; c < V.n_colours; ++c) {
      int first = V.colour_off[c], n8 = V.n8[c], ngen = V.colour_off[c + 1] - first - n8;
      int lanes = ((n8 * 8 + 31) / 32) * 32;
      for (int t = tid; t < lanes; t += nt) fast_patch_lane<P>(V.L, U, F, V.dofs, V.cls, V.cinv8, V.maxl, first, n8, t >> 3, lane);
      for (int w = warp; w < ngen; w += nwarp)
        general_patch_warp<P>(V.L, U, F, V.dofs, V.cls, V.cinv, V.nloc, V.maxl, first + n8 + w, lane, scratch);
      __syncthreads();
    }
  };
  auto residual = [&](int l) {
    const FusedLevel<T>& V = D.lev[l];
    const T* U = sm + V.offU; const T* F = sm + V.offF; T* R = sm + V.offR;
    const int nu = V.L.n_ux + V.L.n_uy;
    double mp = 0.0;
    for (int g = tid; g < V.L.n_total - 1; g += nt) {
      R[g] = F[g] - row_KU<P>(V.L, U, g);
      if (g >= nu) mp += (double)mean_coef<P>(V.L, g - nu) * (double)U[g];
    }
    double s = block_sum(mp, red);
    if (tid == 0) R[V.L.n_total - 1] = (T)((double)F[V.L.n_total - 1] - s);
    __syncthreads();
  };
  for (int l = lc; l >= 1; --l) {
    for (int k = 0; k < D.nu1; ++k) smooth(l);
    residual(l);
    const FusedLevel<T>& V = D.lev[l];
    const FusedLevel<T>& C = D.lev[l - 1];
    const T* R = sm + V.offR;
    T* Fc = sm + C.offF; T* Uc = sm + C.offU;
    for (int g = tid; g < C.L.n_total; g += nt) {
      Fc[g] = (g == C.L.n_total - 1) ? R[V.L.n_total - 1] : restrict_elem(V.L, C.L, V.tp, V.tq, R, g);
      Uc[g] = T(0);
    }
    __syncthreads();
  }
  {  // exact coarsest solve, one warp per row of K_0^{-1}
    const FusedLevel<T>& C = D.lev[0];
    const T* G = sm + C.offF; T* U0 = sm + C.offU;
    for (int i = warp; i < D.ndof0; i += nwarp) {
      const T* row = D.coarse_inv + (size_t)i * D.ndof0;
      T acc = T(0);
#pragma unroll 4
      for (int j = lane; j < D.ndof0; j += 32) acc = fma(row[j], G[j], acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) U0[i] = acc;
    }
    __syncthreads();
  }
  for (int l = 1; l <= lc; ++l) {
    const FusedLevel<T>& V = D.lev[l];
    const FusedLevel<T>& C = D.lev[l - 1];
    T* U = sm + V.offU; const T* Uc = sm + C.offU;
    for (int g = tid; g < V.L.n_total; g += nt)
      U[g] += (g == V.L.n_total - 1) ? Uc[C.L.n_total - 1] : prolong_elem(V.L, C.L, V.tp, V.tq, Uc, g);
    __syncthreads();
    for (int k = 0; k < D.nu2; ++k) smooth(l);
  }
  {
    const FusedLevel<T>& V = D.lev[lc];
    const T* U = sm + V.offU;
    for (int i = tid; i < V.L.n_total; i += nt) Uio[i] = U[i];
  }
}

// ---- the coarse end of the V-cycle in one thread-block cluster ---------------------------
// The same phases as k_fused_coarse, but spread over the C blocks of one cluster (C SMs of
// FP64 throughput instead of one) with the level vectors in global memory (they stay in
// L2): a phase's work is split over all warps of the cluster and phases are separated by
// the cluster barrier (hardware barrier with release / acquire semantics at cluster scope),
// not by kernel launches.
template <typename T>
struct ClusterLevel {
  LevelTab<T> L;
  Xfer<T> tp, tq;                   // transfer from the level below into this one (l >= 1)
  const T *cinv, *cinv8;
  const int *dofs, *cls, *nloc;
  int maxl, n_colours;
  int colour_off[kMaxColours + 1], n8[kMaxColours];
  T *U, *F, *R;
};

template <typename T>
struct ClusterDesc {
  int nlev, nu1, nu2, ndof0, maxl;
  const T* coarse_inv;
  double* part;                     // one partial sum per block (lambda row of the residual)
  ClusterLevel<T> lev[kMaxFused];
};

template <int P, typename T>
__global__ void __launch_bounds__(1024) k_cluster_coarse(ClusterDesc<T> D, const T* __restrict__ Ftop, T* __restrict__ Utop,
                                                         int load_u) {
  extern __shared__ unsigned char smem_raw[];
  T* scratch_all = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  const unsigned rank = blockIdx.x, C = gridDim.x;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  const int gtid = rank * nt + tid, gnt = C * nt, gwarp = rank * nwarp + warp, gnwarp = C * nwarp;
  const int lc = D.nlev - 1;
  T* scratch = scratch_all + warp * D.maxl;
  auto csync = []() { asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory"); };
  auto Uof = [&](int l) { return l == lc ? Utop : D.lev[l].U; };
  auto Fof = [&](int l) { return l == lc ? Ftop : (const T*)D.lev[l].F; };
  if (!load_u) {
    for (int i = gtid; i < D.lev[lc].L.n_total; i += gnt) Utop[i] = T(0);
    csync();
  }
  auto smooth = [&](int l) {
    const ClusterLevel<T>& V = D.lev[l];
    T* U = Uof(l); const T* F = Fof(l);
    for (int c = 0; c < V.n_colours; ++c) {
      int first = V.colour_off[c], n8 = V.n8[c], ngen = V.colour_off[c + 1] - first - n8;
      int lanes = ((n8 * 8 + 31) / 32) * 32;
      for (int t = gtid - lane; t < lanes; t += gnt)           // whole warps (shuffles span the warp)
        fast_patch_lane<P>(V.L, U, F, V.dofs, V.cls, V.cinv8, V.maxl, first, n8, (t + lane) >> 3, lane);
      for (int w = gwarp; w < ngen; w += gnwarp)
        general_patch_warp<P>(V.L, U, F, V.dofs, V.cls, V.cinv, V.nloc, V.maxl, first + n8 + w, lane, scratch);
      csync();
    }
  };
  for (int l = lc; l >= 1; --l) {
    for (int k = 0; k < D.nu1; ++k) smooth(l);
    const ClusterLevel<T>& V = D.lev[l];
    const ClusterLevel<T>& Cl = D.lev[l - 1];
    {  // residual (all rows but lambda) and this block's share of m . p
      const T* U = Uof(l); const T* F = Fof(l); T* R = V.R;
      const int nu = V.L.n_ux + V.L.n_uy;
      double mp = 0.0;
      for (int g = gtid; g < V.L.n_total - 1; g += gnt) {
        R[g] = F[g] - row_KU<P>(V.L, U, g);
        if (g >= nu) mp += (double)mean_coef<P>(V.L, g - nu) * (double)U[g];
      }
      double sblk = block_sum(mp, red);
      if (tid == 0) D.part[rank] = sblk;
      csync();
      if (gtid == 0) {
        double sm = 0.0;
        for (unsigned b = 0; b < C; ++b) sm += D.part[b];
        R[V.L.n_total - 1] = (T)((double)F[V.L.n_total - 1] - sm);
      }
      csync();
    }
    {  // restriction into level l-1, and U_{l-1} = 0
      const T* R = V.R;
      T* Fc = Cl.F; T* Uc = Cl.U;
      for (int g = gtid; g < Cl.L.n_total; g += gnt) {
        Fc[g] = (g == Cl.L.n_total - 1) ? R[V.L.n_total - 1] : restrict_elem(V.L, Cl.L, V.tp, V.tq, R, g);
        Uc[g] = T(0);
      }
      csync();
    }
  }
  {  // exact coarsest solve, one warp per row of K_0^{-1}
    const T* G = D.lev[0].F; T* U0 = D.lev[0].U;
    for (int i = gwarp; i < D.ndof0; i += gnwarp) {
      const T* row = D.coarse_inv + (size_t)i * D.ndof0;
      T acc = T(0);
#pragma unroll 4
      for (int j = lane; j < D.ndof0; j += 32) acc = fma(row[j], G[j], acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) U0[i] = acc;
    }
    csync();
  }
  for (int l = 1; l <= lc; ++l) {
    const ClusterLevel<T>& V = D.lev[l];
    const ClusterLevel<T>& Cl = D.lev[l - 1];
    T* U = Uof(l); const T* Uc = Cl.U;
    for (int g = gtid; g < V.L.n_total; g += gnt)
      U[g] += (g == V.L.n_total - 1) ? Uc[Cl.L.n_total - 1] : prolong_elem(V.L, Cl.L, V.tp, V.tq, Uc, g);
    csync();
    for (int k = 0; k < D.nu2; ++k) smooth(l);
  }
}

// ---- mixed precision helpers ---------------------------------------------------------
static __global__ void k_to_float(int n, const double* __restrict__ a, float* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// Discrete streamfunction of a velocity correction by integration along y of its u_x
// block: psi(ix, k+1) = psi(ix, k) + e_x(ix, k) / dcoef_k, psi = 0 on the bottom wall.
// One warp per interior column: each lane sums a contiguous run, then a warp scan.
// psi is stored on the (n+p-2)^2 interior, FP64.
static __global__ void k_integrate_psi(int nint, int nxu, const double* __restrict__ inv_dcoef,
                                const float* __restrict__ e, double* __restrict__ psi) {
  int ix = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // interior column
  int lane = threadIdx.x & 31;
  if (ix >= nint) return;
  int per = (nint + 31) / 32;
  int k0 = lane * per, k1 = min(k0 + per, nint);
  double run = 0.0;
  for (int k = k0; k < k1; ++k) run = fma((double)e[k * nxu + ix], inv_dcoef[k], run);
  double incl = run;                      // inclusive scan of the lane totals
  for (int o = 1; o < 32; o <<= 1) {
    double v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  double acc = incl - run;                // exclusive prefix
  for (int k = k0; k < k1; ++k) {
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

// ---- lockstep batches of any mesh sizes: one launch per V-cycle step over every solve -------
// The solves of a batch share p and the cycle shape but may differ in mesh size and number
// of grids.  Their V-cycles are aligned from the finest grid down: at depth t (0 = finest) a
// solve with L grids is on its level L - 1 - t.  A launch covers up to kMixChunk solves of any
// sizes (blockIdx.y = solve), their descriptors for that depth in the kernel parameters;
// larger batches are cut into chunks that run as parallel branches of one graph.  A block
// whose solve is converged, past its coarsest level, not on a level that takes part in the
// step, or beyond that solve's work, returns at once.
template <typename T>
struct MixLevel {
  int level;                      // level index in the solve's hierarchy, -1 past its coarsest
  int lpr;                        // lanes per 8-DOF patch row of the level's colour kernel
  LevelTab<T> L, Lc;              // this level and (level >= 1) the next coarser one
  Xfer<T> tp, tq;                 // transfers between Lc and L
  const T *cinv, *cinv8, *kinv;   // local inverses; kinv: the coarsest level's dense inverse
  T *U, *F, *R, *Uc, *Fc;
  const int *dofs, *cls, *nloc;
  int maxl;
  int first[kMaxColours], n8[kMaxColours], cnt[kMaxColours];
  double* part;                   // residual partials (two per block of 256 rows)
  double* norm2;                  // ||F - K U||^2 of the finest level
  const int* active;              // 1 while the solve is iterating
};

constexpr int kMixChunk = 24;     // solves per launch (descriptors in the kernel parameters)

template <typename T>
struct MixArgs {
  int count;
  MixLevel<T> s[kMixChunk];
};

template <int P, typename T>
__global__ void __launch_bounds__(256) k_mix_colour(const __grid_constant__ MixArgs<T> A, int c) {
  const MixLevel<T>& d = A.s[blockIdx.y];
  if (d.level < 1 || !*d.active) return;
  const int wpb = blockDim.x >> 5, ppw = d.lpr == 2 ? 2 : 4;
  const int n8 = d.n8[c], ngen = d.cnt[c] - n8;
  const int nb8 = (n8 + ppw * wpb - 1) / (ppw * wpb), nbg = (ngen + wpb - 1) / wpb;
  if ((int)blockIdx.x >= nb8 + nbg) return;
  const LevelTab<T> L = d.L;
  T* U = d.U;
  const T* F = d.F;
  const int *dofs = d.dofs, *cls = d.cls, *nloc = d.nloc;
  const T *cinv = d.cinv, *cinv8 = d.cinv8;
  const int maxl = d.maxl, first = d.first[c];
  // the block walks the solve's blocks with the grid's stride (a descriptor read serves
  // several rounds of patches)
  for (int b = blockIdx.x; b < nb8 + nbg; b += gridDim.x) {
    if (d.lpr == 2)
      mult_colour_block<P, T, 2>(L, U, F, dofs, cls, cinv, cinv8, nloc, maxl, first, n8, ngen, nb8, b);
    else
      mult_colour_block<P, T, 1, 2>(L, U, F, dofs, cls, cinv, cinv8, nloc, maxl, first, n8, ngen, nb8, b);
  }
}

// R = F - K U with per-block partials; any_level: also for solves on their coarsest level
// (the finest level of a one-grid solve, for its norm)
template <int P, typename T>
__global__ void __launch_bounds__(256) k_mix_residual(const __grid_constant__ MixArgs<T> A,
                                                      int any_level) {
  __shared__ double sh[32];
  const MixLevel<T>& d = A.s[blockIdx.y];
  if (d.level < (any_level ? 0 : 1) || !*d.active) return;
  const LevelTab<T> L = d.L;
  if ((int)(blockIdx.x * blockDim.x) >= L.n_total - 1) return;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, mp = 0.0;
  if (g < L.n_total - 1) {
    T r = d.F[g] - row_KU<P, T, 2, 2>(L, d.U, g);
    d.R[g] = r;
    r2 = (double)r * (double)r;
    int off = g - L.n_ux - L.n_uy;
    if (off >= 0) mp = (double)mean_coef<P>(L, off) * (double)d.U[g];
  }
  double s1 = block_sum(r2, sh);
  double s2 = block_sum(mp, sh);
  if (threadIdx.x == 0) { d.part[2 * blockIdx.x] = s1; d.part[2 * blockIdx.x + 1] = s2; }
}

template <typename T>
__global__ void k_mix_residual_finish(const __grid_constant__ MixArgs<T> A, int any_level,
                                      int want_norm, int rows_per_part) {
  __shared__ double sh[32];
  const MixLevel<T>& d = A.s[blockIdx.x];
  if (d.level < (any_level ? 0 : 1) || !*d.active) return;
  const int n_total = d.L.n_total, nparts = (n_total - 1 + rows_per_part - 1) / rows_per_part;
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) { a += d.part[2 * i]; c += d.part[2 * i + 1]; }
  double s1 = block_sum(a, sh);
  double s2 = block_sum(c, sh);
  if (threadIdx.x == 0) {
    double rl = (double)d.F[n_total - 1] - s2;
    d.R[n_total - 1] = (T)rl;
    if (want_norm) *d.norm2 = s1 + rl * rl;
  }
}

// coarse F = P^T R
template <typename T>
__global__ void k_mix_restrict(const __grid_constant__ MixArgs<T> A) {
  const MixLevel<T>& d = A.s[blockIdx.y];
  if (d.level < 1 || !*d.active) return;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = d.Lc.n_total;
  if (g >= nc) return;
  d.Fc[g] = (g == nc - 1) ? d.R[d.L.n_total - 1] : restrict_elem(d.L, d.Lc, d.tp, d.tq, d.R, g);
}

// U += P Uc
template <typename T>
__global__ void k_mix_prolong_add(const __grid_constant__ MixArgs<T> A) {
  const MixLevel<T>& d = A.s[blockIdx.y];
  if (d.level < 1 || !*d.active) return;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = d.L.n_total;
  if (g >= nf) return;
  d.U[g] += (g == nf - 1) ? d.Uc[d.Lc.n_total - 1] : prolong_elem(d.L, d.Lc, d.tp, d.tq, d.Uc, g);
}

template <typename T>
__global__ void k_mix_zero(const __grid_constant__ MixArgs<T> A) {
  const MixLevel<T>& d = A.s[blockIdx.y];
  if (d.level < 1 || !*d.active) return;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < d.L.n_total) d.U[g] = T(0);
}

// U = K_0^{-1} F for the solves on their coarsest level at this depth, one block per solve
template <typename T>
__global__ void k_mix_coarse(const __grid_constant__ MixArgs<T> A) {
  const MixLevel<T>& d = A.s[blockIdx.x];
  if (d.level != 0 || !*d.active) return;
  extern __shared__ unsigned char smem_raw[];
  T* g = reinterpret_cast<T*>(smem_raw);
  const int n = d.L.n_total;
  for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = d.F[i];
  __syncthreads();
  int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x >> 5; i < n; i += nw) {
    const T* row = d.kinv + (size_t)i * n;
    T acc = T(0);
#pragma unroll 4
    for (int j = lane; j < n; j += 32) acc = fma(row[j], g[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) d.U[i] = acc;
  }
}

}  // namespace dev
}  // namespace igamg
