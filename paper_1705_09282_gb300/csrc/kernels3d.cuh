// Device kernels of the 3D (unit cube) V-cycle: Algorithm 1 with the multiplicative
// Schwarz smoother over vector-potential supports (Sec. 5.2), the transfers of Sec. 5.1 per
// tensor direction, templated on the degree P and on the value type T.
//
// Row evaluation: every row is three boxes of neighbours, each long along one axis
// (2P+1 or 2P positions) and 2P-1 wide across, read with one fused multiply-add per
// neighbour from the row's class record (records and layout: Stencils3 in
// igamg_internal.h).  Neighbour indices are clamped into range (their coefficients are
// zero), so no lane branches on where its row sits.
#pragma once
#include "kernels.cuh"

namespace igamg {
namespace dev {

template <typename T>
struct LevelTab3 {
  int n, ni, nq;                         // ni = n+p-2 (free degree-p indices 1..ni), nq = n+p-1
  int n_uc, n_u, n_p, n_total;
  const int *cm0, *cm1, *cm2, *cm3;      // class -> record, per row kind
  const T *rc0, *rc1, *rc2, *rc3;        // records, per row kind
  const T* srow;                         // per-row records (generalized Oseen), or null
  const T* sext;                         // mapped domains: per u_x / u_y row the 2P x 2P x (2Q+1)
                                         // coefficients on the other of the two, or null
};

template <int P>
struct Rec3 {
  static constexpr int Q = P - 1, W = 2 * Q + 1;
  static constexpr int B0 = (2 * P + 1) * W * W, B1 = 2 * P * W * W, RU = B0 + 2 * B1 + 1;
  static constexpr int TC = 2 * P + 1, NC = 2 * TC + 1;
};

__host__ __device__ __forceinline__ int sel3(int c, int a, int b, int d) { return c == 0 ? a : (c == 1 ? b : d); }

// row g -> kind (0..2 velocity component, 3 pressure) and full indices (x, y, z)
template <typename T>
__host__ __device__ __forceinline__ void decode3(const LevelTab3<T>& L, int g, int& kind, int& x, int& y, int& z) {
  kind = (g >= L.n_uc) + (g >= 2 * L.n_uc) + (g >= L.n_u);
  int base = kind < 3 ? kind * L.n_uc : L.n_u;
  int r = g - base;
  int dx = kind == 0 ? L.ni : L.nq, dy = kind == 1 ? L.ni : L.nq;
  int t = r / dx;
  x = r - t * dx;
  z = t / dy;
  y = t - z * dy;
  x += kind == 0; y += kind == 1; z += kind == 2;
}

// Per-axis data of block blk along axis a: valid full-index range [lo, hi] (local index =
// full - lo) and stride.
template <typename T>
__host__ __device__ __forceinline__ void axis3(const LevelTab3<T>& L, int blk, int a, int& lo, int& hi, int& stride) {
  bool own = blk < 3 && a == blk;
  lo = own ? 1 : 0;
  hi = own ? L.ni : L.nq - 1;
  int dx = blk == 0 ? L.ni : L.nq, dy = blk == 1 ? L.ni : L.nq;
  stride = a == 0 ? 1 : (a == 1 ? dx : dx * dy);
}

// sum over one box: LEN positions along axis c (from pos_c + org), 2Q+1 across on the two
// other axes (from pos - Q), coefficients coef[(a W + e1) W + e2].
template <int P, int LEN, typename T>
__host__ __device__ __forceinline__ T box3(const LevelTab3<T>& L, const T* __restrict__ coef, const T* __restrict__ U,
                                  int blk, int c, int org, int x, int y, int z) {
  constexpr int Q = P - 1, W = 2 * Q + 1;
  const int o1 = c == 2 ? 0 : c + 1, o2 = c == 0 ? 2 : c - 1;
  const int pc = sel3(c, x, y, z), p1 = sel3(o1, x, y, z), p2 = sel3(o2, x, y, z);
  int loc, hic, sc, lo1, hi1, s1, lo2, hi2, s2;
  axis3(L, blk, c, loc, hic, sc);
  axis3(L, blk, o1, lo1, hi1, s1);
  axis3(L, blk, o2, lo2, hi2, s2);
  const T* base = U + (blk < 3 ? blk * L.n_uc : L.n_u);
  int A[LEN], B1[W], B2[W];
#pragma unroll
  for (int a = 0; a < LEN; ++a) A[a] = (clampi(pc + org + a, loc, hic) - loc) * sc;
#pragma unroll
  for (int e = 0; e < W; ++e) {
    B1[e] = (clampi(p1 - Q + e, lo1, hi1) - lo1) * s1;
    B2[e] = (clampi(p2 - Q + e, lo2, hi2) - lo2) * s2;
  }
  T s0 = T(0), sA = T(0), sB = T(0), sC = T(0);
#pragma unroll
  for (int a = 0; a < LEN; ++a)
#pragma unroll
    for (int e1 = 0; e1 < W; ++e1)
#pragma unroll
      for (int e2 = 0; e2 < W; ++e2) {
        const int j = (a * W + e1) * W + e2;
        T v = base[A[a] + B1[e1] + B2[e2]];
        if ((j & 3) == 0) s0 = fma(coef[j], v, s0);
        else if ((j & 3) == 1) sA = fma(coef[j], v, sA);
        else if ((j & 3) == 2) sB = fma(coef[j], v, sB);
        else sC = fma(coef[j], v, sC);
      }
  return (s0 + sA) + (sB + sC);
}

// extra box of a u_x (kind 0) or u_y (kind 1) row on a mapped domain: the other component's
// columns x + ox .. x + ox + 2P - 1, y + oy .. y + oy + 2P - 1, z - Q .. z + Q (ox, oy = -P, -Q
// for u_x rows, -Q, -P for u_y rows), coefficients se[(a 2P + b) W + c]; clamped positions
// carry zero coefficients
template <int P, typename T>
__host__ __device__ __forceinline__ T ext3(const LevelTab3<T>& L, const T* __restrict__ se, const T* __restrict__ U,
                                  int kind, int x, int y, int z) {
  constexpr int Q = P - 1, W = 2 * Q + 1, L2 = 2 * P;
  const int ob = 1 - kind;
  const int ox = kind == 0 ? -P : -Q, oy = kind == 0 ? -Q : -P;
  int lo0, hi0, s0, lo1, hi1, s1, lo2, hi2, s2;
  axis3(L, ob, 0, lo0, hi0, s0);
  axis3(L, ob, 1, lo1, hi1, s1);
  axis3(L, ob, 2, lo2, hi2, s2);
  const T* base = U + ob * L.n_uc;
  int A[L2], B[L2], Cz[W];
#pragma unroll
  for (int a = 0; a < L2; ++a) {
    A[a] = (clampi(x + ox + a, lo0, hi0) - lo0) * s0;
    B[a] = (clampi(y + oy + a, lo1, hi1) - lo1) * s1;
  }
#pragma unroll
  for (int c = 0; c < W; ++c) Cz[c] = (clampi(z - Q + c, lo2, hi2) - lo2) * s2;
  T sa = T(0), sb = T(0);
#pragma unroll
  for (int a = 0; a < L2; ++a)
#pragma unroll
    for (int b = 0; b < L2; ++b)
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const int j = (a * L2 + b) * W + c;
        const T v = base[A[a] + B[b] + Cz[c]];
        if (j & 1) sb = fma(se[j], v, sb);
        else sa = fma(se[j], v, sa);
      }
  return sa + sb;
}

template <int P>
__host__ __device__ constexpr int ext3_len() { return 4 * P * P * (2 * P - 1); }

// record of row g = (kind; x, y, z)
template <int P, typename T>
__host__ __device__ __forceinline__ const T* rec3(const LevelTab3<T>& L, int kind, int x, int y, int z, int g) {
  using R = Rec3<P>;
  if (L.srow) return L.srow + (size_t)g * R::RU;
  const int lastp = L.n + P - 1, lastq = L.n + P - 2;
  int cx = cls1d<P>(x, kind == 0 ? lastp : lastq);
  int cy = cls1d<P>(y, kind == 1 ? lastp : lastq);
  int cz = cls1d<P>(z, kind == 2 ? lastp : lastq);
  int cl = (cz * R::NC + cy) * R::NC + cx;
  const int* cm = kind == 0 ? L.cm0 : (kind == 1 ? L.cm1 : (kind == 2 ? L.cm2 : L.cm3));
  const T* rc = kind == 0 ? L.rc0 : (kind == 1 ? L.rc1 : (kind == 2 ? L.rc2 : L.rc3));
  return rc + (size_t)cm[cl] * R::RU;
}

// (K U)_g for one row g (not lambda); *m gets the row's mean coefficient (p rows) or 0.
template <int P, typename T>
__host__ __device__ __forceinline__ T row3(const LevelTab3<T>& L, const T* __restrict__ U, int g, T* m = nullptr) {
  using R = Rec3<P>;
  int kind, x, y, z;
  decode3(L, g, kind, x, y, z);
  const T* rc = rec3<P>(L, kind, x, y, z, g);
  const bool vel = kind < 3;
  // box 0: own component (velocity rows) or u_x (pressure rows)
  T acc = box3<P, 2 * P + 1>(L, rc, U, vel ? kind : 0, vel ? kind : 0, vel ? -P : -(P - 1), x, y, z);
  // box 1: pressure (velocity rows) or u_y (pressure rows)
  acc += box3<P, 2 * P>(L, rc + R::B0, U, vel ? 3 : 1, vel ? kind : 1, vel ? -P : -(P - 1), x, y, z);
  if (!vel) {
    acc += box3<P, 2 * P>(L, rc + R::B0 + R::B1, U, 2, 2, -(P - 1), x, y, z);
    acc = fma(rc[R::RU - 1], U[L.n_total - 1], acc);
    if (m) *m = rc[R::RU - 1];
  } else {
    if (L.sext && kind < 2) acc += ext3<P>(L, L.sext + (size_t)g * ext3_len<P>(), U, kind, x, y, z);
    if (m) *m = T(0);
  }
  return acc;
}

// R = F - K U (every row but lambda); per-block partial sums of R^2 and of m.p.
template <int P, typename T>
__global__ void __launch_bounds__(256) k_residual3(LevelTab3<T> L, const T* __restrict__ U, const T* __restrict__ F,
                                                   T* __restrict__ R, double* __restrict__ part) {
  __shared__ double sh[32];
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, mp = 0.0;
  if (g < L.n_total - 1) {
    T m;
    T r = F[g] - row3<P>(L, U, g, &m);
    R[g] = r;
    r2 = (double)r * (double)r;
    mp = (double)m * (double)U[g];
  }
  double s1 = block_sum(r2, sh);
  double s2 = block_sum(mp, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1; part[2 * blockIdx.x + 1] = s2; }
}

// One colour of the multiplicative sweep (eq. MSM).  Blocks [0, nb8): four 8-DOF patches
// per warp, lane = (patch, local row); blocks [nb8, ...): one warp per larger patch.
template <int P, typename T>
__global__ void __launch_bounds__(256) k_mult_colour3(LevelTab3<T> L, T* __restrict__ U, const T* __restrict__ F,
                                                      const int* __restrict__ dofs, const int* __restrict__ cls,
                                                      const T* __restrict__ cinv, const T* __restrict__ cinv8,
                                                      const int* __restrict__ nloc, int maxl, int first, int n8,
                                                      int ngen, int nb8) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if ((int)blockIdx.x < nb8) {
    const int grp = (blockIdx.x * 8 + wib) * 4 + (lane >> 3), row = lane & 7;
    const bool active = grp < n8;
    const int patch = first + (active ? grp : 0);
    const int g = dofs[(size_t)patch * maxl + row];
    T r = F[g] - row3<P>(L, U, g);
    const T* A = cinv8 + (size_t)cls[patch] * 64 + row * 8;
    T d0 = T(0), d1 = T(0);
#pragma unroll
    for (int s = 0; s < 8; s += 2) {
      d0 = fma(A[s], __shfl_sync(0xffffffffu, r, (lane & ~7) + s), d0);
      d1 = fma(A[s + 1], __shfl_sync(0xffffffffu, r, (lane & ~7) + s + 1), d1);
    }
    if (active) U[g] += d0 + d1;
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  T* r = reinterpret_cast<T*>(smem_raw) + wib * maxl;
  const int w = ((int)blockIdx.x - nb8) * 8 + wib;
  if (w >= ngen) return;
  const int patch = first + n8 + w;
  const int c = cls[patch], nl = nloc[c];
  const int* pd = dofs + (size_t)patch * maxl;
  for (int k = lane; k < nl; k += 32) { int g = pd[k]; r[k] = F[g] - row3<P>(L, U, g); }
  __syncwarp();
  const T* A = cinv + (size_t)c * maxl * maxl;
  for (int k = lane; k < nl; k += 32) U[pd[k]] += dot_n(A + (size_t)k * maxl, r, nl);
}

// One colour of the multiplicative sweep, row-parallel: one thread per local row of a
// patch (slot), patches packed whole into blocks of S slots (S = 256, or 1024 on levels
// with larger patches).  Each thread forms its row's local residual into shared memory;
// after the barrier it applies its row of the patch's bordered inverse to the patch's
// residual and updates its own unknown.
template <int P, int S, typename T>
__global__ void __launch_bounds__(S) k_mult_rows3(LevelTab3<T> L, T* __restrict__ U, const T* __restrict__ F,
                                                  const int* __restrict__ slot_g, const int* __restrict__ slot_c,
                                                  const unsigned* __restrict__ slot_kb,
                                                  const T* __restrict__ cinv, const long long* __restrict__ cinv_off,
                                                  int first_slot) {
  __shared__ T r[S];
  const int s = first_slot + blockIdx.x * S + threadIdx.x;
  const int g = slot_g[s];
  T rv = T(0);
  if (g >= 0) rv = F[g] - row3<P>(L, U, g);
  r[threadIdx.x] = rv;
  __syncthreads();
  if (g < 0) return;
  const unsigned kb = slot_kb[s];
  const int k = kb & 0x3ff, nl = (kb >> 10) & 0x3ff, base = kb >> 20;
  U[g] += dot_n(cinv + cinv_off[slot_c[s]] + (size_t)k * nl, r + base, nl);
}

// The same colour step with each row's three neighbour boxes evaluated by three different
// threads (warps [0, S/32) box 0 with F, the next S/32 warps box 1, the last S/32 box 2 and
// the lambda term), so every thread's chain of loads and multiply-adds is about a third as
// long: for levels where a colour has too few rows to hide that latency.  Every warp runs
// one box shape, so no warp diverges; the partial sums meet in shared memory.
template <int P, int S, typename T>
__global__ void __launch_bounds__(3 * S) k_mult_rows3x(LevelTab3<T> L, T* __restrict__ U, const T* __restrict__ F,
                                                       const int* __restrict__ slot_g, const int* __restrict__ slot_c,
                                                       const unsigned* __restrict__ slot_kb,
                                                       const T* __restrict__ cinv, const long long* __restrict__ cinv_off,
                                                       int first_slot) {
  using R = Rec3<P>;
  __shared__ T part[3][S];
  const int w = threadIdx.x / S, t = threadIdx.x - w * S;
  const int s = first_slot + blockIdx.x * S + t;
  const int g = slot_g[s];
  T acc = T(0);
  if (g >= 0) {
    int kind, x, y, z;
    decode3(L, g, kind, x, y, z);
    const T* rc = rec3<P>(L, kind, x, y, z, g);
    const bool vel = kind < 3;
    if (w == 0) {
      acc = F[g] - box3<P, 2 * P + 1>(L, rc, U, vel ? kind : 0, vel ? kind : 0, vel ? -P : -(P - 1), x, y, z);
    } else if (w == 1) {
      acc = -box3<P, 2 * P>(L, rc + R::B0, U, vel ? 3 : 1, vel ? kind : 1, vel ? -P : -(P - 1), x, y, z);
    } else if (!vel) {
      acc = -fma(rc[R::RU - 1], U[L.n_total - 1], box3<P, 2 * P>(L, rc + R::B0 + R::B1, U, 2, 2, -(P - 1), x, y, z));
    } else if (L.sext && kind < 2) {
      acc = -ext3<P>(L, L.sext + (size_t)g * ext3_len<P>(), U, kind, x, y, z);
    }
  }
  part[w][t] = acc;
  __syncthreads();
  if (w == 0) part[0][t] = acc + (part[1][t] + part[2][t]);
  __syncthreads();
  if (w != 0 || g < 0) return;
  const unsigned kb = slot_kb[s];
  const int k = kb & 0x3ff, nl = (kb >> 10) & 0x3ff, base = kb >> 20;
  U[g] += dot_n(cinv + cinv_off[slot_c[s]] + (size_t)k * nl, &part[0][0] + base, nl);
}

// block and local (x, y, z) of entry g (not lambda) on a level
template <typename T>
__device__ __forceinline__ void split3(const LevelTab3<T>& L, int g, int& blk, int& x, int& y, int& z, int& dx, int& dy) {
  blk = (g >= L.n_uc) + (g >= 2 * L.n_uc) + (g >= L.n_u);
  int r = g - (blk < 3 ? blk * L.n_uc : L.n_u);
  dx = blk == 0 ? L.ni : L.nq;
  dy = blk == 1 ? L.ni : L.nq;
  int t = r / dx;
  x = r - t * dx;
  z = t / dy;
  y = t - z * dy;
}

// (P u_c) at fine entry g (not lambda): the 3 x 3 x 3 tensor product of 1D knot-insertion
// weights (degree p along the component's own axis, p-1 across; all p-1 for the pressure).
template <typename T>
__device__ __forceinline__ T prolong3_elem(const LevelTab3<T>& Lf, const LevelTab3<T>& Lc, const Xfer<T>& tp,
                                           const Xfer<T>& tq, const T* __restrict__ uc, int g) {
  int blk, x, y, z, dx, dy;
  split3(Lf, g, blk, x, y, z, dx, dy);
  const Xfer<T>& X = blk == 0 ? tp : tq;
  const Xfer<T>& Y = blk == 1 ? tp : tq;
  const Xfer<T>& Z = blk == 2 ? tp : tq;
  const int cdx = blk == 0 ? Lc.ni : Lc.nq, cdy = blk == 1 ? Lc.ni : Lc.nq;
  const T* src = uc + (blk < 3 ? blk * Lc.n_uc : Lc.n_u);
  const int cx0 = X.c0[x], cy0 = Y.c0[y], cz0 = Z.c0[z];
  T acc = T(0);
#pragma unroll
  for (int kz = 0; kz < kWP; ++kz) {
    int cz = min(cz0 + kz, Z.nc - 1);            // weights past the end are zero
    T sy = T(0);
#pragma unroll
    for (int ky = 0; ky < kWP; ++ky) {
      int cy = min(cy0 + ky, Y.nc - 1);
      const T* rowp = src + ((size_t)cz * cdy + cy) * cdx;
      T sx = T(0);
#pragma unroll
      for (int kx = 0; kx < kWP; ++kx) sx = fma(X.pv[x * kWP + kx], rowp[min(cx0 + kx, X.nc - 1)], sx);
      sy = fma(Y.pv[y * kWP + ky], sx, sy);
    }
    acc = fma(Z.pv[z * kWP + kz], sy, acc);
  }
  return acc;
}

// (P^T r_f) at coarse entry g (not lambda): the 5 x 5 x 5 tensor product of the transposed weights.
template <typename T>
__device__ __forceinline__ T restrict3_elem(const LevelTab3<T>& Lf, const LevelTab3<T>& Lc, const Xfer<T>& tp,
                                            const Xfer<T>& tq, const T* __restrict__ rf, int g) {
  int blk, x, y, z, dx, dy;
  split3(Lc, g, blk, x, y, z, dx, dy);
  const Xfer<T>& X = blk == 0 ? tp : tq;
  const Xfer<T>& Y = blk == 1 ? tp : tq;
  const Xfer<T>& Z = blk == 2 ? tp : tq;
  const int fdx = blk == 0 ? Lf.ni : Lf.nq, fdy = blk == 1 ? Lf.ni : Lf.nq;
  const T* src = rf + (blk < 3 ? blk * Lf.n_uc : Lf.n_u);
  const int fx0 = X.f0[x], fy0 = Y.f0[y], fz0 = Z.f0[z];
  T acc = T(0);
#pragma unroll
  for (int kz = 0; kz < kWR; ++kz) {
    int fz = min(fz0 + kz, Z.nf - 1);
    T sy = T(0);
#pragma unroll
    for (int ky = 0; ky < kWR; ++ky) {
      int fy = min(fy0 + ky, Y.nf - 1);
      const T* rowp = src + ((size_t)fz * fdy + fy) * fdx;
      T sx = T(0);
#pragma unroll
      for (int kx = 0; kx < kWR; ++kx) sx = fma(X.rv[x * kWR + kx], rowp[min(fx0 + kx, X.nf - 1)], sx);
      sy = fma(Y.rv[y * kWR + ky], sx, sy);
    }
    acc = fma(Z.rv[z * kWR + kz], sy, acc);
  }
  return acc;
}

// u_f += P u_c (lambda added); one thread per fine entry.
template <typename T>
__global__ void k_prolong_add3(LevelTab3<T> Lf, LevelTab3<T> Lc, Xfer<T> tp, Xfer<T> tq, const T* __restrict__ uc,
                               T* __restrict__ uf) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lf.n_total) return;
  uf[g] += (g == Lf.n_total - 1) ? uc[Lc.n_total - 1] : prolong3_elem(Lf, Lc, tp, tq, uc, g);
}

// g_c = P^T r_f (lambda copied); one thread per coarse entry.
template <typename T>
__global__ void k_restrict3(LevelTab3<T> Lf, LevelTab3<T> Lc, Xfer<T> tp, Xfer<T> tq, const T* __restrict__ rf,
                            T* __restrict__ gc) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lc.n_total) return;
  gc[g] = (g == Lc.n_total - 1) ? rf[Lf.n_total - 1] : restrict3_elem(Lf, Lc, tp, tq, rf, g);
}

// ---- the coarse end of the 3D V-cycle in one thread-block cluster -----------------------
// As k_cluster_coarse (2D): the phases of Algorithm 1 for levels 0..lc spread over the
// blocks of one cluster, separated by the cluster barrier, vectors in global memory (L2).
// A colour is processed one slot block (k_mult_rows3's packing) per block iteration: with
// 128- or 256-slot blocks each row's three neighbour boxes go to three groups of S threads, as
// in k_mult_rows3x; with 1024-slot blocks (levels whose patches exceed 256 rows) one thread per row.
constexpr int kMaxFused3 = 6;

template <typename T>
struct Cluster3Level {
  LevelTab3<T> L;
  Xfer<T> tp, tq;                   // transfer from the level below into this one (l >= 1)
  const T* cinv;                    // cinv_all of the level
  const long long* cinv_off;
  const int *slot_g, *slot_c, *colour_blk;
  const unsigned* slot_kb;
  int n_colours, maxl, row_slots;
  T *U, *F, *R;
};

template <typename T>
struct Cluster3Desc {
  int nlev, nu1, nu2, ndof0;
  const T* coarse_inv;
  double* part;
  Cluster3Level<T> lev[kMaxFused3];
};

template <int P, typename T>
__global__ void __launch_bounds__(1024) k_cluster3(Cluster3Desc<T> D, const T* __restrict__ Ftop, T* __restrict__ Utop,
                                                   int load_u) {
  using R = Rec3<P>;
  __shared__ T part3[1024];
  __shared__ double red[32];
  const unsigned rank = blockIdx.x, C = gridDim.x;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  const int gtid = rank * nt + tid, gnt = C * nt, gwarp = rank * nwarp + warp, gnwarp = C * nwarp;
  const int lc = D.nlev - 1;
  auto csync = []() { asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory"); };
  auto Uof = [&](int l) { return l == lc ? Utop : D.lev[l].U; };
  auto Fof = [&](int l) { return l == lc ? Ftop : (const T*)D.lev[l].F; };
  if (!load_u) {
    for (int i = gtid; i < D.lev[lc].L.n_total; i += gnt) Utop[i] = T(0);
    csync();
  }
  auto smooth = [&](int l) {
    const Cluster3Level<T>& V = D.lev[l];
    T* U = Uof(l); const T* F = Fof(l);
    const int S = V.row_slots;
    for (int c = 0; c < V.n_colours; ++c) {
      const int b0 = V.colour_blk[c], b1 = V.colour_blk[c + 1];
      for (int b = b0 + (int)rank; b < b1; b += (int)C) {
        if (S <= 256) {
          const int w = tid / S, t = tid - w * S;
          const int s = b * S + t;
          const int g = w < 3 ? V.slot_g[s] : -1;
          T acc = T(0);
          if (g >= 0) {
            int kind, x, y, z;
            decode3(V.L, g, kind, x, y, z);
            const T* rc = rec3<P>(V.L, kind, x, y, z, g);
            const bool vel = kind < 3;
            if (w == 0)
              acc = F[g] - box3<P, 2 * P + 1>(V.L, rc, U, vel ? kind : 0, vel ? kind : 0, vel ? -P : -(P - 1), x, y, z);
            else if (w == 1)
              acc = -box3<P, 2 * P>(V.L, rc + R::B0, U, vel ? 3 : 1, vel ? kind : 1, vel ? -P : -(P - 1), x, y, z);
            else if (!vel)
              acc = -fma(rc[R::RU - 1], U[V.L.n_total - 1], box3<P, 2 * P>(V.L, rc + R::B0 + R::B1, U, 2, 2, -(P - 1), x, y, z));
            else if (V.L.sext && kind < 2)
              acc = -ext3<P>(V.L, V.L.sext + (size_t)g * ext3_len<P>(), U, kind, x, y, z);
          }
          part3[tid] = acc;
          __syncthreads();
          if (w == 0) part3[t] = acc + (part3[S + t] + part3[2 * S + t]);
          __syncthreads();
          if (w == 0 && g >= 0) {
            const unsigned kb = V.slot_kb[s];
            const int k = kb & 0x3ff, nl = (kb >> 10) & 0x3ff, base = kb >> 20;
            U[g] += dot_n(V.cinv + V.cinv_off[V.slot_c[s]] + (size_t)k * nl, part3 + base, nl);
          }
          __syncthreads();
        } else {
          const int s = b * S + tid;
          const int g = tid < S ? V.slot_g[s] : -1;
          T rv = T(0);
          if (g >= 0) rv = F[g] - row3<P>(V.L, U, g);
          part3[tid] = rv;
          __syncthreads();
          if (g >= 0) {
            const unsigned kb = V.slot_kb[s];
            const int k = kb & 0x3ff, nl = (kb >> 10) & 0x3ff, base = kb >> 20;
            U[g] += dot_n(V.cinv + V.cinv_off[V.slot_c[s]] + (size_t)k * nl, part3 + base, nl);
          }
          __syncthreads();
        }
      }
      csync();
    }
  };
  for (int l = lc; l >= 1; --l) {
    for (int k = 0; k < D.nu1; ++k) smooth(l);
    const Cluster3Level<T>& V = D.lev[l];
    const Cluster3Level<T>& Cl = D.lev[l - 1];
    {  // residual (all rows but lambda) and this block's share of m . p
      const T* U = Uof(l); const T* F = Fof(l); T* Rv = V.R;
      double mp = 0.0;
      for (int g = gtid; g < V.L.n_total - 1; g += gnt) {
        T m;
        Rv[g] = F[g] - row3<P>(V.L, U, g, &m);
        mp += (double)m * (double)U[g];
      }
      double sblk = block_sum(mp, red);
      if (tid == 0) D.part[rank] = sblk;
      csync();
      if (gtid == 0) {
        double sm = 0.0;
        for (unsigned b = 0; b < C; ++b) sm += D.part[b];
        Rv[V.L.n_total - 1] = (T)((double)F[V.L.n_total - 1] - sm);
      }
      csync();
    }
    {  // restriction into level l-1, and U_{l-1} = 0
      const T* Rv = V.R;
      T* Fc = Cl.F; T* Uc = Cl.U;
      for (int g = gtid; g < Cl.L.n_total; g += gnt) {
        Fc[g] = (g == Cl.L.n_total - 1) ? Rv[V.L.n_total - 1] : restrict3_elem(V.L, Cl.L, V.tp, V.tq, Rv, g);
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
    const Cluster3Level<T>& V = D.lev[l];
    const Cluster3Level<T>& Cl = D.lev[l - 1];
    T* U = Uof(l); const T* Uc = Cl.U;
    for (int g = gtid; g < V.L.n_total; g += gnt)
      U[g] += (g == V.L.n_total - 1) ? Uc[Cl.L.n_total - 1] : prolong3_elem(V.L, Cl.L, V.tp, V.tq, Uc, g);
    csync();
    for (int k = 0; k < D.nu2; ++k) smooth(l);
  }
}

}  // namespace dev
}  // namespace igamg
