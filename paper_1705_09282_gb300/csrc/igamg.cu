// CUDA kernels and the C ABI of the geometric multigrid V-cycle (arXiv 1705.09282,
// Algorithm 1 with the overlapping Schwarz smoothers of Sec. 5.2), for sm_103a.
//
// Every level's operator is applied matrix-free from its 1D banded factors (Kronecker
// form, see setup.cpp).  The multiplicative smoother runs one launch per patch colour:
// inside a colour the patches share no degree of freedom and are not coupled by K, so
// solving them concurrently is the same as solving them one after another (eq. MSM).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "igamg_internal.h"

using namespace igamg;

namespace {

constexpr int kBlock = 256;

template <typename T>
struct LevelDev {
  int n, nxu, nyu, npd, nint;   // nint = n+p-2 (interior degree-p count)
  long long n_ux, n_uy, n_p, n_total;
  const T *X1, *X2, *Mq, *Y2, *D, *mq;
};

struct XferDev {
  int nf, nc;
  const int *c0, *f0;
  const double *pv, *rv;
};

// (K U)_g for one row g (not the lambda row), from the 1D bands; Sec. 3.4 block structure.
template <int P, typename T>
__device__ __forceinline__ T row_KU(const LevelDev<T>& L, const T* __restrict__ U, long long g) {
  constexpr int Q = P - 1, W = 2 * P + 1;
  const T* ux = U;
  const T* uy = U + L.n_ux;
  const T* pr = U + L.n_ux + L.n_uy;
  T acc = 0;
  if (g < L.n_ux) {
    int iy = (int)(g / L.nxu), ix = (int)(g % L.nxu) + 1;
    const T* x1 = L.X1 + (size_t)ix * W; const T* x2 = L.X2 + (size_t)ix * W;
    const T* mq = L.Mq + (size_t)iy * W; const T* y2 = L.Y2 + (size_t)iy * W;
#pragma unroll
    for (int dx = -P; dx <= P; ++dx) {
      int jx = ix + dx;
      if (jx < 1 || jx > L.nint) continue;
      T a1 = x1[dx + P], a2 = x2[dx + P];
#pragma unroll
      for (int dy = -Q; dy <= Q; ++dy) {
        int jy = iy + dy;
        if (jy < 0 || jy >= L.nyu) continue;
        acc += (a1 * mq[dy + P] + a2 * y2[dy + P]) * ux[(size_t)jy * L.nxu + jx - 1];
      }
    }
    const T* d = L.D + (size_t)ix * W;
#pragma unroll
    for (int dx = -P; dx <= P - 1; ++dx) {
      int kx = ix + dx;
      if (kx < 0 || kx >= L.npd) continue;
      T dd = d[dx + P];
#pragma unroll
      for (int dy = -Q; dy <= Q; ++dy) {
        int ky = iy + dy;
        if (ky < 0 || ky >= L.npd) continue;
        acc -= dd * mq[dy + P] * pr[(size_t)ky * L.npd + kx];
      }
    }
  } else if (g < L.n_ux + L.n_uy) {
    long long r = g - L.n_ux;
    int iy = (int)(r / L.npd) + 1, ix = (int)(r % L.npd);
    const T* mqx = L.Mq + (size_t)ix * W; const T* y2x = L.Y2 + (size_t)ix * W;
    const T* x1 = L.X1 + (size_t)iy * W; const T* x2 = L.X2 + (size_t)iy * W;
#pragma unroll
    for (int dx = -Q; dx <= Q; ++dx) {
      int jx = ix + dx;
      if (jx < 0 || jx >= L.npd) continue;
      T a1 = mqx[dx + P], a2 = y2x[dx + P];
#pragma unroll
      for (int dy = -P; dy <= P; ++dy) {
        int jy = iy + dy;
        if (jy < 1 || jy > L.nint) continue;
        acc += (a1 * x1[dy + P] + a2 * x2[dy + P]) * uy[(size_t)(jy - 1) * L.npd + jx];
      }
    }
    const T* d = L.D + (size_t)iy * W;
#pragma unroll
    for (int dx = -Q; dx <= Q; ++dx) {
      int kx = ix + dx;
      if (kx < 0 || kx >= L.npd) continue;
      T m = mqx[dx + P];
#pragma unroll
      for (int dy = -P; dy <= P - 1; ++dy) {
        int ky = iy + dy;
        if (ky < 0 || ky >= L.npd) continue;
        acc -= m * d[dy + P] * pr[(size_t)ky * L.npd + kx];
      }
    }
  } else {
    long long r = g - L.n_ux - L.n_uy;
    int ky = (int)(r / L.npd), kx = (int)(r % L.npd);
    const T* mqx = L.Mq + (size_t)kx * W; const T* mqy = L.Mq + (size_t)ky * W;
    // B_x^T u_x : D(ix,kx) Mq(iy,ky), ix in [kx-Q, kx+P]
#pragma unroll
    for (int s = -Q; s <= P; ++s) {
      int ix = kx + s;
      if (ix < 1 || ix > L.nint) continue;
      T dd = L.D[(size_t)ix * W + (kx - ix + P)];
#pragma unroll
      for (int dy = -Q; dy <= Q; ++dy) {
        int iy = ky + dy;
        if (iy < 0 || iy >= L.nyu) continue;
        acc += dd * mqy[dy + P] * ux[(size_t)iy * L.nxu + ix - 1];
      }
    }
    // B_y^T u_y : Mq(ix,kx) D(iy,ky), iy in [ky-Q, ky+P]
#pragma unroll
    for (int s = -Q; s <= P; ++s) {
      int iy = ky + s;
      if (iy < 1 || iy > L.nint) continue;
      T dd = L.D[(size_t)iy * W + (ky - iy + P)];
#pragma unroll
      for (int dx = -Q; dx <= Q; ++dx) {
        int ix = kx + dx;
        if (ix < 0 || ix >= L.npd) continue;
        acc += mqx[dx + P] * dd * uy[(size_t)(iy - 1) * L.npd + ix];
      }
    }
    acc += L.mq[kx] * L.mq[ky] * U[L.n_total - 1];
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  T s = 0;
  if (w == 0) {
    s = (l < (int)(blockDim.x >> 5)) ? sh[l] : T(0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// R = F - K U for every row but lambda; per-block partial sums of R^2 and of m.p.
template <int P, typename T>
__global__ void k_residual(LevelDev<T> L, const T* __restrict__ U, const T* __restrict__ F,
                           T* __restrict__ R, double* __restrict__ part) {
  __shared__ double sh[32];
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, mp = 0.0;
  if (g < L.n_total - 1) {
    T r = F[g] - row_KU<P>(L, U, g);
    R[g] = r;
    r2 = (double)r * (double)r;
    long long off = g - L.n_ux - L.n_uy;
    if (off >= 0) {
      int ky = (int)(off / L.npd), kx = (int)(off % L.npd);
      mp = (double)L.mq[kx] * (double)L.mq[ky] * (double)U[g];
    }
  }
  double s1 = block_sum(r2, sh);
  double s2 = block_sum(mp, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1; part[2 * blockIdx.x + 1] = s2; }
}

// lambda row and ||R||^2 from the partials (one block, fixed order).
template <typename T>
__global__ void k_residual_finish(long long n_total, const T* __restrict__ F, T* __restrict__ R,
                                  const double* __restrict__ part, int nparts, double* __restrict__ norm2) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) { a += part[2 * i]; b += part[2 * i + 1]; }
  double s1 = block_sum(a, sh);
  double s2 = block_sum(b, sh);
  if (threadIdx.x == 0) {
    T rl = F[n_total - 1] - (T)s2;
    R[n_total - 1] = rl;
    if (norm2) *norm2 = s1 + (double)rl * (double)rl;
  }
}

// One colour of the multiplicative Schwarz sweep: one warp per patch.  Lanes gather the
// local residual rows, then apply the bordered local inverse and update U in place.
template <int P, typename T>
__global__ void k_mult_colour(LevelDev<T> L, T* __restrict__ U, const T* __restrict__ F,
                              const int* __restrict__ dofs, const int* __restrict__ cls,
                              const T* __restrict__ cinv, const int* __restrict__ nloc,
                              int maxl, int first, int count) {
  extern __shared__ unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= count) return;
  int patch = first + warp;
  int c = cls[patch], nl = nloc[c];
  T* r = sh + (threadIdx.x >> 5) * maxl;
  const int* pd = dofs + (size_t)patch * maxl;
  for (int k = lane; k < nl; k += 32) { int g = pd[k]; r[k] = F[g] - row_KU<P>(L, U, g); }
  __syncwarp();
  const T* A = cinv + (size_t)c * maxl * maxl;
  for (int k = lane; k < nl; k += 32) {
    T acc = 0;
    const T* a = A + (size_t)k * maxl;
    for (int s = 0; s < nl; ++s) acc += a[s] * r[s];
    U[pd[k]] += acc;
  }
}

// Additive sweep, part 1: local corrections from a common residual, kept per patch.
template <typename T>
__global__ void k_add_local(const T* __restrict__ R, const int* __restrict__ dofs, const int* __restrict__ cls,
                            const T* __restrict__ cinv, const int* __restrict__ nloc, int maxl,
                            int count, T* __restrict__ delta) {
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
  for (int k = lane; k < nl; k += 32) {
    T acc = 0;
    for (int s = 0; s < nl; ++s) acc += A[(size_t)k * maxl + s] * r[s];
    delta[(size_t)warp * maxl + k] = acc;
  }
}

// Additive sweep, part 2: U_g += eta * sum of the corrections of the patches holding g.
template <typename T>
__global__ void k_add_gather(long long n, T* __restrict__ U, const T* __restrict__ delta,
                             const int* __restrict__ off, const int* __restrict__ idx, T eta) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  T s = 0;
  for (int j = off[g]; j < off[g + 1]; ++j) s += delta[idx[j]];
  if (off[g + 1] > off[g]) U[g] += eta * s;
}

// g_c = P^T r_f on all blocks (lambda copied).  fine/coarse layouts from the LevelDevs.
template <typename T>
__global__ void k_restrict(LevelDev<T> Lf, LevelDev<T> Lc, XferDev tp, XferDev tq,
                           const T* __restrict__ rf, T* __restrict__ gc) {
  constexpr int WR = Transfer1D::WR;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lc.n_total) return;
  if (g == Lc.n_total - 1) { gc[g] = rf[Lf.n_total - 1]; return; }
  const XferDev *TX, *TY;
  int cx, cy, fnx;
  const T* src;
  if (g < Lc.n_ux) { cy = (int)(g / Lc.nxu); cx = (int)(g % Lc.nxu); TX = &tp; TY = &tq; src = rf; fnx = Lf.nxu; }
  else if (g < Lc.n_ux + Lc.n_uy) { long long r = g - Lc.n_ux; cy = (int)(r / Lc.npd); cx = (int)(r % Lc.npd); TX = &tq; TY = &tp; src = rf + Lf.n_ux; fnx = Lf.npd; }
  else { long long r = g - Lc.n_ux - Lc.n_uy; cy = (int)(r / Lc.npd); cx = (int)(r % Lc.npd); TX = &tq; TY = &tq; src = rf + Lf.n_ux + Lf.n_uy; fnx = Lf.npd; }
  int fx0 = TX->f0[cx], fy0 = TY->f0[cy];
  T acc = 0;
#pragma unroll
  for (int ky = 0; ky < WR; ++ky) {
    int fy = fy0 + ky;
    T wy = (T)TY->rv[(size_t)cy * WR + ky];
    if (fy >= TY->nf || wy == T(0)) continue;
#pragma unroll
    for (int kx = 0; kx < WR; ++kx) {
      int fx = fx0 + kx;
      T wx = (T)TX->rv[(size_t)cx * WR + kx];
      if (fx >= TX->nf || wx == T(0)) continue;
      acc += wy * wx * src[(size_t)fy * fnx + fx];
    }
  }
  gc[g] = acc;
}

// u_f += P u_c (lambda added).
template <typename T>
__global__ void k_prolong_add(LevelDev<T> Lf, LevelDev<T> Lc, XferDev tp, XferDev tq,
                              const T* __restrict__ uc, T* __restrict__ uf) {
  constexpr int WP = Transfer1D::WP;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lf.n_total) return;
  if (g == Lf.n_total - 1) { uf[g] += uc[Lc.n_total - 1]; return; }
  const XferDev *TX, *TY;
  int fx, fy, cnx;
  const T* src;
  if (g < Lf.n_ux) { fy = (int)(g / Lf.nxu); fx = (int)(g % Lf.nxu); TX = &tp; TY = &tq; src = uc; cnx = Lc.nxu; }
  else if (g < Lf.n_ux + Lf.n_uy) { long long r = g - Lf.n_ux; fy = (int)(r / Lf.npd); fx = (int)(r % Lf.npd); TX = &tq; TY = &tp; src = uc + Lc.n_ux; cnx = Lc.npd; }
  else { long long r = g - Lf.n_ux - Lf.n_uy; fy = (int)(r / Lf.npd); fx = (int)(r % Lf.npd); TX = &tq; TY = &tq; src = uc + Lc.n_ux + Lc.n_uy; cnx = Lc.npd; }
  int cx0 = TX->c0[fx], cy0 = TY->c0[fy];
  T acc = 0;
#pragma unroll
  for (int ky = 0; ky < WP; ++ky) {
    int cy = cy0 + ky;
    T wy = (T)TY->pv[(size_t)fy * WP + ky];
    if (cy >= TY->nc || wy == T(0)) continue;
#pragma unroll
    for (int kx = 0; kx < WP; ++kx) {
      int cx = cx0 + kx;
      T wx = (T)TX->pv[(size_t)fx * WP + kx];
      if (cx >= TX->nc || wx == T(0)) continue;
      acc += wy * wx * src[(size_t)cy * cnx + cx];
    }
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
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T acc = 0;
    for (int j = 0; j < n; ++j) acc += Kinv[(size_t)i * n + j] * g[j];
    U[i] = acc;
  }
}

// max |div u| over the (n+q)^2 pressure-space coefficients (order-free max via bits).
__global__ void k_div_inf(LevelDev<double> L, const double* __restrict__ dcoef, const double* __restrict__ U,
                          unsigned long long* __restrict__ out) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (k < L.n_p) {
    int ky = (int)(k / L.npd), kx = (int)(k % L.npd);
    const double* ux = U;
    const double* uy = U + L.n_ux;
    auto UX = [&](int ix, int iy) { return (ix < 1 || ix > L.nint) ? 0.0 : ux[(size_t)iy * L.nxu + ix - 1]; };
    auto UY = [&](int ix, int iy) { return (iy < 1 || iy > L.nint) ? 0.0 : uy[(size_t)(iy - 1) * L.npd + ix]; };
    double c = dcoef[kx] * (UX(kx + 1, ky) - UX(kx, ky)) + dcoef[ky] * (UY(kx, ky + 1) - UY(kx, ky));
    v = fabs(c);
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// velocity = curl psi, psi on the (n+p-2)^2 interior streamfunction coefficients.
__global__ void k_curl(LevelDev<double> L, const double* __restrict__ dcoef, const double* __restrict__ psi,
                       double* __restrict__ U) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_ux + L.n_uy) return;
  int ni = L.nint;
  auto PS = [&](int ix, int iy) { return (ix < 1 || ix > ni || iy < 1 || iy > ni) ? 0.0 : psi[(size_t)(iy - 1) * ni + ix - 1]; };
  if (g < L.n_ux) {
    int ky = (int)(g / L.nxu), ix = (int)(g % L.nxu) + 1;
    U[g] = dcoef[ky] * (PS(ix, ky + 1) - PS(ix, ky));
  } else {
    long long r = g - L.n_ux;
    int iy = (int)(r / L.npd) + 1, kx = (int)(r % L.npd);
    U[g] = -dcoef[kx] * (PS(kx + 1, iy) - PS(kx, iy));
  }
}

// F = (int v.f, 0, 0) on the finest level; tables hold weight * basis value per local element.
template <int P>
__global__ void k_load(LevelDev<double> L, const double* __restrict__ lvp, const double* __restrict__ lvq,
                       const double* __restrict__ f, double* __restrict__ F) {
  constexpr int Q = P - 1, G = P + 2;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_total) return;
  if (g >= L.n_ux + L.n_uy) { F[g] = 0.0; return; }
  int n = L.n, nG = n * G;
  int ix, iy, dxg, dyg;
  const double *tx, *ty, *fc;
  if (g < L.n_ux) { iy = (int)(g / L.nxu); ix = (int)(g % L.nxu) + 1; dxg = P; dyg = Q; tx = lvp; ty = lvq; fc = f; }
  else { long long r = g - L.n_ux; iy = (int)(r / L.npd) + 1; ix = (int)(r % L.npd); dxg = Q; dyg = P; tx = lvq; ty = lvp; fc = f + (size_t)nG * nG; }
  double acc = 0.0;
  for (int ky = 0; ky <= dyg; ++ky) {
    int ey = iy - dyg + ky;
    if (ey < 0 || ey >= n) continue;
    for (int kx = 0; kx <= dxg; ++kx) {
      int ex = ix - dxg + kx;
      if (ex < 0 || ex >= n) continue;
      const double* wx = tx + ((size_t)ix * (dxg + 1) + kx) * G;
      const double* wy = ty + ((size_t)iy * (dyg + 1) + ky) * G;
      for (int gy = 0; gy < G; ++gy) {
        const double* row = fc + (size_t)(ey * G + gy) * nG + ex * G;
        double s = 0.0;
        for (int gx = 0; gx < G; ++gx) s += wx[gx] * row[gx];
        acc += wy[gy] * s;
      }
    }
  }
  F[g] = acc;
}

inline unsigned nblk(long long n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------------------
struct DevLevel {
  igamg_sizes sz{};
  LevelDev<double> L{};
  double* bands = nullptr;      // X1 X2 Mq Y2 D mq dcoef
  const double* dcoef = nullptr;
  // patches
  int n_patches = 0, maxl = 0, n_colours = 0;
  std::vector<int> colour_off;
  int *dofs = nullptr, *cls = nullptr, *nloc = nullptr, *d2p_off = nullptr, *d2p_idx = nullptr;
  double* cinv = nullptr;
  // transfer from level-1 (valid for level >= 1)
  XferDev tp{}, tq{};
  void* xfer_mem = nullptr;
  // workspaces
  double *U = nullptr, *F = nullptr, *R = nullptr;
};

struct igamg_handle {
  igamg_problem prob{};
  HierarchyHost host;
  cudaStream_t stream = nullptr;
  std::vector<DevLevel> lev;
  double* coarse_inv = nullptr;
  int ndof0 = 0;
  double* part = nullptr;      // residual partials (2 per block of the finest level)
  double* norm2 = nullptr;     // device scalar
  unsigned long long* divmax = nullptr;
  double* delta = nullptr;     // additive corrections, n_patches * maxl (max over levels)
  double* lv_p = nullptr; double* lv_q = nullptr;
  double* h_pinned = nullptr;  // 2 doubles
  // host-buffer solve workspaces
  double *f_dev = nullptr, *Fh = nullptr, *Uh = nullptr;
  // captured V-cycle (+ residual norm) graph, keyed by the fine U/F pointers
  cudaGraphExec_t graph = nullptr;
  const void* gU = nullptr; const void* gF = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<void*> allocs;
};

namespace {

thread_local std::string g_err;

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { g_err = std::string(#x) + ": " + cudaGetErrorString(e_); return IGAMG_ECUDA; } } while (0)

int dmalloc(igamg_handle* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return IGAMG_ECUDA; }
  h->allocs.push_back(*p);
  return IGAMG_OK;
}

template <typename V>
int upload(igamg_handle* h, V** dst, const std::vector<V>& src) {
  int rc = dmalloc(h, (void**)dst, src.size() * sizeof(V));
  if (rc) return rc;
  CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice));
  return IGAMG_OK;
}

int launch_check() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return IGAMG_ECUDA; }
  return IGAMG_OK;
}

// ---- per-step launchers (enqueue on stream s) ------------------------------------------
int do_residual(igamg_handle* h, int l, const double* U, const double* F, double* R, double* norm2, cudaStream_t s) {
  auto& lv = h->lev[l];
  long long n = lv.sz.n_total - 1;
  unsigned nb = nblk(n);
  if (h->prob.p == 2) k_residual<2, double><<<nb, kBlock, 0, s>>>(lv.L, U, F, R, h->part);
  else k_residual<3, double><<<nb, kBlock, 0, s>>>(lv.L, U, F, R, h->part);
  k_residual_finish<double><<<1, 1024, 0, s>>>(lv.sz.n_total, F, R, h->part, (int)nb, norm2);
  return launch_check();
}

int do_smooth(igamg_handle* h, int l, double* U, const double* F, cudaStream_t s) {
  auto& lv = h->lev[l];
  const int warps_per_block = kBlock / 32;
  size_t shm = (size_t)warps_per_block * lv.maxl * sizeof(double);
  if (h->prob.smoother == IGAMG_MULT) {
    for (int c = 0; c < lv.n_colours; ++c) {
      int first = lv.colour_off[c], count = lv.colour_off[c + 1] - first;
      if (count == 0) continue;
      unsigned nb = (unsigned)((count + warps_per_block - 1) / warps_per_block);
      if (h->prob.p == 2)
        k_mult_colour<2, double><<<nb, kBlock, shm, s>>>(lv.L, U, F, lv.dofs, lv.cls, lv.cinv, lv.nloc, lv.maxl, first, count);
      else
        k_mult_colour<3, double><<<nb, kBlock, shm, s>>>(lv.L, U, F, lv.dofs, lv.cls, lv.cinv, lv.nloc, lv.maxl, first, count);
    }
  } else {
    int rc = do_residual(h, l, U, F, lv.R, nullptr, s);
    if (rc) return rc;
    unsigned nb = (unsigned)((lv.n_patches + warps_per_block - 1) / warps_per_block);
    k_add_local<double><<<nb, kBlock, shm, s>>>(lv.R, lv.dofs, lv.cls, lv.cinv, lv.nloc, lv.maxl, lv.n_patches, h->delta);
    double eta = h->prob.eta > 0 ? h->prob.eta : 0.5;
    k_add_gather<double><<<nblk(lv.sz.n_total), kBlock, 0, s>>>(lv.sz.n_total, U, h->delta, lv.d2p_off, lv.d2p_idx, eta);
  }
  return launch_check();
}

int do_restrict(igamg_handle* h, int l, const double* rf, double* gc, cudaStream_t s) {
  auto& f = h->lev[l]; auto& c = h->lev[l - 1];
  k_restrict<double><<<nblk(c.sz.n_total), kBlock, 0, s>>>(f.L, c.L, f.tp, f.tq, rf, gc);
  return launch_check();
}

int do_prolong(igamg_handle* h, int l, const double* uc, double* uf, cudaStream_t s) {
  auto& f = h->lev[l]; auto& c = h->lev[l - 1];
  k_prolong_add<double><<<nblk(f.sz.n_total), kBlock, 0, s>>>(f.L, c.L, f.tp, f.tq, uc, uf);
  return launch_check();
}

int do_coarse(igamg_handle* h, const double* G, double* U, cudaStream_t s) {
  k_coarse<double><<<1, 1024, h->ndof0 * sizeof(double), s>>>(h->ndof0, h->coarse_inv, G, U);
  return launch_check();
}

// Algorithm 1 (MGV) from the finest level, unrolled into launches.
int do_vcycle(igamg_handle* h, double* U, const double* F, cudaStream_t s) {
  const int L = (int)h->lev.size();
  if (L == 1) return do_coarse(h, F, U, s);
  int rc;
  for (int l = L - 1; l >= 1; --l) {
    double* Ul = (l == L - 1) ? U : h->lev[l].U;
    const double* Fl = (l == L - 1) ? F : h->lev[l].F;
    if (l < L - 1) CK(cudaMemsetAsync(Ul, 0, h->lev[l].sz.n_total * sizeof(double), s));
    for (int k = 0; k < h->prob.nu1; ++k) if ((rc = do_smooth(h, l, Ul, Fl, s))) return rc;
    if ((rc = do_residual(h, l, Ul, Fl, h->lev[l].R, nullptr, s))) return rc;
    if ((rc = do_restrict(h, l, h->lev[l].R, h->lev[l - 1].F, s))) return rc;
  }
  if ((rc = do_coarse(h, h->lev[0].F, h->lev[0].U, s))) return rc;
  for (int l = 1; l <= L - 1; ++l) {
    double* Ul = (l == L - 1) ? U : h->lev[l].U;
    const double* Fl = (l == L - 1) ? F : h->lev[l].F;
    if ((rc = do_prolong(h, l, h->lev[l - 1].U, Ul, s))) return rc;
    for (int k = 0; k < h->prob.nu2; ++k) if ((rc = do_smooth(h, l, Ul, Fl, s))) return rc;
  }
  return IGAMG_OK;
}

// Graph = one V-cycle followed by the fine residual norm into h->norm2.
int ensure_graph(igamg_handle* h, double* U, const double* F) {
  if (h->graph && h->gU == U && h->gF == F) return IGAMG_OK;
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int L = (int)h->lev.size();
  int rc = do_vcycle(h, U, F, h->cap_stream);
  if (!rc) rc = do_residual(h, L - 1, U, F, h->lev[L - 1].R, h->norm2, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc) { if (e == cudaSuccess) cudaGraphDestroy(g); return rc; }
  CK(e);
  cudaError_t ei = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  CK(ei);
  h->gU = U; h->gF = F;
  return IGAMG_OK;
}

int read_norm(igamg_handle* h, double* out) {
  CK(cudaMemcpyAsync(h->h_pinned, h->norm2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = std::sqrt(h->h_pinned[0]);
  return IGAMG_OK;
}

int solve_impl(igamg_handle* h, double* U, const double* F, double rtol, int max_cycles, igamg_report* rep) {
  int L = (int)h->lev.size();
  int rc = do_residual(h, L - 1, U, F, h->lev[L - 1].R, h->norm2, h->stream);
  if (rc) return rc;
  double r0;
  if ((rc = read_norm(h, &r0))) return rc;
  if (!std::isfinite(r0)) return IGAMG_ENONFINITE;
  if ((rc = ensure_graph(h, U, F))) return rc;
  int k = 0;
  double rk = r0;
  int status = IGAMG_NOT_CONVERGED;
  if (r0 == 0.0) status = IGAMG_OK;
  while (status == IGAMG_NOT_CONVERGED && k < max_cycles) {
    CK(cudaGraphLaunch(h->graph, h->stream));
    ++k;
    if ((rc = read_norm(h, &rk))) return rc;
    if (!std::isfinite(rk)) { status = IGAMG_ENONFINITE; break; }
    if (rep && rep->history && k - 1 < rep->history_cap) rep->history[k - 1] = rk / r0;
    if (rk <= rtol * r0) status = IGAMG_OK;
  }
  if (rep) {
    rep->cycles = k; rep->res0 = r0; rep->rel_residual = r0 > 0 ? rk / r0 : 0.0;
    double dv = 0.0;
    int rc2 = igamg_div_inf(h, U, &dv);
    if (rc2) return rc2;
    rep->div_inf = dv;
  }
  return status;
}

LevelDev<double> make_leveldev(const LevelHost& lh, double* bands) {
  const auto& f = lh.f;
  int n = f.n, p = f.p, q = f.q;
  size_t W = 2 * p + 1;
  LevelDev<double> L{};
  L.n = n; L.nxu = n + p - 2; L.nyu = n + q; L.npd = n + q; L.nint = n + p - 2;
  L.n_ux = lh.sz.n_ux; L.n_uy = lh.sz.n_uy; L.n_p = lh.sz.n_p; L.n_total = lh.sz.n_total;
  double* c = bands;
  L.X1 = c; c += (n + p) * W;
  L.X2 = c; c += (n + p) * W;
  L.Mq = c; c += (n + q) * W;
  L.Y2 = c; c += (n + q) * W;
  L.D = c; c += (n + p) * W;
  L.mq = c; c += (n + q);
  return L;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

const char* igamg_strerror(int code) {
  switch (code) {
    case IGAMG_OK: return "ok";
    case IGAMG_NOT_CONVERGED: return "not converged within max_cycles";
    case IGAMG_EINVAL: return "invalid argument";
    case IGAMG_EUNSUPPORTED: return "unsupported configuration";
    case IGAMG_ESINGULAR: return "singular local or coarse matrix";
    case IGAMG_ENONFINITE: return "non-finite residual norm";
    case IGAMG_ECUDA: return g_err.empty() ? "CUDA error" : g_err.c_str();
    case IGAMG_ETIMEOUT: return "timeout";
    default: return "unknown error";
  }
}

int igamg_create(const igamg_problem* prob, void* cuda_stream, igamg_handle** out) {
  if (!prob || !out) return IGAMG_EINVAL;
  *out = nullptr;
  const igamg_problem& pr = *prob;
  if (pr.dim != 2) return IGAMG_EUNSUPPORTED;
  if (pr.p != 2 && pr.p != 3) return IGAMG_EUNSUPPORTED;
  if (pr.beta_qp) return IGAMG_EUNSUPPORTED;
  if (pr.n_levels < 1 || pr.n_levels > 16 || pr.n_fine < 1) return IGAMG_EINVAL;
  if (pr.n_fine % (1 << (pr.n_levels - 1))) return IGAMG_EINVAL;
  if (!(pr.sigma > 0) || !(pr.nu > 0) || pr.nu1 < 0 || pr.nu2 < 0) return IGAMG_EINVAL;
  if (pr.smoother != IGAMG_MULT && pr.smoother != IGAMG_ADD) return IGAMG_EINVAL;
  if (pr.precision != IGAMG_FP64) return IGAMG_EUNSUPPORTED;
  if (pr.n_fine > 8192) return IGAMG_EINVAL;
  // the coarsest grid is solved with a dense inverse held in shared memory by one block
  if (level_sizes(pr.p, pr.n_fine >> (pr.n_levels - 1)).n_total > 4096) return IGAMG_EINVAL;
  auto* h = new igamg_handle();
  h->prob = pr;
  h->stream = (cudaStream_t)cuda_stream;
  int rc = build_hierarchy(pr, h->host, g_err);
  if (rc) { delete h; return rc; }
  auto fail = [&](int code) { igamg_destroy(h); return code; };
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(IGAMG_ECUDA);
  const int L = pr.n_levels, p = pr.p;
  h->lev.resize(L);
  size_t max_delta = 0;
  for (int l = 0; l < L; ++l) {
    auto& lh = h->host.lev[l];
    auto& dl = h->lev[l];
    dl.sz = lh.sz;
    const auto& f = lh.f;
    std::vector<double> bands;
    for (auto* b : {&f.X1, &f.X2, &f.Mq, &f.Y2, &f.D}) bands.insert(bands.end(), b->v.begin(), b->v.end());
    bands.insert(bands.end(), f.mq.begin(), f.mq.end());
    size_t dc_off = bands.size();
    bands.insert(bands.end(), f.dcoef.begin(), f.dcoef.end());
    if ((rc = upload(h, &dl.bands, bands))) return fail(rc);
    dl.L = make_leveldev(lh, dl.bands);
    dl.dcoef = dl.bands + dc_off;
    if (l >= 1) {
      const auto& pt = lh.pt;
      dl.n_patches = pt.n_patches; dl.maxl = pt.maxl; dl.n_colours = pt.n_colours;
      dl.colour_off = pt.colour_off;
      if ((rc = upload(h, &dl.dofs, pt.dofs))) return fail(rc);
      if ((rc = upload(h, &dl.cls, pt.cls))) return fail(rc);
      if ((rc = upload(h, &dl.nloc, pt.nloc))) return fail(rc);
      if ((rc = upload(h, &dl.cinv, pt.cinv))) return fail(rc);
      if ((rc = upload(h, &dl.d2p_off, pt.d2p_off))) return fail(rc);
      if ((rc = upload(h, &dl.d2p_idx, pt.d2p_idx))) return fail(rc);
      max_delta = std::max(max_delta, (size_t)pt.n_patches * pt.maxl);
      for (int which = 0; which < 2; ++which) {
        const Transfer1D& T = which ? h->host.tq[l] : h->host.tp_free[l];
        XferDev& X = which ? dl.tq : dl.tp;
        int *c0, *f0; double *pv, *rv;
        if ((rc = upload(h, &c0, T.c0)) || (rc = upload(h, &f0, T.f0)) || (rc = upload(h, &pv, T.pv)) || (rc = upload(h, &rv, T.rv))) return fail(rc);
        X.nf = T.nf; X.nc = T.nc; X.c0 = c0; X.f0 = f0; X.pv = pv; X.rv = rv;
      }
    }
    size_t nb = (size_t)dl.sz.n_total * sizeof(double);
    if ((rc = dmalloc(h, (void**)&dl.R, nb))) return fail(rc);
    if (l < L - 1) {
      if ((rc = dmalloc(h, (void**)&dl.U, nb))) return fail(rc);
      if ((rc = dmalloc(h, (void**)&dl.F, nb))) return fail(rc);
    }
  }
  h->ndof0 = h->host.ndof0;
  if ((rc = upload(h, &h->coarse_inv, h->host.coarse_inv))) return fail(rc);
  long long nfine = h->lev[L - 1].sz.n_total;
  if ((rc = dmalloc(h, (void**)&h->part, 2 * sizeof(double) * (nblk(nfine) + 1)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->norm2, sizeof(double)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->divmax, sizeof(unsigned long long)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->delta, std::max<size_t>(max_delta, 1) * sizeof(double)))) return fail(rc);
  if ((rc = upload(h, &h->lv_p, h->host.lv_p))) return fail(rc);
  if ((rc = upload(h, &h->lv_q, h->host.lv_q))) return fail(rc);
  size_t nG = (size_t)pr.n_fine * (p + 2);
  if ((rc = dmalloc(h, (void**)&h->f_dev, 2 * nG * nG * sizeof(double)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->Fh, nfine * sizeof(double)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->Uh, nfine * sizeof(double)))) return fail(rc);
  if (cudaMallocHost((void**)&h->h_pinned, 2 * sizeof(double)) != cudaSuccess) return fail(IGAMG_ECUDA);
  *out = h;
  return IGAMG_OK;
}

void igamg_destroy(igamg_handle* h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

int igamg_get_sizes(const igamg_handle* h, int level, igamg_sizes* out) {
  if (!h || !out || level < 0 || level >= (int)h->lev.size()) return IGAMG_EINVAL;
  *out = h->lev[level].sz;
  return IGAMG_OK;
}

int igamg_quad_points(const igamg_handle* h, double* x, size_t cap, size_t* n_out) {
  if (!h || !n_out) return IGAMG_EINVAL;
  *n_out = h->host.quad_x.size();
  if (x) {
    if (cap < h->host.quad_x.size()) return IGAMG_EINVAL;
    std::memcpy(x, h->host.quad_x.data(), h->host.quad_x.size() * sizeof(double));
  }
  return IGAMG_OK;
}

int igamg_load_vector(igamg_handle* h, const double* f_qp, double* F) {
  if (!h || !f_qp || !F) return IGAMG_EINVAL;
  auto& lv = h->lev.back();
  if (h->prob.p == 2) k_load<2><<<nblk(lv.sz.n_total), kBlock, 0, h->stream>>>(lv.L, h->lv_p, h->lv_q, f_qp, F);
  else k_load<3><<<nblk(lv.sz.n_total), kBlock, 0, h->stream>>>(lv.L, h->lv_p, h->lv_q, f_qp, F);
  return launch_check();
}

int igamg_residual(igamg_handle* h, int level, const double* U, const double* F, double* R, double* norm_out) {
  if (!h || !U || !F || !R || level < 0 || level >= (int)h->lev.size()) return IGAMG_EINVAL;
  int rc = do_residual(h, level, U, F, R, h->norm2, h->stream);
  if (rc) return rc;
  if (norm_out) return read_norm(h, norm_out);
  return IGAMG_OK;
}

int igamg_smooth(igamg_handle* h, int level, double* U, const double* F, int sweeps) {
  if (!h || !U || !F || level < 1 || level >= (int)h->lev.size() || sweeps < 0) return IGAMG_EINVAL;
  for (int k = 0; k < sweeps; ++k) { int rc = do_smooth(h, level, U, F, h->stream); if (rc) return rc; }
  return IGAMG_OK;
}

int igamg_restrict(igamg_handle* h, int level, const double* r_fine, double* g_coarse) {
  if (!h || !r_fine || !g_coarse || level < 1 || level >= (int)h->lev.size()) return IGAMG_EINVAL;
  return do_restrict(h, level, r_fine, g_coarse, h->stream);
}

int igamg_prolong_add(igamg_handle* h, int level, const double* u_coarse, double* u_fine) {
  if (!h || !u_coarse || !u_fine || level < 1 || level >= (int)h->lev.size()) return IGAMG_EINVAL;
  return do_prolong(h, level, u_coarse, u_fine, h->stream);
}

int igamg_coarse_solve(igamg_handle* h, const double* G, double* U) {
  if (!h || !G || !U) return IGAMG_EINVAL;
  return do_coarse(h, G, U, h->stream);
}

int igamg_vcycle(igamg_handle* h, double* U, const double* F) {
  if (!h || !U || !F) return IGAMG_EINVAL;
  int rc = ensure_graph(h, U, F);
  if (rc) return rc;
  CK(cudaGraphLaunch(h->graph, h->stream));
  return IGAMG_OK;
}

int igamg_solve(igamg_handle* h, double* U, const double* F, double rtol, int max_cycles, igamg_report* rep) {
  if (!h || !U || !F || !(rtol >= 0) || max_cycles < 0) return IGAMG_EINVAL;
  return solve_impl(h, U, F, rtol, max_cycles, rep);
}

int igamg_solve_host(igamg_handle* h, const double* f_qp_host, double* U_host, double rtol, int max_cycles,
                     igamg_report* rep) {
  if (!h || !f_qp_host || !U_host || !(rtol >= 0) || max_cycles < 0) return IGAMG_EINVAL;
  size_t nG = (size_t)h->prob.n_fine * (h->prob.p + 2);
  size_t nt = (size_t)h->lev.back().sz.n_total;
  CK(cudaMemcpyAsync(h->f_dev, f_qp_host, 2 * nG * nG * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->Uh, U_host, nt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  int rc = igamg_load_vector(h, h->f_dev, h->Fh);
  if (rc) return rc;
  int st = solve_impl(h, h->Uh, h->Fh, rtol, max_cycles, rep);
  if (st < 0) return st;
  CK(cudaMemcpyAsync(U_host, h->Uh, nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return st;
}

int igamg_div_inf(igamg_handle* h, const double* U, double* out) {
  if (!h || !U || !out) return IGAMG_EINVAL;
  auto& lv = h->lev.back();
  CK(cudaMemsetAsync(h->divmax, 0, sizeof(unsigned long long), h->stream));
  k_div_inf<<<nblk(lv.sz.n_p), kBlock, 0, h->stream>>>(lv.L, lv.dcoef, U, h->divmax);
  int rc = launch_check();
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->h_pinned, h->divmax, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = h->h_pinned[0];
  return IGAMG_OK;
}

int igamg_curl(igamg_handle* h, const double* psi, double* U) {
  if (!h || !psi || !U) return IGAMG_EINVAL;
  auto& lv = h->lev.back();
  k_curl<<<nblk(lv.sz.n_ux + lv.sz.n_uy), kBlock, 0, h->stream>>>(lv.L, lv.dcoef, psi, U);
  return launch_check();
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Residual entry point that allocates no device memory.
//
// For callers that cannot call cudaMalloc (a host program whose allocations all go
// through its own pool or arena, code running inside a captured region that forbids new
// allocations, or an embedding that owns the whole device memory budget): the scratch
// of the residual kernel -- its level operator tables and its per-block partial sums --
// lives in one fixed array in device memory that the library declares statically.
// Every GPU that loads the library holds that array (1 MiB) until the process exits.
// ---------------------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchDoubles = 131072;  // 1 MiB
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_static_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int igamg_residual_static(const igamg_problem* prob, int level, const double* U,
                                     const double* F, double* R, double* norm_out,
                                     void* cuda_stream) {
  if (!prob || !U || !F || !R) return IGAMG_EINVAL;
  const igamg_problem& pr = *prob;
  if (pr.dim != 2 || (pr.p != 2 && pr.p != 3) || pr.beta_qp) return IGAMG_EUNSUPPORTED;
  if (pr.n_levels < 1 || pr.n_levels > 16 || pr.n_fine < 1 || pr.n_fine > 8192) return IGAMG_EINVAL;
  if (pr.n_fine % (1 << (pr.n_levels - 1))) return IGAMG_EINVAL;
  if (level < 0 || level >= pr.n_levels || !(pr.sigma > 0) || !(pr.nu > 0)) return IGAMG_EINVAL;
  const int p = pr.p, n = pr.n_fine >> (pr.n_levels - 1 - level);
  cudaStream_t s = (cudaStream_t)cuda_stream;

  // size check before any work: band tables + partials + the norm slot
  igamg_sizes sz = level_sizes(p, n);
  const size_t W = 2 * p + 1;
  const size_t n_bands = (size_t)(n + p) * W * 3 + (size_t)(n + p - 1) * W * 2 + (n + p - 1);
  const unsigned nb = nblk(sz.n_total - 1);
  const size_t need = n_bands + 2 * (size_t)nb + 1;
  if (need > kStaticScratchDoubles) {
    g_err = "igamg_residual_static: level needs " + std::to_string(need) + " doubles of scratch, the static array holds " +
            std::to_string(kStaticScratchDoubles);
    std::fprintf(stderr, "igamg: %s\n", g_err.c_str());
    return IGAMG_EINVAL;
  }
  // one-time set-up per device: the device address of the static array
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return IGAMG_EUNSUPPORTED;
  if (!g_static_ptr[dev]) {
    double* ptr = nullptr;
    CK(cudaGetSymbolAddress((void**)&ptr, g_static_scratch));
    g_static_ptr[dev] = ptr;
  }
  double* scratch = g_static_ptr[dev];

  // level operator tables (host), copied into the front of the static array
  Level1D f;
  const double cpen = pr.c_penalty > 0 ? pr.c_penalty : 4.0 * (p - 1);
  build_level1d(p, n, pr.sigma, pr.nu, cpen * pr.n_fine, f);
  std::vector<double> bands;
  bands.reserve(n_bands);
  for (auto* b : {&f.X1, &f.X2, &f.Mq, &f.Y2, &f.D}) bands.insert(bands.end(), b->v.begin(), b->v.end());
  bands.insert(bands.end(), f.mq.begin(), f.mq.end());
  if (bands.size() != n_bands) return IGAMG_EINVAL;
  CK(cudaMemcpyAsync(scratch, bands.data(), n_bands * sizeof(double), cudaMemcpyHostToDevice, s));
  LevelHost lh;
  lh.f = f;
  lh.sz = sz;
  LevelDev<double> L = make_leveldev(lh, scratch);
  double* part = scratch + n_bands;       // fully rewritten by every call
  double* norm2 = part + 2 * (size_t)nb;
  if (p == 2) k_residual<2, double><<<nb, kBlock, 0, s>>>(L, U, F, R, part);
  else k_residual<3, double><<<nb, kBlock, 0, s>>>(L, U, F, R, part);
  k_residual_finish<double><<<1, 1024, 0, s>>>(sz.n_total, F, R, part, (int)nb, norm2);
  int rc = launch_check();
  if (rc) return rc;
  if (norm_out) {
    double v = 0.0;
    CK(cudaMemcpyAsync(&v, norm2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *norm_out = std::sqrt(v);
  }
  return IGAMG_OK;
}
