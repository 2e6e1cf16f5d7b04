// C ABI and launch orchestration of the geometric multigrid V-cycle (arXiv 1705.09282,
// Algorithm 1 with the overlapping Schwarz smoothers of Sec. 5.2), for sm_103a.
//
// Generalized Stokes levels on the square apply their operator matrix-free from class
// stencils built from the 1D factors (setup.cpp); generalized Oseen and mapped levels read one
// stored record per row, and the finest Oseen residual may apply its advection term element
// by element instead (kernels_adv.cuh; the faster form per precision is kept at creation).
// The multiplicative smoother runs one launch per patch colour (or a pipelined tile sweep,
// per level as the autotuner chose): inside a colour the patches share no degree of freedom
// and are not coupled by K, so solving them concurrently is the same as solving them one
// after another (eq. MSM).  A V-cycle (and, in the FP32 mode, one step of FP64 iterative
// refinement around an FP32 V-cycle) is captured once into a CUDA graph and replayed;
// independent solves step either in lockstep launches or each on its own stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "igamg3d.h"
#include "igamg_internal.h"
#include "kernels.cuh"
#include "kernels_adv.cuh"
#include "krylov.h"

using namespace igamg;
using namespace igamg::dev;

namespace {

constexpr int kBlock = 256;
inline unsigned nblk(long long n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

// max |div u| over the (n+q)^2 pressure-space coefficients (order-free max via bits).
__global__ void k_div_inf(LevelTab<double> L, const double* __restrict__ dcoef, const double* __restrict__ U,
                          unsigned long long* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (k < L.n_p) {
    int ky = k / L.npd, kx = k - ky * L.npd;
    const double* ux = U;
    const double* uy = U + L.n_ux;
    auto UX = [&](int ix, int iy) { return (ix < 1 || ix > L.nint) ? 0.0 : ux[iy * L.nxu + ix - 1]; };
    auto UY = [&](int ix, int iy) { return (iy < 1 || iy > L.nint) ? 0.0 : uy[(iy - 1) * L.npd + ix]; };
    double c = dcoef[kx] * (UX(kx + 1, ky) - UX(kx, ky)) + dcoef[ky] * (UY(kx, ky + 1) - UY(kx, ky));
    v = fabs(c);
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// Streamfunction of a (divergence-free) velocity by integration of its u_x block along y:
// psi(ix, k+1) = psi(ix, k) + u_x(ix, k) / dcoef_k, psi = 0 on the bottom wall; one warp
// per interior column (lane runs, then a warp scan), FP64.
__global__ void k_streamfunction(int nint, int nxu, const double* __restrict__ inv_dcoef, const double* __restrict__ U,
                                 double* __restrict__ psi) {
  int ix = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (ix >= nint) return;
  int per = (nint + 31) / 32;
  int k0 = lane * per, k1 = min(k0 + per, nint);
  double run = 0.0;
  for (int k = k0; k < k1; ++k) run = fma(U[k * nxu + ix], inv_dcoef[k], run);
  double incl = run;
  for (int o = 1; o < 32; o <<= 1) {
    double v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  double acc = incl - run;
  for (int k = k0; k < k1; ++k) {
    acc = fma(U[k * nxu + ix], inv_dcoef[k], acc);
    psi[k * nint + ix] = acc;
  }
}

// psi (interior, FP64) = scale * grid[1..H-2, 1..W-2] of a network output grid (H = W = n+p).
__global__ void k_grid_to_psi(int nint, const float* __restrict__ grid, double scale, double* __restrict__ psi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nint * nint) return;
  int y = i / nint, x = i - y * nint;
  psi[i] = scale * (double)grid[(y + 1) * (nint + 2) + x + 1];
}

// pressure coefficients (npd x npd) = scale * grid[0..npd-1, 0..npd-1] of an H x H grid.
__global__ void k_grid_to_pressure(int npd, const float* __restrict__ grid, int H, double scale,
                                   double* __restrict__ pr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npd * npd) return;
  int y = i / npd, x = i - y * npd;
  pr[i] = scale * (double)grid[y * H + x];
}

// Five dot products x_k . y_k at once (grid-stride, fixed-order block partials part[k][b]).
constexpr int kDotGrid = 304;
__global__ void __launch_bounds__(256) k_dots5(int n, const double* __restrict__ x0, const double* __restrict__ y0,
                                               const double* __restrict__ x1, const double* __restrict__ y1,
                                               const double* __restrict__ x2, const double* __restrict__ y2,
                                               const double* __restrict__ x3, const double* __restrict__ y3,
                                               const double* __restrict__ x4, const double* __restrict__ y4,
                                               double* __restrict__ part) {
  __shared__ double sh[32];
  double s[5] = {0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    s[0] = fma(x0[i], y0[i], s[0]); s[1] = fma(x1[i], y1[i], s[1]); s[2] = fma(x2[i], y2[i], s[2]);
    s[3] = fma(x3[i], y3[i], s[3]); s[4] = fma(x4[i], y4[i], s[4]);
  }
  for (int k = 0; k < 5; ++k) {
    double t = block_sum(s[k], sh);
    if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_dots5_finish(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x >= 5) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += part[threadIdx.x * nb + b];
  out[threadIdx.x] = t;
}

// mapped domains: the parametric load J^T f at every quadrature point (f and fh may alias)
__global__ void k_pullback(int npts, const double* __restrict__ jt, const double* f, double* fh) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const double fx = f[i], fy = f[npts + i];
  const double* t = jt + (size_t)4 * i;              // t[2k + c] = dX_c / dxi_k
  fh[i] = t[0] * fx + t[1] * fy;
  fh[npts + i] = t[2] * fx + t[3] * fy;
}

// U = a U + b Z
__global__ void k_axpby(int n, double a, double b, const double* __restrict__ Z, double* __restrict__ U) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) U[i] = a * U[i] + b * Z[i];
}

// velocity = curl psi, psi on the (n+p-2)^2 interior streamfunction coefficients.
__global__ void k_curl(LevelTab<double> L, const double* __restrict__ dcoef, const double* __restrict__ psi,
                       double* __restrict__ U) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_ux + L.n_uy) return;
  int ni = L.nint;
  auto PS = [&](int ix, int iy) { return (ix < 1 || ix > ni || iy < 1 || iy > ni) ? 0.0 : psi[(iy - 1) * ni + ix - 1]; };
  if (g < L.n_ux) {
    int ky = g / L.nxu, ix = g - ky * L.nxu + 1;
    U[g] = dcoef[ky] * (PS(ix, ky + 1) - PS(ix, ky));
  } else {
    int r = g - L.n_ux;
    int iy = r / L.npd + 1, kx = r - (iy - 1) * L.npd;
    U[g] = -dcoef[kx] * (PS(kx + 1, iy) - PS(kx, iy));
  }
}

// F = (int v.f, 0, 0) on the finest level; tables hold weight * basis value per local element.
template <int P>
__global__ void k_load(LevelTab<double> L, const double* __restrict__ lvp, const double* __restrict__ lvq,
                       const double* __restrict__ f, double* __restrict__ F) {
  constexpr int Q = P - 1, G = P + 2;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_total) return;
  if (g >= L.n_ux + L.n_uy) { F[g] = 0.0; return; }
  int n = L.n, nG = n * G;
  int ix, iy, dxg, dyg;
  const double *tx, *ty, *fc;
  if (g < L.n_ux) { iy = g / L.nxu; ix = g - iy * L.nxu + 1; dxg = P; dyg = Q; tx = lvp; ty = lvq; fc = f; }
  else { int r = g - L.n_ux; iy = r / L.npd + 1; ix = r - (iy - 1) * L.npd; dxg = Q; dyg = P; tx = lvq; ty = lvp; fc = f + (size_t)nG * nG; }
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

template <typename T>
struct TypedLevel {
  LevelTab<T> L{};
  T* cinv = nullptr;
  T* cinv8 = nullptr;
  Xfer<T> tp{}, tq{};            // transfer from level l-1 into level l (l >= 1)
  T *U = nullptr, *F = nullptr, *R = nullptr;
  unsigned* prog = nullptr;      // pipelined sweep: colour steps finished per tile
};

template <typename T>
struct Typed {
  std::vector<TypedLevel<T>> lev;
  T* coarse_inv = nullptr;
  T* delta = nullptr;
  int fused_lc = -1;            // levels 0..fused_lc run in one launch, or -1 (per-level launches)
  int fused_kind = 1;           // 1: one block (k_fused_coarse); C > 1: one cluster of C blocks
  int fused_max = -1;           // deepest feasible one-block choice (descriptor is built for it)
  size_t fused_smem = 0;
  FusedDesc<T> fused{};
  int cluster_max = -1;         // deepest feasible cluster choice
  size_t cluster_smem = 0;
  ClusterDesc<T> cdesc{};
  AdvTab<T> adv{};              // generalized Oseen on the square: matrix-free advection tables
  int adv_mf = 0;               // 1: the finest level's residual applies the advection matrix-free
};

struct LevelCommon {
  igamg_sizes sz{};
  int n_patches = 0, maxl = 0, n_colours = 0;
  std::vector<int> colour_off, n8;
  int *dofs = nullptr, *cls = nullptr, *nloc = nullptr, *d2p_off = nullptr, *d2p_idx = nullptr;
  double* dcoef = nullptr;      // derivative coefficients (n+p-1), device
  double* inv_dcoef = nullptr;  // their reciprocals
  // pipelined multiplicative sweep (k_sweep_tiles): tiles of tw x tw patch positions, or
  // ntx = 0 where the level uses one launch per colour
  int tw = 0, ntx = 0, nty = 0;
  int *tile_list = nullptr, *tile_off = nullptr, *tile_n8 = nullptr;
  int lpr = 1;                  // lanes per local row of an 8-DOF patch in the colour kernels
  int tpb = 0;                  // threads per block of the colour kernels (0: colour_block())
  int ch = 4;                   // multiply-add chains per row in the one-lane FP64 colour kernel (4 or 2;
                                // the FP32 kernels, latency-bound, keep 4)
};

}  // namespace

// Workspace and captured graphs of one lockstep batch (a fixed list of handles and vectors).
struct BatchCache {
  // creation serials of the handles, then the U and F addresses of every solve (serials, not
  // handle addresses: a handle destroyed and re-created at the same address must not match)
  std::vector<unsigned long long> key;
  int count = 0;
  int* flags = nullptr;                // device: 1 while a solve is active
  double* norms = nullptr;             // device: ||F - K U||^2 per solve
  int* h_flags = nullptr;              // pinned host copies
  double* h_norms = nullptr;
  cudaStream_t stream = nullptr;       // the batch's own stream (the graphs fork from it)
  cudaEvent_t ev = nullptr;
  std::vector<cudaStream_t> side;      // capture streams of the branches after the first
  std::vector<cudaEvent_t> side_ev;
  std::vector<MixLevel<double>> mix;   // descriptors, solve-major, nd depths per solve
  int nd = 0;                          // depths: the most grids of any solve
  std::vector<std::vector<int>> branch;  // solve indices of each branch (at most kMixChunk)
  cudaGraphExec_t g_res = nullptr;     // residual norms of all active solves
  cudaGraphExec_t g_cycle = nullptr;   // one V-cycle, then the residual norms
};

static unsigned long long next_serial() {
  static std::atomic<unsigned long long> counter{0};
  return ++counter;
}

static void batch_cache_free(BatchCache* c) {
  if (!c) return;
  if (c->g_res) cudaGraphExecDestroy(c->g_res);
  if (c->g_cycle) cudaGraphExecDestroy(c->g_cycle);
  if (c->flags) cudaFree(c->flags);
  if (c->norms) cudaFree(c->norms);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->h_norms) cudaFreeHost(c->h_norms);
  for (auto st : c->side) cudaStreamDestroy(st);
  for (auto e : c->side_ev) cudaEventDestroy(e);
  if (c->ev) cudaEventDestroy(c->ev);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

struct igamg_handle {
  igamg_problem prob{};
  HierarchyHost host;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  std::vector<LevelCommon> lc;
  Typed<double> d;
  Typed<float> f;
  int ndof0 = 0;
  double* part = nullptr;      // residual partials (2 per block of the finest level)
  double* norm2 = nullptr;     // device: [0] squared residual norm, [1] holds the sweep
                               // timeout flag (an int in its first four bytes)
  int* sweep_err = nullptr;    // = (int*)(norm2 + 1): read back with the norm
  int stall_tile = -1;         // IGAMG_TEST_STALL_TILE: a tile that never reports progress,
                               // to exercise the sweep's timeout path in tests
  unsigned long long* divmax = nullptr;
  double *lv_p = nullptr, *lv_q = nullptr;
  double* h_pinned = nullptr;  // 2 doubles
  double *f_dev = nullptr, *Fh = nullptr, *Uh = nullptr;   // host-buffer solve workspaces
  double* psi = nullptr;       // FP32 mode: streamfunction of the correction (fine interior)
  // captured graphs: [0] solve step, [1] public V-cycle (starts with the residual in FP32 mode)
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  const void* gU[3] = {nullptr, nullptr, nullptr};
  const void* gF[3] = {nullptr, nullptr, nullptr};
  std::vector<void*> allocs;
  cudaStream_t exec_stream = nullptr;  // used by igamg_solve_batch
  cudaEvent_t ev = nullptr;
  igamg3d_handle* d3 = nullptr;        // dim = 3: everything lives in the 3D driver
  KrylovWork kw;                       // FGMRES modes
  double* zeros = nullptr;             // a zero right-hand side (K z = -(0 - K z))
  double* jt = nullptr;                // mapped domains: J^T at the finest quadrature points
  double* dots = nullptr;              // warm-start scalings: 5 x kDotGrid partials, then 5 sums
  BatchCache* bc = nullptr;            // lockstep batches led by this handle (igamg_solve_batch)
  unsigned long long serial = next_serial();   // unique per handle created in this process
};

namespace {

thread_local std::string g_err;

}  // namespace

void igamg::set_error(const std::string& msg) { g_err = msg; }

namespace {

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { g_err = std::string(#x) + ": " + cudaGetErrorString(e_); return IGAMG_ECUDA; } } while (0)

int dmalloc(igamg_handle* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return IGAMG_ECUDA; }
  h->allocs.push_back(*p);
  return IGAMG_OK;
}

template <typename V, typename S>
int upload_as(igamg_handle* h, V** dst, const std::vector<S>& src) {
  std::vector<V> tmp(src.begin(), src.end());
  int rc = dmalloc(h, (void**)dst, tmp.size() * sizeof(V));
  if (rc) return rc;
  CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(V), cudaMemcpyHostToDevice));
  return IGAMG_OK;
}

int launch_check() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return IGAMG_ECUDA; }
  return IGAMG_OK;
}

// Threads per block of the colour kernel: 128 (default; a colour's blocks then spread evenly
// over the 152 SMs: ~455 blocks of 16 patches on a 256^2 level instead of ~228 of 32), or
// IGAMG_COLOUR_BLOCK = 32 .. 256.
int colour_block() {
  static const int tpb = [] {
    const char* e = std::getenv("IGAMG_COLOUR_BLOCK");
    int v = e ? std::atoi(e) : 128;
    return (v >= 32 && v <= 256 && v % 32 == 0) ? v : 128;   // launch bounds: 256
  }();
  return tpb;
}

// Colour kernel form: one lane per row (k_mult_colour, default) or split rows
// (k_mult_colour_split, IGAMG_SPLIT_COLOUR=1; measured 10 % slower on the 256^2 sweep).
// Per-row operator records (Oseen) always use the former.
bool split_colour(bool per_row_records) {
  static const int mode = [] {
    const char* e = std::getenv("IGAMG_SPLIT_COLOUR");
    return e ? std::atoi(e) : 0;
  }();
  return mode == 1 && !per_row_records;
}

// FP32 V-cycles (refinement step or FGMRES preconditioner) on this handle
bool fp32_base(const igamg_problem& pr) {
  return pr.precision == IGAMG_FP32_IR || pr.precision == IGAMG_FGMRES_FP32;
}

template <typename T> Typed<T>& typed(igamg_handle* h);
template <> Typed<double>& typed<double>(igamg_handle* h) { return h->d; }
template <> Typed<float>& typed<float>(igamg_handle* h) { return h->f; }

// ---- per-step launchers (enqueue on stream s) ------------------------------------------
// Tiles of the matrix-free Oseen residual (k_residual_adv) on a level of n elements.
int adv_tiles_x(int p, int n) {
  const int te = p == 2 ? AdvShape<2>::TE : AdvShape<3>::TE;
  return (n + p - 1 + te - 1) / te;
}

template <typename T>
int do_residual(igamg_handle* h, int l, const T* U, const T* F, T* R, double* norm2, cudaStream_t s) {
  auto& ty = typed<T>(h);
  auto& L = ty.lev[l].L;
  if (ty.adv_mf && l == (int)ty.lev.size() - 1) {
    LevelTab<T> Ls = L;
    Ls.srow = nullptr;                     // the Stokes part from the class stencils
    const int tx = adv_tiles_x(h->prob.p, L.n);
    const unsigned nb = (unsigned)(tx * tx);
    if (h->prob.p == 2)
      k_residual_adv<2, T><<<nb, kAdvThreads, AdvShape<2>::smem<T>(), s>>>(Ls, ty.adv, U, F, R, h->part, tx);
    else
      k_residual_adv<3, T><<<nb, kAdvThreads, AdvShape<3>::smem<T>(), s>>>(Ls, ty.adv, U, F, R, h->part, tx);
    k_residual_finish<T><<<1, 1024, 0, s>>>(L.n_total, F, R, h->part, (int)nb, norm2);
    return launch_check();
  }
  unsigned nb = nblk(L.n_total - 1);
  if (h->prob.p == 2) k_residual<2, T><<<nb, kBlock, 0, s>>>(L, U, F, R, h->part);
  else k_residual<3, T><<<nb, kBlock, 0, s>>>(L, U, F, R, h->part);
  k_residual_finish<T><<<1, 1024, 0, s>>>(L.n_total, F, R, h->part, (int)nb, norm2);
  return launch_check();
}

template <typename T>
int do_smooth(igamg_handle* h, int l, T* U, const T* F, cudaStream_t s) {
  auto& lc = h->lc[l];
  auto& tl = typed<T>(h).lev[l];
  size_t shm = (size_t)(kBlock / 32) * lc.maxl * sizeof(T);
  if (h->prob.smoother == IGAMG_MULT && split_colour(tl.L.srow != nullptr)) {
    size_t shm16 = (size_t)16 * lc.maxl * sizeof(T);
    for (int c = 0; c < lc.n_colours; ++c) {
      int first = lc.colour_off[c], count = lc.colour_off[c + 1] - first;
      if (count == 0) continue;
      int n8 = lc.n8[c], ngen = count - n8;
      int nb8 = (n8 + 31) / 32, nbg = (ngen + 15) / 16;
      unsigned nb = (unsigned)(nb8 + nbg);
      if (h->prob.p == 2)
        k_mult_colour_split<2, T><<<nb, 512, shm16, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
      else
        k_mult_colour_split<3, T><<<nb, 512, shm16, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
    }
  } else if (h->prob.smoother == IGAMG_MULT) {
    const int tpb = lc.tpb > 0 ? lc.tpb : colour_block(), wpb = tpb / 32;
    const size_t shmc = (size_t)wpb * lc.maxl * sizeof(T);
    const int ppw = lc.lpr == 2 ? 2 : 4;            // 8-DOF patches per warp
    for (int c = 0; c < lc.n_colours; ++c) {
      int first = lc.colour_off[c], count = lc.colour_off[c + 1] - first;
      if (count == 0) continue;
      int n8 = lc.n8[c], ngen = count - n8;
      int nb8 = (n8 + ppw * wpb - 1) / (ppw * wpb), nbg = (ngen + wpb - 1) / wpb;
      unsigned nb = (unsigned)(nb8 + nbg);
      if (h->prob.p == 2) {
        if (lc.lpr == 2)
          k_mult_colour<2, T, 2><<<nb, tpb, shmc, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
        else if (lc.ch == 2 && sizeof(T) == 8)
          k_mult_colour<2, T, 1, 2><<<nb, tpb, shmc, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
        else
          k_mult_colour<2, T><<<nb, tpb, shmc, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
      } else {
        if (lc.lpr == 2)
          k_mult_colour<3, T, 2><<<nb, tpb, shmc, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
        else if (lc.ch == 2 && sizeof(T) == 8)
          k_mult_colour<3, T, 1, 2><<<nb, tpb, shmc, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
        else
          k_mult_colour<3, T><<<nb, tpb, shmc, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
      }
    }
  } else {
    int rc = do_residual<T>(h, l, U, F, tl.R, nullptr, s);
    if (rc) return rc;
    unsigned nb = (unsigned)((lc.n_patches + kBlock / 32 - 1) / (kBlock / 32));
    if (h->prob.p == 2)
      k_add_local<2, T><<<nb, kBlock, shm, s>>>(tl.R, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, lc.n_patches, typed<T>(h).delta);
    else
      k_add_local<3, T><<<nb, kBlock, shm, s>>>(tl.R, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, lc.n_patches, typed<T>(h).delta);
    T eta = (T)(h->prob.eta > 0 ? h->prob.eta : 0.3);
    k_add_gather<T><<<nblk(lc.sz.n_total), kBlock, 0, s>>>((int)lc.sz.n_total, U, typed<T>(h).delta, lc.d2p_off, lc.d2p_idx, eta);
  }
  return launch_check();
}

// Threads per block of the pipelined sweep (tiled levels; a level that is one tile runs in
// one block of kSoloThreads) and the dynamic shared memory of its wall patches.
constexpr int kTileThreads = 128, kSoloThreads = 512;
template <typename T>
size_t tile_smem(int maxl, int threads = kTileThreads) { return (size_t)(threads / 32) * maxl * sizeof(T); }

// Pipelined multiplicative sweep (k_sweep_tiles): all colours of `sweeps` sweeps in one
// cooperative launch, one block per tile.
template <typename T>
int do_sweep_tiles(igamg_handle* h, int l, T* U, const T* F, int sweeps, cudaStream_t s) {
  auto& lc = h->lc[l];
  auto& tl = typed<T>(h).lev[l];
  TileSched ts{lc.ntx, lc.nty, lc.n_colours, lc.tile_list, lc.tile_off, lc.tile_n8, tl.prog, h->sweep_err,
               h->stall_tile};
  const bool solo = lc.ntx * lc.nty == 1;
  const int nthr = solo ? kSoloThreads : kTileThreads;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(lc.ntx * lc.nty));
  cfg.blockDim = dim3(nthr);
  cfg.dynamicSmemBytes = tile_smem<T>(lc.maxl, nthr);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int steps = sweeps * lc.n_colours;
  const T* ci = tl.cinv;
  const T* ci8 = tl.cinv8;
  const int* nloc = lc.nloc;
  cudaError_t e;
  if (h->prob.p == 2)
    e = solo ? cudaLaunchKernelEx(&cfg, k_sweep_tiles<2, T, kSoloThreads>, tl.L, U, F, (const int*)lc.dofs,
                                  (const int*)lc.cls, ci, ci8, nloc, lc.maxl, ts, steps)
             : cudaLaunchKernelEx(&cfg, k_sweep_tiles<2, T, kTileThreads>, tl.L, U, F, (const int*)lc.dofs,
                                  (const int*)lc.cls, ci, ci8, nloc, lc.maxl, ts, steps);
  else
    e = solo ? cudaLaunchKernelEx(&cfg, k_sweep_tiles<3, T, kSoloThreads>, tl.L, U, F, (const int*)lc.dofs,
                                  (const int*)lc.cls, ci, ci8, nloc, lc.maxl, ts, steps)
             : cudaLaunchKernelEx(&cfg, k_sweep_tiles<3, T, kTileThreads>, tl.L, U, F, (const int*)lc.dofs,
                                  (const int*)lc.cls, ci, ci8, nloc, lc.maxl, ts, steps);
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return IGAMG_ECUDA; }
  return IGAMG_OK;
}

// nu sweeps of the level's smoother: one pipelined launch where the level has a tile
// schedule (multiplicative smoother), else one do_smooth per sweep.
template <typename T>
int do_smooth_n(igamg_handle* h, int l, T* U, const T* F, int sweeps, cudaStream_t s) {
  if (sweeps <= 0) return IGAMG_OK;
  if (h->prob.smoother == IGAMG_MULT && h->lc[l].ntx > 0) return do_sweep_tiles<T>(h, l, U, F, sweeps, s);
  for (int k = 0; k < sweeps; ++k) {
    int rc = do_smooth<T>(h, l, U, F, s);
    if (rc) return rc;
  }
  return IGAMG_OK;
}

template <typename T>
int do_restrict(igamg_handle* h, int l, const T* rf, T* gc, cudaStream_t s) {
  auto& f = typed<T>(h).lev[l];
  auto& c = typed<T>(h).lev[l - 1];
  k_restrict<T><<<nblk(c.L.n_total), kBlock, 0, s>>>(f.L, c.L, f.tp, f.tq, rf, gc);
  return launch_check();
}

template <typename T>
int do_prolong(igamg_handle* h, int l, const T* uc, T* uf, cudaStream_t s) {
  auto& f = typed<T>(h).lev[l];
  auto& c = typed<T>(h).lev[l - 1];
  k_prolong_add<T><<<nblk(f.L.n_total), kBlock, 0, s>>>(f.L, c.L, f.tp, f.tq, uc, uf);
  return launch_check();
}

template <typename T>
int do_coarse(igamg_handle* h, const T* G, T* U, cudaStream_t s) {
  k_coarse<T><<<1, 1024, h->ndof0 * sizeof(T), s>>>(h->ndof0, typed<T>(h).coarse_inv, G, U);
  return launch_check();
}

template <typename T>
int do_cluster(igamg_handle* h, const T* Fin, T* Uio, int load_u, cudaStream_t s) {
  auto& ty = typed<T>(h);
  ty.cdesc.nlev = ty.fused_lc + 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ty.fused_kind);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = ty.cluster_smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ty.fused_kind; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = h->prob.p == 2 ? cudaLaunchKernelEx(&cfg, k_cluster_coarse<2, T>, ty.cdesc, Fin, Uio, load_u)
                                 : cudaLaunchKernelEx(&cfg, k_cluster_coarse<3, T>, ty.cdesc, Fin, Uio, load_u);
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return IGAMG_ECUDA; }
  return IGAMG_OK;
}

template <typename T>
int do_fused(igamg_handle* h, const T* Fin, T* Uio, int load_u, cudaStream_t s) {
  auto& ty = typed<T>(h);
  if (ty.fused_kind > 1) return do_cluster<T>(h, Fin, Uio, load_u, s);
  ty.fused.nlev = ty.fused_lc + 1;
  if (h->prob.p == 2) k_fused_coarse<2, T><<<1, 1024, ty.fused_smem, s>>>(ty.fused, Fin, Uio, load_u);
  else k_fused_coarse<3, T><<<1, 1024, ty.fused_smem, s>>>(ty.fused, Fin, Uio, load_u);
  return launch_check();
}

// Algorithm 1 from level l, recursively, in place on Ul (zeroed first if zero): gamma
// coarse cycles per level, the second and later ones continuing from the previous result
// (gamma = 2: the W-cycle).  Per-level launches throughout.
template <typename T>
int do_cycle(igamg_handle* h, int l, T* Ul, const T* Fl, bool zero, cudaStream_t s) {
  auto& ty = typed<T>(h);
  if (l == 0) return do_coarse<T>(h, Fl, Ul, s);
  int rc;
  if (zero) CK(cudaMemsetAsync(Ul, 0, ty.lev[l].L.n_total * sizeof(T), s));
  if ((rc = do_smooth_n<T>(h, l, Ul, Fl, h->prob.nu1, s))) return rc;
  if ((rc = do_residual<T>(h, l, Ul, Fl, ty.lev[l].R, nullptr, s))) return rc;
  if ((rc = do_restrict<T>(h, l, ty.lev[l].R, ty.lev[l - 1].F, s))) return rc;
  const int gamma = std::max(1, h->prob.gamma);
  for (int g = 0; g < gamma; ++g)
    if ((rc = do_cycle<T>(h, l - 1, ty.lev[l - 1].U, ty.lev[l - 1].F, g == 0, s))) return rc;
  if ((rc = do_prolong<T>(h, l, ty.lev[l - 1].U, Ul, s))) return rc;
  if ((rc = do_smooth_n<T>(h, l, Ul, Fl, h->prob.nu2, s))) return rc;
  return IGAMG_OK;
}

// Algorithm 1 (MGV) from the finest level, unrolled into launches; the coarsest levels
// (0 .. fused_lc) run inside one block when they fit in its shared memory.
template <typename T>
int do_vcycle(igamg_handle* h, T* U, const T* F, cudaStream_t s) {
  auto& ty = typed<T>(h);
  const int L = (int)ty.lev.size();
  if (L == 1) return do_coarse<T>(h, F, U, s);
  if (h->prob.gamma > 1) return do_cycle<T>(h, L - 1, U, F, false, s);
  int rc;
  const int lc = ty.fused_lc;
  if (lc == L - 1) return do_fused<T>(h, F, U, 1, s);
  if (lc >= 1) {
    for (int l = L - 1; l > lc; --l) {
      T* Ul = (l == L - 1) ? U : ty.lev[l].U;
      const T* Fl = (l == L - 1) ? F : ty.lev[l].F;
      if (l < L - 1) CK(cudaMemsetAsync(Ul, 0, ty.lev[l].L.n_total * sizeof(T), s));
      if ((rc = do_smooth_n<T>(h, l, Ul, Fl, h->prob.nu1, s))) return rc;
      if ((rc = do_residual<T>(h, l, Ul, Fl, ty.lev[l].R, nullptr, s))) return rc;
      if ((rc = do_restrict<T>(h, l, ty.lev[l].R, ty.lev[l - 1].F, s))) return rc;
    }
    if ((rc = do_fused<T>(h, ty.lev[lc].F, ty.lev[lc].U, 0, s))) return rc;
    for (int l = lc + 1; l <= L - 1; ++l) {
      T* Ul = (l == L - 1) ? U : ty.lev[l].U;
      const T* Fl = (l == L - 1) ? F : ty.lev[l].F;
      if ((rc = do_prolong<T>(h, l, ty.lev[l - 1].U, Ul, s))) return rc;
      if ((rc = do_smooth_n<T>(h, l, Ul, Fl, h->prob.nu2, s))) return rc;
    }
    return IGAMG_OK;
  }
  for (int l = L - 1; l >= 1; --l) {
    T* Ul = (l == L - 1) ? U : ty.lev[l].U;
    const T* Fl = (l == L - 1) ? F : ty.lev[l].F;
    if (l < L - 1) CK(cudaMemsetAsync(Ul, 0, ty.lev[l].L.n_total * sizeof(T), s));
    if ((rc = do_smooth_n<T>(h, l, Ul, Fl, h->prob.nu1, s))) return rc;
    if ((rc = do_residual<T>(h, l, Ul, Fl, ty.lev[l].R, nullptr, s))) return rc;
    if ((rc = do_restrict<T>(h, l, ty.lev[l].R, ty.lev[l - 1].F, s))) return rc;
  }
  if ((rc = do_coarse<T>(h, ty.lev[0].F, ty.lev[0].U, s))) return rc;
  for (int l = 1; l <= L - 1; ++l) {
    T* Ul = (l == L - 1) ? U : ty.lev[l].U;
    const T* Fl = (l == L - 1) ? F : ty.lev[l].F;
    if ((rc = do_prolong<T>(h, l, ty.lev[l - 1].U, Ul, s))) return rc;
    if ((rc = do_smooth_n<T>(h, l, Ul, Fl, h->prob.nu2, s))) return rc;
  }
  return IGAMG_OK;
}

// Full multigrid (nested iteration) on K e = r with r in the finest level's F workspace and
// e written to its U workspace: r restricted to every level, the coarsest solved exactly,
// then on each finer level one cycle from the prolongated coarser solution.
template <typename T>
int do_fmg(igamg_handle* h, cudaStream_t s) {
  auto& ty = typed<T>(h);
  const int L = (int)ty.lev.size();
  int rc;
  for (int l = L - 1; l >= 1; --l)
    if ((rc = do_restrict<T>(h, l, ty.lev[l].F, ty.lev[l - 1].F, s))) return rc;
  if ((rc = do_coarse<T>(h, ty.lev[0].F, ty.lev[0].U, s))) return rc;
  for (int l = 1; l <= L - 1; ++l) {
    CK(cudaMemsetAsync(ty.lev[l].U, 0, ty.lev[l].L.n_total * sizeof(T), s));
    if ((rc = do_prolong<T>(h, l, ty.lev[l - 1].U, ty.lev[l].U, s))) return rc;
    if ((rc = do_cycle<T>(h, l, ty.lev[l].U, ty.lev[l].F, false, s))) return rc;
  }
  return IGAMG_OK;
}

// FP32 mode, one refinement step: given R64 = F - K U (FP64), an FP32 V-cycle (or, with
// fmg, an FP32 full-multigrid pass) on K e = R64, then U += (curl psi(e), e_p, e_lambda) in
// FP64 and R64 = F - K U with its norm.
int do_ir_step(igamg_handle* h, double* U, const double* F, cudaStream_t s, bool fmg = false) {
  const int L = (int)h->d.lev.size();
  auto& top32 = h->f.lev[L - 1];
  double* R64 = h->d.lev[L - 1].R;
  const auto& Ld = h->d.lev[L - 1].L;
  k_to_float<<<nblk(Ld.n_total), kBlock, 0, s>>>(Ld.n_total, R64, top32.F);
  int rc;
  if (fmg) {
    if ((rc = do_fmg<float>(h, s))) return rc;
  } else {
    CK(cudaMemsetAsync(top32.U, 0, Ld.n_total * sizeof(float), s));
    if ((rc = do_vcycle<float>(h, top32.U, top32.F, s))) return rc;
  }
  k_integrate_psi<<<nblk((long long)Ld.nint * 32, 128), 128, 0, s>>>(Ld.nint, Ld.nxu, h->lc[L - 1].inv_dcoef, top32.U, h->psi);
  k_curl_update<<<nblk(Ld.n_total), kBlock, 0, s>>>(Ld, h->lc[L - 1].dcoef, h->psi, top32.U, U);
  if ((rc = launch_check())) return rc;
  return do_residual<double>(h, L - 1, U, F, R64, h->norm2, s);
}

// one solve step: FP64 mode -> V-cycle + residual norm; FP32 mode -> refinement step.
int do_step(igamg_handle* h, double* U, const double* F, cudaStream_t s) {
  const int L = (int)h->d.lev.size();
  if (fp32_base(h->prob)) return do_ir_step(h, U, F, s);
  int rc = do_vcycle<double>(h, U, F, s);
  if (rc) return rc;
  return do_residual<double>(h, L - 1, U, F, h->d.lev[L - 1].R, h->norm2, s);
}

// first solve step with fmg (R64 = F - K U on entry): U += FMG(R64), then R64 and its norm.
int do_fmg_step(igamg_handle* h, double* U, const double* F, cudaStream_t s) {
  const int L = (int)h->d.lev.size();
  if (fp32_base(h->prob)) return do_ir_step(h, U, F, s, true);
  auto& top = h->d.lev[L - 1];
  const int n = top.L.n_total;
  CK(cudaMemcpyAsync(top.F, top.R, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int rc = do_fmg<double>(h, s);
  if (rc) return rc;
  k_axpby<<<nblk(n), kBlock, 0, s>>>(n, 1.0, 1.0, top.U, U);
  if ((rc = launch_check())) return rc;
  return do_residual<double>(h, L - 1, U, F, top.R, h->norm2, s);
}

// kind 0: solve step; kind 1: public V-cycle (FP32 mode starts by forming R64); kind 2:
// the full-multigrid first step
int ensure_graph(igamg_handle* h, int kind, double* U, const double* F) {
  if (h->graph[kind] && h->gU[kind] == U && h->gF[kind] == F) return IGAMG_OK;
  if (h->graph[kind]) { cudaGraphExecDestroy(h->graph[kind]); h->graph[kind] = nullptr; }
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int L = (int)h->d.lev.size();
  int rc = IGAMG_OK;
  if (kind == 1 && fp32_base(h->prob))
    rc = do_residual<double>(h, L - 1, U, F, h->d.lev[L - 1].R, nullptr, h->cap_stream);
  if (!rc) rc = kind == 2 ? do_fmg_step(h, U, F, h->cap_stream) : do_step(h, U, F, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc) { if (e == cudaSuccess) cudaGraphDestroy(g); return rc; }
  CK(e);
  cudaError_t ei = cudaGraphInstantiate(&h->graph[kind], g, 0);
  cudaGraphDestroy(g);
  CK(ei);
  h->gU[kind] = U; h->gF[kind] = F;
  return IGAMG_OK;
}

// A pipelined sweep gave up waiting (the flag beside the norm): its tiles' step counters
// may disagree, so all of them and the flag are reset before the timeout is reported.
int sweep_timeout(igamg_handle* h, cudaStream_t s) {
  for (size_t l = 0; l < h->lc.size(); ++l) {
    const size_t nt = (size_t)h->lc[l].ntx * h->lc[l].nty;
    if (!nt) continue;
    if (l < h->d.lev.size() && h->d.lev[l].prog) CK(cudaMemsetAsync(h->d.lev[l].prog, 0, nt * sizeof(unsigned), s));
    if (l < h->f.lev.size() && h->f.lev[l].prog) CK(cudaMemsetAsync(h->f.lev[l].prog, 0, nt * sizeof(unsigned), s));
  }
  CK(cudaMemsetAsync(h->sweep_err, 0, sizeof(int), s));
  CK(cudaStreamSynchronize(s));
  g_err = "a pipelined smoothing sweep gave up waiting for a neighbouring tile";
  return IGAMG_ETIMEOUT;
}

bool sweep_flag(const double* pinned_pair) {
  int flag = 0;
  std::memcpy(&flag, pinned_pair + 1, sizeof(int));
  return flag != 0;
}

int read_norm(igamg_handle* h, double* out, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->h_pinned, h->norm2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (sweep_flag(h->h_pinned)) return sweep_timeout(h, s);
  *out = std::sqrt(h->h_pinned[0]);
  return IGAMG_OK;
}
int read_norm(igamg_handle* h, double* out) { return read_norm(h, out, h->stream); }

int div_inf_impl(igamg_handle* h, const double* U, double* out, cudaStream_t s) {
  const int L = (int)h->d.lev.size();
  auto& Lt = h->d.lev[L - 1].L;
  CK(cudaMemsetAsync(h->divmax, 0, sizeof(unsigned long long), s));
  k_div_inf<<<nblk(Lt.n_p), kBlock, 0, s>>>(Lt, h->lc[L - 1].dcoef, U, h->divmax);
  int rc = launch_check();
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->h_pinned, h->divmax, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *out = h->h_pinned[0];
  return IGAMG_OK;
}
int div_inf_impl(igamg_handle* h, const double* U, double* out) { return div_inf_impl(h, U, out, h->stream); }

// Several independent solves at once, each on its handle's own execution stream: one
// round launches one captured step per unfinished solve, then reads all their norms.
// Small solves are latency bound, so running them side by side fills the GPU.
int solve_impl(igamg_handle* h, double* U, const double* F, double rtol, int max_cycles, igamg_report* rep,
               double atol);

// ---- lockstep batches ---------------------------------------------------------------------
// Solves of one cycle shape (2D, FP64, multiplicative V-cycles, same p, sweeps, domain and
// operator form; any mesh sizes and numbers of grids) step their V-cycles together, aligned
// from the finest grid down: every colour, residual, transfer and coarse solve of a depth is
// one launch over all solves of the batch (blockIdx.y = solve, descriptors in a device
// array), captured once into a graph; converged solves are switched off by a device flag
// that their blocks read first.  Per solve the arithmetic is the per-handle V-cycle's
// (per-level launches).

bool batchable(const igamg_handle* h) {
  const auto& pr = h->prob;
  return !h->d3 && pr.precision == IGAMG_FP64 && pr.smoother == IGAMG_MULT && pr.gamma <= 1 && !pr.fmg &&
         !split_colour(h->d.lev.back().L.srow != nullptr);
}

// Handles whose solves can share lockstep launches: the same p (colour count) and cycle shape,
// the same operator form (generalized Stokes or Oseen, square or mapped); mesh sizes and
// numbers of grids may differ.
bool mix_compatible(const igamg_handle* a, const igamg_handle* b) {
  const auto &x = a->prob, &y = b->prob;
  return x.p == y.p && x.nu1 == y.nu1 && x.nu2 == y.nu2 && x.geometry == y.geometry &&
         (x.beta_qp == nullptr) == (y.beta_qp == nullptr);
}

// Descriptors of every solve at every depth (solve-major): depth t is level L - 1 - t of a
// solve with L grids.
void mix_descriptors(int n, igamg_handle** hs, double** Us, const double** Fs, const BatchCache& bc, int nd,
                     std::vector<MixLevel<double>>& D) {
  for (int i = 0; i < n; ++i) {
    igamg_handle* h = hs[i];
    const int L = (int)h->d.lev.size();
    const size_t base = D.size();
    D.resize(base + nd);
    for (int t = 0; t < nd; ++t) {
      MixLevel<double>& d = D[base + t];
      d = MixLevel<double>{};
      const int l = L - 1 - t;
      d.level = l;
      d.active = bc.flags + i;
      d.norm2 = bc.norms + i;
      d.part = h->part;
      if (l < 0) continue;
      const auto& tl = h->d.lev[l];
      const auto& lc = h->lc[l];
      d.L = tl.L;
      d.U = l == L - 1 ? Us[i] : tl.U;
      d.F = l == L - 1 ? const_cast<double*>(Fs[i]) : tl.F;
      d.R = tl.R;
      d.kinv = h->d.coarse_inv;
      if (l >= 1) {
        const auto& tc = h->d.lev[l - 1];
        d.Lc = tc.L;
        d.Uc = tc.U;
        d.Fc = tc.F;
        d.tp = tl.tp;
        d.tq = tl.tq;
        d.cinv = tl.cinv;
        d.cinv8 = tl.cinv8;
        d.dofs = lc.dofs;
        d.cls = lc.cls;
        d.nloc = lc.nloc;
        d.maxl = lc.maxl;
        d.lpr = 1;            // one lane per row: the batch launches are throughput-bound
        for (int c = 0; c < lc.n_colours && c < kMaxColours; ++c) {
          d.first[c] = lc.colour_off[c];
          d.cnt[c] = lc.colour_off[c + 1] - lc.colour_off[c];
          d.n8[c] = lc.n8[c];
        }
      }
    }
  }
}

// One V-cycle of every solve (top residual norms included when cycle), or only the residual
// norms, as launches over all solves of the batch (blockIdx.y = solve).
int batch_launches(igamg_handle** all, const std::vector<int>& idx, const std::vector<MixLevel<double>>& mix, int nd,
                   bool cycle, cudaStream_t s) {
  const int n = (int)idx.size(), p = all[idx[0]]->prob.p;
  std::vector<igamg_handle*> hv(n);
  for (int i = 0; i < n; ++i) hv[i] = all[idx[i]];
  igamg_handle** hs = hv.data();
  const unsigned ns = (unsigned)n;
  std::vector<MixArgs<double>> A(nd);             // the chunk's descriptors, one block per depth
  for (int t = 0; t < nd; ++t) {
    A[t].count = n;
    for (int i = 0; i < n; ++i) A[t].s[i] = mix[(size_t)idx[i] * nd + t];
  }
  const int tpb = 128, wpb = tpb / 32;
  auto lev = [&](int i, int t) { return (int)hs[i]->d.lev.size() - 1 - t; };
  auto max_over = [&](int t, int min_level, auto f) {
    long long m = 0;
    for (int i = 0; i < n; ++i) { int l = lev(i, t); if (l >= min_level) m = std::max(m, (long long)f(i, l)); }
    return (unsigned)std::max(1LL, m);
  };
  auto residual = [&](int t, int any, int want) {
    unsigned nb = max_over(t, any ? 0 : 1, [&](int i, int l) { return nblk(hs[i]->d.lev[l].L.n_total - 1); });
    if (p == 2) k_mix_residual<2, double><<<dim3(nb, ns), kBlock, 0, s>>>(A[t], any);
    else k_mix_residual<3, double><<<dim3(nb, ns), kBlock, 0, s>>>(A[t], any);
    k_mix_residual_finish<double><<<ns, 1024, 0, s>>>(A[t], any, want, kBlock);
  };
  auto smooth = [&](int t) {
    const int C = hs[0]->lc.back().n_colours;
    const size_t shm = (size_t)wpb * max_over(t, 1, [&](int i, int l) { return hs[i]->lc[l].maxl; }) * sizeof(double);
    for (int c = 0; c < C; ++c) {
      unsigned nb = max_over(t, 1, [&](int i, int l) {
        const auto& lc = hs[i]->lc[l];
        const int ppw = 4;
        const int n8 = lc.n8[c], ngen = lc.colour_off[c + 1] - lc.colour_off[c] - n8;
        return (n8 + ppw * wpb - 1) / (ppw * wpb) + (ngen + wpb - 1) / wpb;
      });
      if (p == 2) k_mix_colour<2, double><<<dim3(nb, ns), tpb, shm, s>>>(A[t], c);
      else k_mix_colour<3, double><<<dim3(nb, ns), tpb, shm, s>>>(A[t], c);
    }
  };
  if (cycle) {
    const int nu1 = hs[0]->prob.nu1, nu2 = hs[0]->prob.nu2;
    for (int t = 0; t < nd; ++t) {
      if (t > 0) {
        unsigned nb = max_over(t, 1, [&](int i, int l) { return nblk(hs[i]->d.lev[l].L.n_total); });
        k_mix_zero<double><<<dim3(nb, ns), kBlock, 0, s>>>(A[t]);
      }
      for (int k = 0; k < nu1; ++k) smooth(t);
      residual(t, 0, 0);
      unsigned nbr = max_over(t, 1, [&](int i, int l) { return nblk(hs[i]->d.lev[l - 1].L.n_total); });
      k_mix_restrict<double><<<dim3(nbr, ns), kBlock, 0, s>>>(A[t]);
      int smem = 0;
      for (int i = 0; i < n; ++i)
        if (lev(i, t) == 0) smem = std::max(smem, (int)(hs[i]->d.lev[0].L.n_total * sizeof(double)));
      if (smem > 0) k_mix_coarse<double><<<ns, 1024, smem, s>>>(A[t]);
    }
    for (int t = nd - 2; t >= 0; --t) {
      unsigned nb = max_over(t, 1, [&](int i, int l) { return nblk(hs[i]->d.lev[l].L.n_total); });
      k_mix_prolong_add<double><<<dim3(nb, ns), kBlock, 0, s>>>(A[t]);
      for (int k = 0; k < nu2; ++k) smooth(t);
    }
  }
  residual(0, 1, 1);
  return launch_check();
}

// Captures the batch's launches into one graph, its branches side by side.
int batch_capture(igamg_handle** hs, BatchCache& bc, bool cycle, cudaGraphExec_t* out) {
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(bc.stream, cudaStreamCaptureModeThreadLocal));
  int rc = IGAMG_OK;
  cudaError_t e = cudaEventRecord(bc.ev, bc.stream);
  const int nb = (int)bc.branch.size();
  for (int b = 0; b < nb && !rc && e == cudaSuccess; ++b) {
    cudaStream_t st = b == 0 ? bc.stream : bc.side[b - 1];
    if (b > 0) e = cudaStreamWaitEvent(st, bc.ev, 0);
    if (e == cudaSuccess) rc = batch_launches(hs, bc.branch[b], bc.mix, bc.nd, cycle, st);
    if (!rc && b > 0 && e == cudaSuccess) e = cudaEventRecord(bc.side_ev[b - 1], st);
  }
  for (int b = 1; b < nb && !rc && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(bc.stream, bc.side_ev[b - 1], 0);
  cudaError_t ee = cudaStreamEndCapture(bc.stream, &g);
  if (rc || e != cudaSuccess || ee != cudaSuccess) {
    if (ee == cudaSuccess) cudaGraphDestroy(g);
    cudaGetLastError();
    if (!rc) { g_err = cudaGetErrorString(e != cudaSuccess ? e : ee); rc = IGAMG_ECUDA; }
    return rc;
  }
  cudaError_t ei = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CK(ei);
  return IGAMG_OK;
}

int batch_prepare(int n, igamg_handle** hs, double** Us, const double** Fs, BatchCache*& bcr) {
  std::vector<unsigned long long> key;
  for (int i = 0; i < n; ++i) key.push_back(hs[i]->serial);
  for (int i = 0; i < n; ++i) {
    key.push_back((unsigned long long)(uintptr_t)Us[i]);
    key.push_back((unsigned long long)(uintptr_t)Fs[i]);
  }
  igamg_handle* h0 = hs[0];
  if (h0->bc && h0->bc->key == key) { bcr = h0->bc; return IGAMG_OK; }
  batch_cache_free(h0->bc);
  h0->bc = nullptr;
  auto* bc = new BatchCache();
  bc->key = key;
  bc->count = n;
  int rc = IGAMG_OK;
  auto ck = [&](cudaError_t e) { if (e != cudaSuccess && !rc) { g_err = cudaGetErrorString(e); rc = IGAMG_ECUDA; } };
  ck(cudaMalloc((void**)&bc->flags, n * sizeof(int)));
  ck(cudaMalloc((void**)&bc->norms, n * sizeof(double)));
  ck(cudaMallocHost((void**)&bc->h_flags, n * sizeof(int)));
  ck(cudaMallocHost((void**)&bc->h_norms, n * sizeof(double)));
  ck(cudaStreamCreateWithFlags(&bc->stream, cudaStreamNonBlocking));
  ck(cudaEventCreateWithFlags(&bc->ev, cudaEventDisableTiming));
  bc->nd = 0;
  for (int i = 0; i < n; ++i) bc->nd = std::max(bc->nd, (int)hs[i]->d.lev.size());
  // branches of at most kMixChunk solves, run side by side; the solves are dealt round-robin,
  // so every branch holds a share of every mesh size
  const int nbr = (n + kMixChunk - 1) / kMixChunk;
  bc->branch.assign(nbr, {});
  for (int i = 0; i < n; ++i) bc->branch[i % nbr].push_back(i);
  for (int b = 1; b < nbr && !rc; ++b) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ck(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    bc->side.push_back(st);
    bc->side_ev.push_back(ev);
  }
  if (!rc) mix_descriptors(n, hs, Us, Fs, *bc, bc->nd, bc->mix);
  if (!rc) rc = batch_capture(hs, *bc, false, &bc->g_res);
  if (!rc) rc = batch_capture(hs, *bc, true, &bc->g_cycle);
  if (rc) { batch_cache_free(bc); return rc; }
  h0->bc = bc;
  bcr = bc;
  return IGAMG_OK;
}

int div_inf_impl(igamg_handle* h, const double* U, double* out, cudaStream_t s);

// Lockstep solves of several groups (each a list of indices into hs / Us / Fs); the groups
// run side by side on their own streams.  Same contract as the per-handle batch below.
int batch_lockstep(const std::vector<std::vector<int>>& groups, igamg_handle** hs, double** Us, const double** Fs,
                   double rtol, int max_cycles, igamg_report* reps, int* status, const double* atol) {
  struct G {
    std::vector<igamg_handle*> h;
    std::vector<double*> U;
    std::vector<const double*> F;
    std::vector<int> idx;
    BatchCache* bc = nullptr;
    int active = 0;
  };
  std::vector<G> gs(groups.size());
  int rc;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    G& g = gs[gi];
    g.idx = groups[gi];
    for (int i : g.idx) { g.h.push_back(hs[i]); g.U.push_back(Us[i]); g.F.push_back(Fs[i]); }
    if ((rc = batch_prepare((int)g.idx.size(), g.h.data(), g.U.data(), g.F.data(), g.bc))) return rc;
  }
  const int n_all = [&] { int m = 0; for (auto& g : gs) for (int i : g.idx) m = std::max(m, i + 1); return m; }();
  std::vector<double> r0(n_all, 0.0), rk(n_all, 0.0);
  std::vector<int> k(n_all, 0), st(n_all, IGAMG_NOT_CONVERGED);
  for (auto& g : gs) {                                // inputs were produced on the handles' streams
    const int n = (int)g.idx.size();
    cudaStream_t s = g.bc->stream;
    for (auto* h : g.h) {
      CK(cudaEventRecord(h->ev, h->stream));
      CK(cudaStreamWaitEvent(s, h->ev, 0));
    }
    for (int j = 0; j < n; ++j) g.bc->h_flags[j] = 1;
    CK(cudaMemcpyAsync(g.bc->flags, g.bc->h_flags, n * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaGraphLaunch(g.bc->g_res, s));
    CK(cudaMemcpyAsync(g.bc->h_norms, g.bc->norms, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  int active = 0;
  for (auto& g : gs) {
    CK(cudaStreamSynchronize(g.bc->stream));
    g.active = 0;
    for (size_t j = 0; j < g.idx.size(); ++j) {
      const int i = g.idx[j];
      r0[i] = rk[i] = std::sqrt(g.bc->h_norms[j]);
      if (!std::isfinite(r0[i])) st[i] = IGAMG_ENONFINITE;
      else if (r0[i] == 0.0 || (atol && r0[i] <= atol[i])) st[i] = IGAMG_OK;
      g.bc->h_flags[j] = (st[i] == IGAMG_NOT_CONVERGED && max_cycles > 0) ? 1 : 0;
      g.active += g.bc->h_flags[j];
    }
    active += g.active;
  }
  while (active) {
    for (auto& g : gs) {
      if (!g.active) continue;
      const int n = (int)g.idx.size();
      cudaStream_t s = g.bc->stream;
      CK(cudaMemcpyAsync(g.bc->flags, g.bc->h_flags, n * sizeof(int), cudaMemcpyHostToDevice, s));
      CK(cudaGraphLaunch(g.bc->g_cycle, s));
      CK(cudaMemcpyAsync(g.bc->h_norms, g.bc->norms, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    active = 0;
    for (auto& g : gs) {
      if (!g.active) continue;
      CK(cudaStreamSynchronize(g.bc->stream));
      g.active = 0;
      for (size_t j = 0; j < g.idx.size(); ++j) {
        if (!g.bc->h_flags[j]) continue;
        const int i = g.idx[j];
        ++k[i];
        rk[i] = std::sqrt(g.bc->h_norms[j]);
        igamg_report* rep = reps ? &reps[i] : nullptr;
        if (rep && rep->history && k[i] - 1 < rep->history_cap) rep->history[k[i] - 1] = rk[i] / r0[i];
        if (!std::isfinite(rk[i])) st[i] = IGAMG_ENONFINITE;
        else if (rk[i] <= (atol ? atol[i] : rtol * r0[i])) st[i] = IGAMG_OK;
        g.bc->h_flags[j] = (st[i] == IGAMG_NOT_CONVERGED && k[i] < max_cycles) ? 1 : 0;
        g.active += g.bc->h_flags[j];
      }
      active += g.active;
    }
  }
  int worst = IGAMG_OK;
  for (auto& g : gs) {
    CK(cudaEventRecord(g.bc->ev, g.bc->stream));
    for (size_t j = 0; j < g.idx.size(); ++j) {
      const int i = g.idx[j];
      igamg_handle* h = hs[i];
      CK(cudaStreamWaitEvent(h->stream, g.bc->ev, 0));
      if (reps) {
        reps[i].cycles = k[i]; reps[i].res0 = r0[i]; reps[i].rel_residual = r0[i] > 0 ? rk[i] / r0[i] : 0.0;
        double dv = 0.0;
        if ((rc = div_inf_impl(h, Us[i], &dv, h->stream))) return rc;
        reps[i].div_inf = dv;
      }
      if (status) status[i] = st[i];
      if (st[i] < 0 && worst >= 0) worst = st[i];
      if (st[i] == IGAMG_NOT_CONVERGED && worst == IGAMG_OK) worst = IGAMG_NOT_CONVERGED;
    }
  }
  return worst;
}

// IGAMG_LOCKSTEP=0 runs every batch through the per-handle path (for comparisons).
bool lockstep_enabled() {
  static const bool on = [] { const char* e = std::getenv("IGAMG_LOCKSTEP"); return !e || std::atoi(e) != 0; }();
  return on;
}

// Smallest group that steps in lockstep (IGAMG_LOCKSTEP_MIN, default 8).  Measured on GB300:
// 1024 solves of 64^2..128^2 (groups of ~340) run 1.8x faster in lockstep; 5 + 5 solves of
// 256^2 run 10 % slower, because their latency-bound coarse levels then overlap across two
// streams instead of ten.
int lockstep_min() {
  const char* e = std::getenv("IGAMG_LOCKSTEP_MIN");
  int v = e ? std::atoi(e) : 8;
  return v < 2 ? 2 : v;
}

int solve_batch_impl(int n, igamg_handle** hs, double** Us, const double** Fs, double rtol, int max_cycles,
                     igamg_report* reps, int* status, const double* atol = nullptr, bool allow_lockstep = true) {
  if (allow_lockstep && lockstep_enabled()) {
    // groups of batchable handles step in lockstep: first one group per mesh structure with
    // at least lockstep_min() solves (their launches need no padding blocks and each group
    // stops when its own solves have converged), then one mixed-size group per cycle shape
    // from the handles left over, if it reaches lockstep_min()
    std::vector<std::vector<int>> groups;
    std::vector<int> rest;                       // in their original order below
    std::vector<char> used(n, 0);
    auto same_mesh = [&](int a, int b) {
      return mix_compatible(hs[a], hs[b]) && hs[a]->prob.n_fine == hs[b]->prob.n_fine &&
             hs[a]->prob.n_levels == hs[b]->prob.n_levels;
    };
    std::vector<int> left;
    for (int i = 0; i < n; ++i) {
      if (used[i]) continue;
      used[i] = 1;
      if (!batchable(hs[i])) { rest.push_back(i); continue; }
      std::vector<int> g{i};
      for (int j = i + 1; j < n; ++j)
        if (!used[j] && batchable(hs[j]) && same_mesh(i, j)) { g.push_back(j); used[j] = 1; }
      if ((int)g.size() >= lockstep_min()) groups.push_back(g);
      else left.insert(left.end(), g.begin(), g.end());
    }
    std::sort(left.begin(), left.end());
    std::vector<char> used2(n, 0);
    for (size_t a = 0; a < left.size(); ++a) {
      const int i = left[a];
      if (used2[i]) continue;
      used2[i] = 1;
      std::vector<int> g{i};
      for (size_t b = a + 1; b < left.size(); ++b)
        if (!used2[left[b]] && mix_compatible(hs[i], hs[left[b]])) { g.push_back(left[b]); used2[left[b]] = 1; }
      if ((int)g.size() >= lockstep_min()) groups.push_back(g);
      else rest.insert(rest.end(), g.begin(), g.end());
    }
    std::sort(rest.begin(), rest.end());
    if (!groups.empty()) {
      int worst = batch_lockstep(groups, hs, Us, Fs, rtol, max_cycles, reps, status, atol);
      if (worst < 0 || rest.empty()) return worst;
      const int m = (int)rest.size();
      std::vector<igamg_handle*> h2(m);
      std::vector<double*> U2(m);
      std::vector<const double*> F2(m);
      std::vector<double> a2(m);
      std::vector<igamg_report> r2(m);
      std::vector<int> s2(m, 0);
      for (int j = 0; j < m; ++j) {
        const int i = rest[j];
        h2[j] = hs[i]; U2[j] = Us[i]; F2[j] = Fs[i];
        if (atol) a2[j] = atol[i];
        if (reps) r2[j] = reps[i];
      }
      int w2 = solve_batch_impl(m, h2.data(), U2.data(), F2.data(), rtol, max_cycles, reps ? r2.data() : nullptr,
                                s2.data(), atol ? a2.data() : nullptr, false);
      for (int j = 0; j < m; ++j) {
        if (reps) reps[rest[j]] = r2[j];
        if (status) status[rest[j]] = s2[j];
      }
      if (w2 < 0) return w2;
      return (worst == IGAMG_NOT_CONVERGED || w2 == IGAMG_NOT_CONVERGED) ? IGAMG_NOT_CONVERGED : IGAMG_OK;
    }
  }
  bool krylov = false;
  for (int i = 0; i < n; ++i) krylov = krylov || hs[i]->prob.precision >= IGAMG_FGMRES_FP64;
  if (krylov) {   // FGMRES solves are host-driven: run them one after another
    int worst = IGAMG_OK;
    for (int i = 0; i < n; ++i) {
      int st = solve_impl(hs[i], Us[i], Fs[i], rtol, max_cycles, reps ? &reps[i] : nullptr, atol ? atol[i] : -1.0);
      if (status) status[i] = st;
      if (st < 0) return st;
      if (st == IGAMG_NOT_CONVERGED) worst = IGAMG_NOT_CONVERGED;
    }
    return worst;
  }
  std::vector<double> r0(n, 0.0), rk(n, 0.0);
  std::vector<int> k(n, 0), st(n, IGAMG_NOT_CONVERGED);
  int rc;
  for (int i = 0; i < n; ++i) {
    igamg_handle* h = hs[i];
    CK(cudaEventRecord(h->ev, h->stream));
    CK(cudaStreamWaitEvent(h->exec_stream, h->ev, 0));
    int L = (int)h->d.lev.size();
    if ((rc = do_residual<double>(h, L - 1, Us[i], Fs[i], h->d.lev[L - 1].R, h->norm2, h->exec_stream))) return rc;
    CK(cudaMemcpyAsync(h->h_pinned, h->norm2, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->exec_stream));
  }
  for (int i = 0; i < n; ++i) {
    CK(cudaStreamSynchronize(hs[i]->exec_stream));
    if (sweep_flag(hs[i]->h_pinned)) return sweep_timeout(hs[i], hs[i]->exec_stream);
    r0[i] = rk[i] = std::sqrt(hs[i]->h_pinned[0]);
    if (!std::isfinite(r0[i])) st[i] = IGAMG_ENONFINITE;
    else if (r0[i] == 0.0 || (atol && r0[i] <= atol[i])) st[i] = IGAMG_OK;
    if ((rc = ensure_graph(hs[i], 0, Us[i], Fs[i]))) return rc;
    if (hs[i]->prob.fmg && (rc = ensure_graph(hs[i], 2, Us[i], Fs[i]))) return rc;
  }
  // every solve advances on its own: its next cycle is launched as soon as its last norm is
  // back (an event per solve, polled), so solves whose cycles cost different times (p = 2 and
  // p = 3, other mesh sizes) never wait for each other
  auto launch = [&](int i) -> int {
    igamg_handle* h = hs[i];
    CK(cudaGraphLaunch(h->graph[(k[i] == 0 && h->prob.fmg) ? 2 : 0], h->exec_stream));
    CK(cudaMemcpyAsync(h->h_pinned, h->norm2, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->exec_stream));
    CK(cudaEventRecord(h->ev, h->exec_stream));
    ++k[i];
    return IGAMG_OK;
  };
  std::vector<char> busy(n, 0);
  int inflight = 0;
  for (int i = 0; i < n; ++i)
    if (st[i] == IGAMG_NOT_CONVERGED && k[i] < max_cycles) {
      if ((rc = launch(i))) return rc;
      busy[i] = 1;
      ++inflight;
    }
  while (inflight) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      if (!busy[i]) continue;
      igamg_handle* h = hs[i];
      const cudaError_t q = cudaEventQuery(h->ev);
      if (q == cudaErrorNotReady) continue;
      CK(q);
      any = true;
      busy[i] = 0;
      --inflight;
      if (sweep_flag(h->h_pinned)) return sweep_timeout(h, h->exec_stream);
      rk[i] = std::sqrt(h->h_pinned[0]);
      igamg_report* rep = reps ? &reps[i] : nullptr;
      if (rep && rep->history && k[i] - 1 < rep->history_cap) rep->history[k[i] - 1] = rk[i] / r0[i];
      if (!std::isfinite(rk[i])) st[i] = IGAMG_ENONFINITE;
      else if (rk[i] <= (atol ? atol[i] : rtol * r0[i])) st[i] = IGAMG_OK;
      if (st[i] == IGAMG_NOT_CONVERGED && k[i] < max_cycles) {
        if ((rc = launch(i))) return rc;
        busy[i] = 1;
        ++inflight;
      }
    }
    if (!any) std::this_thread::yield();
  }
  for (int i = 0; i < n; ++i) {
    igamg_handle* h = hs[i];
    if (reps) {
      reps[i].cycles = k[i]; reps[i].res0 = r0[i]; reps[i].rel_residual = r0[i] > 0 ? rk[i] / r0[i] : 0.0;
      double dv = 0.0;
      if ((rc = div_inf_impl(h, Us[i], &dv, h->exec_stream))) return rc;
      reps[i].div_inf = dv;
    }
    CK(cudaEventRecord(h->ev, h->exec_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev, 0));
    if (status) status[i] = st[i];
  }
  int worst = IGAMG_OK;
  for (int i = 0; i < n; ++i) {
    if (st[i] < 0) return st[i];
    if (st[i] == IGAMG_NOT_CONVERGED) worst = IGAMG_NOT_CONVERGED;
  }
  return worst;
}

// ---- FGMRES around the V-cycle (krylov.cu) ---------------------------------------------
int kr_precond(void* ctx, const double* v, double* z) {
  auto* h = (igamg_handle*)ctx;
  cudaStream_t s = h->stream;
  const int L = (int)h->d.lev.size();
  const auto& Ld = h->d.lev[L - 1].L;
  CK(cudaMemsetAsync(z, 0, Ld.n_total * sizeof(double), s));
  if (h->prob.precision == IGAMG_FGMRES_FP64) return do_vcycle<double>(h, z, v, s);
  auto& top32 = h->f.lev[L - 1];
  k_to_float<<<nblk(Ld.n_total), kBlock, 0, s>>>(Ld.n_total, v, top32.F);
  CK(cudaMemsetAsync(top32.U, 0, Ld.n_total * sizeof(float), s));
  int rc = do_vcycle<float>(h, top32.U, top32.F, s);
  if (rc) return rc;
  k_integrate_psi<<<nblk((long long)Ld.nint * 32, 128), 128, 0, s>>>(Ld.nint, Ld.nxu, h->lc[L - 1].inv_dcoef, top32.U, h->psi);
  k_curl_update<<<nblk(Ld.n_total), kBlock, 0, s>>>(Ld, h->lc[L - 1].dcoef, h->psi, top32.U, z);
  return launch_check();
}

int kr_apply(void* ctx, const double* z, double* w) {
  auto* h = (igamg_handle*)ctx;
  const int L = (int)h->d.lev.size();
  int rc = do_residual<double>(h, L - 1, z, h->zeros, w, nullptr, h->stream);     // w = -K z
  if (rc) return rc;
  return krylov_negate(w, h->d.lev[L - 1].L.n_total, h->stream);
}

int kr_residual(void* ctx, const double* U, const double* F, double* R, double* norm) {
  auto* h = (igamg_handle*)ctx;
  const int L = (int)h->d.lev.size();
  int rc = do_residual<double>(h, L - 1, U, F, R, h->norm2, h->stream);
  if (rc) return rc;
  return read_norm(h, norm);
}

int fgmres_impl(igamg_handle* h, double* U, const double* F, double rtol, int max_cycles, igamg_report* rep,
                double atol) {
  KrylovOps ops;
  ops.ctx = h; ops.stream = h->stream;
  ops.precond = kr_precond; ops.apply = kr_apply; ops.residual = kr_residual;
  int st = fgmres_solve(ops, h->kw, U, F, rtol, atol, max_cycles, rep);
  if (st < 0) return st;
  if (rep) {
    double dv = 0.0;
    int rc = div_inf_impl(h, U, &dv);
    if (rc) return rc;
    rep->div_inf = dv;
  }
  return st;
}

int solve_impl(igamg_handle* h, double* U, const double* F, double rtol, int max_cycles, igamg_report* rep,
               double atol) {
  if (h->prob.precision >= IGAMG_FGMRES_FP64) return fgmres_impl(h, U, F, rtol, max_cycles, rep, atol);
  int L = (int)h->d.lev.size();
  int rc = do_residual<double>(h, L - 1, U, F, h->d.lev[L - 1].R, h->norm2, h->stream);
  if (rc) return rc;
  double r0;
  if ((rc = read_norm(h, &r0))) return rc;
  if (!std::isfinite(r0)) return IGAMG_ENONFINITE;
  if ((rc = ensure_graph(h, 0, U, F))) return rc;
  if (h->prob.fmg && (rc = ensure_graph(h, 2, U, F))) return rc;
  int k = 0;
  double rk = r0;
  int status = IGAMG_NOT_CONVERGED;
  if (r0 == 0.0 || (atol >= 0 && r0 <= atol)) status = IGAMG_OK;
  while (status == IGAMG_NOT_CONVERGED && k < max_cycles) {
    CK(cudaGraphLaunch(h->graph[(k == 0 && h->prob.fmg) ? 2 : 0], h->stream));
    ++k;
    if ((rc = read_norm(h, &rk))) return rc;
    if (!std::isfinite(rk)) { status = IGAMG_ENONFINITE; break; }
    if (rep && rep->history && k - 1 < rep->history_cap) rep->history[k - 1] = rk / r0;
    if (rk <= (atol >= 0 ? atol : rtol * r0)) status = IGAMG_OK;
  }
  if (rep) {
    rep->cycles = k; rep->res0 = r0; rep->rel_residual = r0 > 0 ? rk / r0 : 0.0;
    double dv = 0.0;
    if ((rc = div_inf_impl(h, U, &dv))) return rc;
    rep->div_inf = dv;
  }
  return status;
}

template <typename T>
LevelTab<T> make_tab(const igamg_sizes& sz, int p, const T* sx, const T* sy, const T* sp, const T* srow = nullptr,
                     const T* sext = nullptr) {
  LevelTab<T> L{};
  L.srow = srow;
  L.sext = sext;
  int n = sz.n;
  L.n = n; L.nxu = n + p - 2; L.npd = n + p - 1; L.nint = n + p - 2; L.lastp = n + p - 1; L.lastq = n + p - 2;
  L.n_ux = (int)sz.n_ux; L.n_uy = (int)sz.n_uy; L.n_p = (int)sz.n_p; L.n_total = (int)sz.n_total;
  L.sx = sx; L.sy = sy; L.sp = sp;
  return L;
}

// Choose the coarse levels that run in one block (multiplicative smoother only): all
// levels with at most 32 (FP64) / 64 (FP32) elements per direction whose vectors fit in
// shared memory, and fill the kernel's level descriptors.
// Descriptor of the cluster form of the coarse end (k_cluster_coarse): every level below
// the finest whose colouring fits the descriptor; the depth and the cluster size are picked
// by the autotuner.
template <typename T>
int setup_cluster(igamg_handle* h, Typed<T>& ty) {
  ty.cluster_max = -1;
  const int L = h->prob.n_levels;
  if (h->prob.smoother != IGAMG_MULT || L < 2) return IGAMG_OK;
  if (std::getenv("IGAMG_NO_CLUSTER")) return IGAMG_OK;
  int best = -1, maxl = 0;
  for (int lc = 1; lc < L && lc < kMaxFused; ++lc) {
    if (h->lc[lc].n_colours > kMaxColours) break;
    best = lc;
  }
  if (best < 1) return IGAMG_OK;
  ClusterDesc<T>& D = ty.cdesc;
  D = ClusterDesc<T>{};
  D.nlev = best + 1; D.nu1 = h->prob.nu1; D.nu2 = h->prob.nu2; D.ndof0 = h->host.ndof0;
  D.coarse_inv = ty.coarse_inv;
  int rc = dmalloc(h, (void**)&D.part, 32 * sizeof(double));
  if (rc) return rc;
  for (int l = 0; l <= best; ++l) {
    ClusterLevel<T>& V = D.lev[l];
    const auto& lc = h->lc[l];
    V.L = ty.lev[l].L; V.tp = ty.lev[l].tp; V.tq = ty.lev[l].tq; V.cinv = ty.lev[l].cinv; V.cinv8 = ty.lev[l].cinv8;
    V.dofs = lc.dofs; V.cls = lc.cls; V.nloc = lc.nloc; V.maxl = lc.maxl; V.n_colours = lc.n_colours;
    for (int k = 0; k <= lc.n_colours && l >= 1; ++k) V.colour_off[k] = lc.colour_off[k];
    for (int k = 0; k < lc.n_colours && l >= 1; ++k) V.n8[k] = lc.n8[k];
    V.U = ty.lev[l].U; V.F = ty.lev[l].F; V.R = ty.lev[l].R;
    maxl = std::max(maxl, lc.maxl);
  }
  D.maxl = std::max(maxl, 1);
  ty.cluster_smem = (size_t)32 * D.maxl * sizeof(T);
  for (auto fn : {(const void*)k_cluster_coarse<2, T>, (const void*)k_cluster_coarse<3, T>}) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ty.cluster_smem) != cudaSuccess) {
      cudaGetLastError();
      return IGAMG_OK;                 // no cluster form on this device: per-level launches
    }
  }
  ty.cluster_max = best;
  return IGAMG_OK;
}

template <typename T>
int setup_fused(igamg_handle* h, Typed<T>& ty) {
  ty.fused_lc = -1;
  const int L = h->prob.n_levels;
  if (h->prob.smoother != IGAMG_MULT || L < 2) return IGAMG_OK;
  const int nmax = sizeof(T) == 8 ? 32 : 64;
  const size_t limit = 200 * 1024;
  int best = -1;
  size_t best_bytes = 0;
  for (int lc = 1; lc < L && lc < kMaxFused; ++lc) {
    if (h->lc[lc].sz.n > nmax) break;
    size_t words = 0;
    int maxl = 0;
    for (int l = 0; l <= lc; ++l) {
      words += 3 * (size_t)((h->lc[l].sz.n_total + 3) / 4 * 4);
      maxl = std::max(maxl, h->lc[l].maxl);
    }
    words += 32 * (size_t)maxl;
    size_t bytes = words * sizeof(T);
    if (bytes > limit) break;
    if (h->lc[lc].n_colours > kMaxColours) break;
    best = lc; best_bytes = bytes;
  }
  ty.fused_max = best;
  if (best < 1) return IGAMG_OK;
  FusedDesc<T>& D = ty.fused;
  D = FusedDesc<T>{};
  D.nlev = best + 1; D.nu1 = h->prob.nu1; D.nu2 = h->prob.nu2; D.ndof0 = h->ndof0 ? h->ndof0 : h->host.ndof0;
  D.coarse_inv = ty.coarse_inv;
  int off = 0;
  int maxl = 0;
  for (int l = 0; l <= best; ++l) {
    FusedLevel<T>& V = D.lev[l];
    const auto& lc = h->lc[l];
    V.L = ty.lev[l].L; V.tp = ty.lev[l].tp; V.tq = ty.lev[l].tq; V.cinv = ty.lev[l].cinv; V.cinv8 = ty.lev[l].cinv8;
    V.dofs = lc.dofs; V.cls = lc.cls; V.nloc = lc.nloc; V.maxl = lc.maxl; V.n_colours = lc.n_colours;
    for (int k = 0; k <= lc.n_colours && l >= 1; ++k) V.colour_off[k] = lc.colour_off[k];
    for (int k = 0; k < lc.n_colours && l >= 1; ++k) V.n8[k] = lc.n8[k];
    int nt = (int)((lc.sz.n_total + 3) / 4 * 4);
    V.offU = off; off += nt;
    V.offF = off; off += nt;
    V.offR = off; off += nt;
    maxl = std::max(maxl, lc.maxl);
  }
  D.scratch_off = off;
  ty.fused_smem = best_bytes;
  ty.fused_lc = best;           // refined by autotune_fused
  cudaError_t e = h->prob.p == 2
      ? cudaFuncSetAttribute(k_fused_coarse<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)best_bytes)
      : cudaFuncSetAttribute(k_fused_coarse<3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)best_bytes);
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return IGAMG_ECUDA; }
  return IGAMG_OK;
}

// Autotuner: time a few V-cycles with each feasible depth of the one-block coarse part
// (none, levels 0..1, 0..2, ...) and keep the fastest.  The choice depends only on the
// shape (p, n_fine, levels, value type, smoother) and is cached per process.
struct TuneKey {
  int p, n, L, bytes, sm, nu1, nu2;
  int rows;                     // 1: per-row operators (Oseen, mapped domains), 0: class stencils
  bool operator<(const TuneKey& o) const {
    return std::tie(p, n, L, bytes, sm, nu1, nu2, rows) < std::tie(o.p, o.n, o.L, o.bytes, o.sm, o.nu1, o.nu2, o.rows);
  }
};
std::map<TuneKey, std::pair<int, int>>& tune_cache() { static std::map<TuneKey, std::pair<int, int>> m; return m; }
std::mutex& tune_mutex() { static std::mutex m; return m; }

// IGAMG_TUNE_CACHE=<file>: the tuned coarse-end choices persist across processes, one line per
// shape ("p n_fine levels bytes smoother nu1 nu2 rows depth kind"), so that a run under a
// profiler reuses what a plain run measured (the profiler's serialised launches would skew a
// fresh tuning).  The file is advisory: unreadable or missing means tune as usual.  Call with
// tune_mutex held.
void tune_file_load() {
  static bool done = false;
  if (done) return;
  done = true;
  const char* path = std::getenv("IGAMG_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  TuneKey k{};
  int d = 0, kind = 0;
  while (std::fscanf(f, "%d %d %d %d %d %d %d %d %d %d", &k.p, &k.n, &k.L, &k.bytes, &k.sm, &k.nu1, &k.nu2, &k.rows, &d,
                     &kind) == 10)
    tune_cache()[k] = {d, kind};
  std::fclose(f);
}

void tune_file_append(const TuneKey& k, int d, int kind) {
  const char* path = std::getenv("IGAMG_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d\n", k.p, k.n, k.L, k.bytes, k.sm, k.nu1, k.nu2, k.rows, d, kind);
  std::fclose(f);
}

template <typename T>
int autotune_fused(igamg_handle* h, Typed<T>& ty) {
  ty.fused_kind = 1;
  if (ty.fused_max < 1 && ty.cluster_max < 1) { ty.fused_lc = -1; return IGAMG_OK; }
  if (h->prob.gamma > 1) { ty.fused_lc = -1; return IGAMG_OK; }   // W-cycles run level by level
  const int L = h->prob.n_levels;
  TuneKey key{h->prob.p, h->prob.n_fine, L, (int)sizeof(T), h->prob.smoother, h->prob.nu1, h->prob.nu2,
              (h->prob.beta_qp || h->prob.geometry != IGAMG_GEOM_SQUARE) ? 1 : 0};
  // fixed choices (tests, experiments): IGAMG_FUSED_LEVELS = depth, IGAMG_FUSED_CLUSTER = blocks
  const char* env = std::getenv("IGAMG_FUSED_LEVELS");
  if (env) {
    const char* ec = std::getenv("IGAMG_FUSED_CLUSTER");
    int kind = ec ? std::atoi(ec) : 1;
    int lim = kind > 1 ? ty.cluster_max : ty.fused_max;
    ty.fused_kind = kind > 1 ? kind : 1;
    ty.fused_lc = std::min(std::atoi(env), lim);
    if (ty.fused_lc < 1) ty.fused_lc = -1;
    return IGAMG_OK;
  }
  {
    std::lock_guard<std::mutex> lk(tune_mutex());
    tune_file_load();
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) { ty.fused_lc = it->second.first; ty.fused_kind = it->second.second; return IGAMG_OK; }
  }
  T* U = ty.lev[L - 1].U;
  T* F = ty.lev[L - 1].F;
  size_t nb = (size_t)ty.lev[L - 1].L.n_total * sizeof(T);
  CK(cudaMemsetAsync(U, 0, nb, h->stream));
  CK(cudaMemsetAsync(F, 0, nb, h->stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // each candidate is timed the way solves run it: one V-cycle captured into a graph,
  // replayed (launch overheads of the per-level path are those of graph replay)
  float best_ms = 1e30f;
  int best = -1;
  const bool verbose = std::getenv("IGAMG_VERBOSE") != nullptr;
  std::vector<std::pair<int, int>> cands{{-1, 1}};
  for (int d = 1; d <= ty.fused_max; ++d) cands.push_back({d, 1});
  for (int C : {4, 8, 16})
    for (int d = 1; d <= ty.cluster_max; ++d) cands.push_back({d, C});
  int best_kind = 1;
  for (auto [cand, kind] : cands) {
    ty.fused_lc = cand;
    ty.fused_kind = kind;
    cudaGraph_t g;
    cudaGraphExec_t ge = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = do_vcycle<T>(h, U, F, h->cap_stream);
    cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc && kind > 1) {                  // this cluster size cannot be launched here: skip it
      if (ec == cudaSuccess) cudaGraphDestroy(g);
      cudaGetLastError();
      if (verbose) std::fprintf(stderr, "igamg: cluster %d unavailable (%s)\n", kind, g_err.c_str());
      continue;
    }
    if (rc) { if (ec == cudaSuccess) cudaGraphDestroy(g); cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    CK(ec);
    cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess && kind > 1) {
      cudaGetLastError();
      if (verbose) std::fprintf(stderr, "igamg: cluster %d graph unavailable (%s)\n", kind, cudaGetErrorString(ei));
      continue;
    }
    CK(ei);
    float ms = 0;
    cudaError_t e = cudaGraphLaunch(ge, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = cudaGraphLaunch(ge, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaGraphExecDestroy(ge);
    CK(e);
    if (verbose) std::fprintf(stderr, "igamg: fused coarse levels %d (blocks %d): %.1f us per V-cycle\n", cand, kind, 1e3f * ms / 5);
    if (ms < best_ms) { best_ms = ms; best = cand; best_kind = kind; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ty.fused_lc = best;
  ty.fused_kind = best_kind;
  if (verbose) std::fprintf(stderr, "igamg: chose fused coarse levels %d (blocks %d)\n", best, best_kind);
  std::lock_guard<std::mutex> lk(tune_mutex());
  tune_cache()[key] = {best, best_kind};
  tune_file_append(key, best, best_kind);
  return IGAMG_OK;
}

bool bf16_operands() {
  const char* e = std::getenv("IGAMG_BF16_OPERANDS");
  return e && std::atoi(e) != 0;
}

// Values rounded to the nearest bfloat16 (ties to even), returned in double.
std::vector<double> round_bf16(const std::vector<double>& v) {
  std::vector<double> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    float f = (float)v[i];
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    std::memcpy(&f, &u, 4);
    out[i] = f;
  }
  return out;
}

// Upload the typed (double or float) copy of every level's tables and workspaces.
template <typename T>
int upload_typed(igamg_handle* h, Typed<T>& ty, size_t max_delta) {
  const int L = h->prob.n_levels, p = h->prob.p;
  ty.lev.resize(L);
  int rc;
  // BF16 operands (FP32 V-cycles only, IGAMG_BF16_OPERANDS=1 at creation): the operator's
  // stencil records and the patch solves' local inverses rounded to bfloat16 (round to
  // nearest even), applied with FP32 accumulation; transfers and the coarsest solve stay FP32
  const bool bf16 = sizeof(T) == 4 && bf16_operands();
  auto ops = [&](const std::vector<double>& v) { return bf16 ? round_bf16(v) : v; };
  for (int l = 0; l < L; ++l) {
    auto& lh = h->host.lev[l];
    auto& tl = ty.lev[l];
    T *sx, *sy, *sp, *srow = nullptr, *sext = nullptr;
    if ((rc = upload_as(h, &sx, ops(lh.st.sx))) || (rc = upload_as(h, &sy, ops(lh.st.sy))) ||
        (rc = upload_as(h, &sp, ops(lh.st.sp))))
      return rc;
    if (!lh.rows.empty() && (rc = upload_as(h, &srow, ops(lh.rows)))) return rc;
    if (!lh.ext.empty() && (rc = upload_as(h, &sext, ops(lh.ext)))) return rc;
    tl.L = make_tab<T>(lh.sz, p, sx, sy, sp, srow, sext);
    if (l >= 1) {
      if ((rc = upload_as(h, &tl.cinv, ops(lh.pt.cinv)))) return rc;
      if ((rc = upload_as(h, &tl.cinv8, ops(lh.pt.cinv8)))) return rc;
      for (int which = 0; which < 2; ++which) {
        const Transfer1D& Tr = which ? h->host.tq[l] : h->host.tp_free[l];
        Xfer<T>& X = which ? tl.tq : tl.tp;
        int *c0, *f0; T *pv, *rv;
        if ((rc = upload_as(h, &c0, Tr.c0)) || (rc = upload_as(h, &f0, Tr.f0)) || (rc = upload_as(h, &pv, Tr.pv)) ||
            (rc = upload_as(h, &rv, Tr.rv))) return rc;
        X.nf = Tr.nf; X.nc = Tr.nc; X.c0 = c0; X.f0 = f0; X.pv = pv; X.rv = rv;
      }
    }
    size_t nb = (size_t)lh.sz.n_total * sizeof(T);
    if ((rc = dmalloc(h, (void**)&tl.R, nb))) return rc;
    if ((rc = dmalloc(h, (void**)&tl.U, nb))) return rc;
    if ((rc = dmalloc(h, (void**)&tl.F, nb))) return rc;
  }
  if ((rc = upload_as(h, &ty.coarse_inv, h->host.coarse_inv))) return rc;
  if ((rc = dmalloc(h, (void**)&ty.delta, std::max<size_t>(max_delta, 1) * sizeof(T)))) return rc;
  // matrix-free advection tables (not with BF16 operands: those round the stored operator)
  const auto& H = h->host;
  const int tx = adv_tiles_x(p, H.n_fine);
  if (!H.adv_bp.empty() && !bf16 && (size_t)tx * tx <= nblk(H.lev.back().sz.n_total) + 1) {
    T *bp, *dp, *bq, *dq, *beta;
    if ((rc = upload_as(h, &bp, H.adv_bp)) || (rc = upload_as(h, &dp, H.adv_dp)) || (rc = upload_as(h, &bq, H.adv_bq)) ||
        (rc = upload_as(h, &dq, H.adv_dq)) || (rc = upload_as(h, &beta, H.adv_beta)))
      return rc;
    ty.adv.n = H.n_fine;
    ty.adv.bp = bp; ty.adv.dp = dp; ty.adv.bq = bq; ty.adv.dq = dq; ty.adv.beta = beta;
    // interior copies: the tables of element p stand for elements p .. n-1-p (checked: uniform
    // B-splines there, equal up to the rounding of their evaluation points), the records of
    // the interior row class (2p+1, 2p+1)
    const int G = p + 2, q = p - 1, nf = H.n_fine;
    // (FP32 only: the FP64 kernel is bound by its FP64 multiply-adds, and the longer code of
    // the constant-operand path measured slower there)
    bool inner = sizeof(T) == 4 && nf >= 2 * p + 1 && (p + 1) * G <= kAdvMaxPG && H.lev.back().st.RU <= kAdvMaxRU && H.lev.back().st.T == 2 * p + 1;
    auto same = [&](const std::vector<double>& tab, int d) {
      const size_t m = (size_t)(d + 1) * G;
      double scale = 0.0;
      for (size_t k = 0; k < m; ++k) scale = std::max(scale, std::fabs(tab[(size_t)p * m + k]));
      for (int e = p; inner && e <= nf - 1 - p; ++e)
        for (size_t k = 0; k < m; ++k)
          if (std::fabs(tab[(size_t)e * m + k] - tab[(size_t)p * m + k]) > 1e-12 * scale) return false;
      return true;
    };
    inner = inner && same(H.adv_bp, p) && same(H.adv_dp, p) && same(H.adv_bq, q) && same(H.adv_dq, q);
    ty.adv.inner = inner ? 1 : 0;
    if (inner) {
      for (int k = 0; k < (p + 1) * G; ++k) {
        ty.adv.ibp[k] = (T)H.adv_bp[(size_t)p * (p + 1) * G + k];
        ty.adv.idp[k] = (T)H.adv_dp[(size_t)p * (p + 1) * G + k];
      }
      for (int k = 0; k < (q + 1) * G; ++k) {
        ty.adv.ibq[k] = (T)H.adv_bq[(size_t)p * (q + 1) * G + k];
        ty.adv.idq[k] = (T)H.adv_dq[(size_t)p * (q + 1) * G + k];
      }
      const Stencils& st = H.lev.back().st;
      const size_t off = ((size_t)st.T * st.NC + st.T) * st.RU;
      for (int j = 0; j < st.RU; ++j) {
        ty.adv.rx[j] = (T)st.sx[off + j];
        ty.adv.ry[j] = (T)st.sy[off + j];
        ty.adv.rp[j] = (T)st.sp[off + j];
      }
    }
    if (p == 2) CK(cudaFuncSetAttribute(k_residual_adv<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdvShape<2>::smem<T>()));
    else CK(cudaFuncSetAttribute(k_residual_adv<3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdvShape<3>::smem<T>()));
  }
  if ((rc = setup_cluster<T>(h, ty))) return rc;
  return setup_fused<T>(h, ty);
}

// Tile forms of the sweep allowed (default) or not (IGAMG_PIPELINE=0: colour launches only);
// read when a handle is created.
bool pipeline_on() {
  const char* e = std::getenv("IGAMG_PIPELINE");
  return !e || std::atoi(e) != 0;
}

// Blocks of k_sweep_tiles that the whole GPU holds at once (a cooperative launch may not
// ask for more).
template <typename T>
int tile_capacity(int p, int maxl) {
  int dev = 0, sms = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cudaError_t e = p == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_tiles<2, T, kTileThreads>, kTileThreads, tile_smem<T>(maxl))
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_tiles<3, T, kTileThreads>, kTileThreads, tile_smem<T>(maxl));
  return e == cudaSuccess ? nb * sms : 0;
}

// The smoother form of each level, chosen at creation (the project's autotuner; thread and
// tile shapes of the multiplicative sweep):
//   colour launches, one lane per patch row   (lpr 1: k_mult_colour, four patches per warp),
//                                              blocks of 128 (or 64, 256) threads
//   colour launches, two lanes per patch row  (lpr 2: two patches per warp; 128 or 64)
//   one block for the whole level             (k_sweep_tiles with one tile of 512 threads)
//   pipelined tiles of (p + 1) m positions    (k_sweep_tiles, 128 threads, m = 1, 2, 4)
// Each candidate is timed the way solves run it: nu1 sweeps of the level captured into a CUDA
// graph, replayed after a warm-up (best of three), on the level's zeroed FP64 workspaces (the
// arithmetic does not depend on the values).  Choices are cached per process by (p, n, per-row
// records, mapped).  IGAMG_PIPELINE=0 leaves out the tile forms; IGAMG_SWEEP_FORM pins one
// ("lanes1", "lanes2", "lanes1_b64", "lanes2_b64", "lanes1_b256", "solo", "tiles1", "tiles2",
// "tiles4").
struct SweepForm { int lpr = 1, tiles = 0, tpb = 0, ch = 4; };   // tiles: 0 colour launches, -1 one block, m > 0
std::map<std::tuple<int, int, int, int>, SweepForm>& form_cache() {
  static std::map<std::tuple<int, int, int, int>, SweepForm> m;
  return m;
}
// guards form_cache and adv_cache: handles may be created from several host threads at once
// (the lookups and inserts are locked; the timings between them are not)
std::mutex& form_mutex() {
  static std::mutex m;
  return m;
}

std::string form_name(const SweepForm& f) {
  if (f.tiles == 0)
    return std::string(f.lpr == 2 ? "lanes2" : "lanes1") + (f.tpb ? "_b" + std::to_string(f.tpb) : "") +
           (f.ch == 2 ? "_c2" : "");
  if (f.tiles < 0) return "solo";
  return "tiles" + std::to_string(f.tiles);
}

// Installs form f on level l (uploading its tile schedule); the step counters must hold
// nt_max entries.  Returns IGAMG_EUNSUPPORTED if the form does not fit the level.
int apply_form(igamg_handle* h, int l, const SweepForm& f) {
  auto& lc = h->lc[l];
  const int p = h->prob.p;
  const PatchTables& pt = h->host.lev[l].pt;
  lc.lpr = f.lpr;
  lc.tpb = f.tpb;
  lc.ch = f.lpr == 1 && f.tiles == 0 ? f.ch : 4;
  lc.ntx = lc.nty = 0;
  if (f.tiles == 0) return IGAMG_OK;
  const int nint = lc.sz.n + p - 2;
  const int tw = f.tiles < 0 ? nint : (p + 1) * f.tiles;
  TileTables tt;
  build_tile_tables(pt, nint, tw, tt);
  const int C = pt.n_colours, nt = tt.ntx * tt.nty;
  // every patch exactly once, in a run of its own colour, its 8-DOF patches first
  std::vector<char> seen(pt.n_patches, 0);
  bool ok = (int)tt.list.size() == pt.n_patches && (int)tt.off.size() == nt * C + 1 && tt.off[nt * C] == pt.n_patches;
  for (int r = 0; ok && r < nt * C; ++r) {
    const int c = r % C;
    ok = tt.off[r] <= tt.off[r + 1] && tt.n8[r] <= tt.off[r + 1] - tt.off[r];
    for (int j = tt.off[r]; ok && j < tt.off[r + 1]; ++j) {
      const int i = tt.list[j];
      const bool is8 = i < pt.colour_off[c] + pt.n8[c];
      ok = i >= pt.colour_off[c] && i < pt.colour_off[c + 1] && !seen[i] && (is8 == (j < tt.off[r] + tt.n8[r]));
      if (ok) seen[i] = 1;
    }
  }
  if (!ok) { g_err = "tile schedule inconsistent with the patch tables"; return IGAMG_EINVAL; }
  int rc;
  if ((rc = upload_as(h, &lc.tile_list, tt.list)) || (rc = upload_as(h, &lc.tile_off, tt.off)) ||
      (rc = upload_as(h, &lc.tile_n8, tt.n8)))
    return rc;
  lc.tw = tw; lc.ntx = tt.ntx; lc.nty = tt.nty;
  return IGAMG_OK;
}

// Graph-replayed time (ms) of nu1 (at least one) sweeps of level l in its current form.
int time_level_sweeps(igamg_handle* h, int l, float* ms_out) {
  auto& tl = h->d.lev[l];
  const int sw = std::max(1, h->prob.nu1);
  cudaGraph_t g;
  cudaGraphExec_t ge = nullptr;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = do_smooth_n<double>(h, l, tl.U, tl.F, sw, h->cap_stream);
  cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc) { if (ec == cudaSuccess) cudaGraphDestroy(g); return rc; }
  CK(ec);
  cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  CK(ei);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  cudaError_t e = cudaGraphLaunch(ge, h->stream);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    float ms = 0;
    e = cudaEventRecord(e0, h->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaGraphExecDestroy(ge);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(e);
  double flag[2];
  CK(cudaMemcpy(flag, h->norm2, sizeof(flag), cudaMemcpyDeviceToHost));
  if (sweep_flag(flag)) return sweep_timeout(h, h->stream);
  *ms_out = best;
  return IGAMG_OK;
}

int setup_sweep_forms(igamg_handle* h) {
  if (const char* e = std::getenv("IGAMG_TEST_STALL_TILE")) h->stall_tile = std::atoi(e);
  if (h->prob.smoother != IGAMG_MULT) return IGAMG_OK;
  const int p = h->prob.p, L = (int)h->lc.size();
  const bool mapped = h->prob.geometry != IGAMG_GEOM_SQUARE;
  const bool tiles_ok = pipeline_on();
  const char* pin = std::getenv("IGAMG_SWEEP_FORM");
  const char* env_lanes = std::getenv("IGAMG_ROW_LANES");
  const char* env_mult = std::getenv("IGAMG_TILE_MULT");
  const bool verbose = std::getenv("IGAMG_VERBOSE") != nullptr;
  int rc;
  for (int l = 1; l < L; ++l) {
    auto& lc = h->lc[l];
    const PatchTables& pt = h->host.lev[l].pt;
    const bool has_pos = (int)pt.pos.size() == pt.n_patches;
    const int nint = lc.sz.n + p - 2;
    int cap = tile_capacity<double>(p, lc.maxl);
    if (fp32_base(h->prob)) cap = std::min(cap, tile_capacity<float>(p, lc.maxl));
    auto ntiles = [&](int m) { const int tw = (p + 1) * m, k = (nint + tw - 1) / tw; return (long long)k * k; };
    std::vector<SweepForm> cands;
    auto add = [&](SweepForm f) {
      if (f.lpr == 2 && mapped) return;                        // the split row has no third box
      if (f.tiles != 0 && (!has_pos || !tiles_ok)) return;
      if (f.tiles > 0 && (ntiles(f.tiles) > cap || ntiles(f.tiles) < 2)) return;
      if (f.tiles < 0 && pt.n_patches > 40000) return;         // one SM would be far too slow
      cands.push_back(f);
    };
    if (pin) {
      std::string w(pin);
      SweepForm f;
      if (w.rfind("lanes2", 0) == 0) f.lpr = 2;
      if (w.find("_b") != std::string::npos) f.tpb = std::atoi(w.c_str() + w.find("_b") + 2);
      if (w.find("_c2") != std::string::npos) f.ch = 2;
      else if (w == "solo") f.tiles = -1;
      else if (w.rfind("tiles", 0) == 0) f.tiles = std::max(1, std::atoi(w.c_str() + 5));
      add(f);
    } else if (env_lanes || env_mult) {                        // experiments: one form
      SweepForm f;
      if (env_mult && tiles_ok) f.tiles = std::max(1, std::atoi(env_mult));
      else if (env_lanes) f.lpr = std::atoi(env_lanes) == 2 ? 2 : 1;
      add(f);
      if (cands.empty() && f.tiles > 0) {                      // widen until the tiles fit
        for (int m = f.tiles + 1; m <= 4096 && cands.empty(); ++m) add(SweepForm{1, m});
      }
    } else {
      for (SweepForm f : {SweepForm{1, 0}, SweepForm{2, 0}, SweepForm{1, 0, 64}, SweepForm{2, 0, 64},
                          SweepForm{1, 0, 256}, SweepForm{1, 0, 0, 2}, SweepForm{1, 0, 64, 2}, SweepForm{1, 0, 256, 2},
                          SweepForm{1, -1}, SweepForm{1, 1}, SweepForm{1, 2}, SweepForm{1, 4}})
        add(f);
    }
    if (cands.empty()) cands.push_back(SweepForm{1, 0});
    // step counters sized for the most tiles any candidate has
    size_t nt_max = 1;
    for (auto& f : cands) if (f.tiles > 0) nt_max = std::max(nt_max, (size_t)ntiles(f.tiles));
    if (has_pos && tiles_ok) {
      for (int which = 0; which < 2; ++which) {
        if (which == 1 && !fp32_base(h->prob)) continue;
        unsigned** prog = which ? &h->f.lev[l].prog : &h->d.lev[l].prog;
        if ((rc = dmalloc(h, (void**)prog, nt_max * sizeof(unsigned)))) return rc;
        CK(cudaMemset(*prog, 0, nt_max * sizeof(unsigned)));
      }
    }
    const auto key = std::make_tuple(p, lc.sz.n, h->prob.beta_qp ? 1 : 0, mapped ? 1 : 0);
    SweepForm chosen = cands[0];
    if (cands.size() > 1) {
      bool cached = false;
      {
        std::lock_guard<std::mutex> lk(form_mutex());
        auto it = form_cache().find(key);
        if (it != form_cache().end()) { cached = true; chosen = it->second; }
      }
      if (!cached) {
        auto& tl = h->d.lev[l];
        const size_t nb = (size_t)tl.L.n_total * sizeof(double);
        CK(cudaMemsetAsync(tl.U, 0, nb, h->stream));
        CK(cudaMemsetAsync(tl.F, 0, nb, h->stream));
        float best = 1e30f;
        for (auto& f : cands) {
          if ((rc = apply_form(h, l, f))) return rc;
          float ms = 0;
          if ((rc = time_level_sweeps(h, l, &ms))) return rc;
          if (verbose) std::fprintf(stderr, "igamg: level %d (n = %d) %s: %.1f us per %d sweep(s)\n", l, lc.sz.n,
                                    form_name(f).c_str(), 1e3f * ms, std::max(1, h->prob.nu1));
          if (ms < best) { best = ms; chosen = f; }
        }
        std::lock_guard<std::mutex> lk(form_mutex());
        form_cache()[key] = chosen;
      }
    }
    if ((rc = apply_form(h, l, chosen))) return rc;
    if (h->d.lev[l].prog) {   // the timing runs advanced different tile sets: start from 0
      CK(cudaMemset(h->d.lev[l].prog, 0, nt_max * sizeof(unsigned)));
    }
    if (verbose) std::fprintf(stderr, "igamg: level %d (n = %d): %s\n", l, lc.sz.n, form_name(chosen).c_str());
  }
  return IGAMG_OK;
}

// Residual form of the finest generalized-Oseen level, per precision: the per-row records
// (Stokes part and advection in one stored record per row) or the advection applied
// matrix-free (k_residual_adv; the Stokes part from the class stencils).  Both are timed at
// creation (best of three runs of 20 launches on the level's zeroed workspaces) and the
// faster is kept; choices are cached per process by (p, n, precision).  IGAMG_ADV_FORM=records
// or =mf pins one.
std::map<std::tuple<int, int, int>, int>& adv_cache() {
  static std::map<std::tuple<int, int, int>, int> m;
  return m;
}

template <typename T>
int time_fine_residual(igamg_handle* h, float* ms_out) {
  auto& tl = typed<T>(h).lev.back();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int rc = IGAMG_OK;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < 4 && !rc && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, h->stream);
    for (int k = 0; k < 20 && !rc && e == cudaSuccess; ++k) rc = do_residual<T>(h, (int)h->lc.size() - 1, tl.U, tl.F, tl.R, h->norm2, h->stream);
    if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best = std::min(best, ms);          // the first run warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  CK(e);
  *ms_out = best / 20;
  return IGAMG_OK;
}

template <typename T>
int choose_adv_form(igamg_handle* h) {
  auto& ty = typed<T>(h);
  ty.adv_mf = 0;
  if (!ty.adv.beta) return IGAMG_OK;
  if (const char* pin = std::getenv("IGAMG_ADV_FORM")) {
    ty.adv_mf = std::string(pin) == "mf" ? 1 : 0;
    return IGAMG_OK;
  }
  const auto key = std::make_tuple(h->prob.p, h->prob.n_fine, (int)sizeof(T));
  {
    std::lock_guard<std::mutex> lk(form_mutex());
    auto it = adv_cache().find(key);
    if (it != adv_cache().end()) { ty.adv_mf = it->second; return IGAMG_OK; }
  }
  auto& tl = ty.lev.back();
  const size_t nb = (size_t)tl.L.n_total * sizeof(T);
  CK(cudaMemsetAsync(tl.U, 0, nb, h->stream));
  CK(cudaMemsetAsync(tl.F, 0, nb, h->stream));
  float ms[2];
  int rc;
  for (int f = 0; f < 2; ++f) {
    ty.adv_mf = f;
    if ((rc = time_fine_residual<T>(h, &ms[f]))) return rc;
  }
  ty.adv_mf = ms[1] < ms[0] ? 1 : 0;
  {
    std::lock_guard<std::mutex> lk(form_mutex());
    adv_cache()[key] = ty.adv_mf;
  }
  if (std::getenv("IGAMG_VERBOSE"))
    std::fprintf(stderr, "igamg: finest residual (%s): records %.1f us, matrix-free %.1f us -> %s\n",
                 sizeof(T) == 8 ? "FP64" : "FP32", 1e3f * ms[0], 1e3f * ms[1], ty.adv_mf ? "matrix-free" : "records");
  return IGAMG_OK;
}

bool any_3d(int n, igamg_handle** hs) {
  for (int i = 0; i < n; ++i) if (hs[i]->d3) return true;
  return false;
}

// Batches holding 3D handles run their solves one after another (each 3D solve already
// fills the GPU); the contract (statuses, reports, return value) is that of the 2D batch.
int batch_3d(int n, igamg_handle** hs, double** Us, const double** Fs, double rtol, const double* atol,
             int max_cycles, igamg_report* reps, int* status) {
  int worst = IGAMG_OK;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]->d3) return IGAMG_EUNSUPPORTED;   // 2D and 3D handles are not mixed in one batch
    int st = h3_solve(hs[i]->d3, Us[i], Fs[i], rtol, max_cycles, reps ? &reps[i] : nullptr, atol ? atol[i] : -1.0);
    if (status) status[i] = st;
    if (st < 0) return st;
    if (st == IGAMG_NOT_CONVERGED) worst = IGAMG_NOT_CONVERGED;
  }
  return worst;
}

int validate(const igamg_problem& pr) {
  if (pr.dim != 2) return IGAMG_EUNSUPPORTED;
  if (pr.p != 2 && pr.p != 3) return IGAMG_EUNSUPPORTED;
  if (pr.n_levels < 1 || pr.n_levels > 16 || pr.n_fine < 1) return IGAMG_EINVAL;
  if (pr.n_fine % (1 << (pr.n_levels - 1))) return IGAMG_EINVAL;
  if (!(pr.sigma > 0) || !(pr.nu > 0) || pr.nu1 < 0 || pr.nu2 < 0) return IGAMG_EINVAL;
  if (pr.smoother != IGAMG_MULT && pr.smoother != IGAMG_ADD) return IGAMG_EINVAL;
  if (pr.precision < IGAMG_FP64 || pr.precision > IGAMG_FGMRES_FP32) return IGAMG_EUNSUPPORTED;
  if (pr.gamma < 0 || pr.gamma > 4 || pr.fmg < 0 || pr.fmg > 1) return IGAMG_EINVAL;
  if (pr.fmg && pr.precision >= IGAMG_FGMRES_FP64) return IGAMG_EUNSUPPORTED;
  if (pr.geometry < IGAMG_GEOM_SQUARE || pr.geometry > IGAMG_GEOM_QUARTER_ANNULUS) return IGAMG_EINVAL;
  if (pr.geometry == IGAMG_GEOM_QUARTER_ANNULUS) {
    if (pr.beta_qp) return IGAMG_EUNSUPPORTED;                 // generalized Stokes only
    const double ri = pr.r_inner > 0 ? pr.r_inner : 0.075, ro = pr.r_outer > 0 ? pr.r_outer : 0.225;
    if (!(ri > 0) || !(ro > ri) || !std::isfinite(ro)) return IGAMG_EINVAL;
  }
  if (pr.n_fine > 8192) return IGAMG_EINVAL;
  // the coarsest grid is solved with a dense inverse held in shared memory by one block
  if (level_sizes(pr.p, pr.n_fine >> (pr.n_levels - 1)).n_total > 4096) return IGAMG_EINVAL;
  return IGAMG_OK;
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
  if (pr.dim == 3) {
    igamg3d_handle* h3 = nullptr;
    int rc3 = h3_create(prob, cuda_stream, &h3);
    if (rc3) return rc3;
    auto* h = new igamg_handle();
    h->prob = pr;
    h->stream = (cudaStream_t)cuda_stream;
    h->d3 = h3;
    *out = h;
    return IGAMG_OK;
  }
  int rc = validate(pr);
  if (rc) return rc;
  auto* h = new igamg_handle();
  h->prob = pr;
  h->stream = (cudaStream_t)cuda_stream;
  rc = build_hierarchy(pr, h->host, g_err);
  if (rc) {
    if (std::getenv("IGAMG_VERBOSE")) std::fprintf(stderr, "igamg: set-up failed (%d): %s\n", rc, g_err.c_str());
    delete h;
    return rc;
  }
  auto fail_at = [&](int code, int line) {
    if (std::getenv("IGAMG_VERBOSE")) std::fprintf(stderr, "igamg: create failed (%d) at igamg.cu:%d: %s\n", code, line, g_err.c_str());
    igamg_destroy(h);
    return code;
  };
#define fail(code) fail_at((code), __LINE__)
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(IGAMG_ECUDA);
  const int L = pr.n_levels, p = pr.p;
  h->lc.resize(L);
  size_t max_delta = 0;
  for (int l = 0; l < L; ++l) {
    auto& lh = h->host.lev[l];
    auto& lc = h->lc[l];
    lc.sz = lh.sz;
    if ((rc = upload_as(h, &lc.dcoef, lh.f.dcoef))) return fail(rc);
    std::vector<double> inv(lh.f.dcoef.size());
    for (size_t k = 0; k < inv.size(); ++k) inv[k] = 1.0 / lh.f.dcoef[k];
    if ((rc = upload_as(h, &lc.inv_dcoef, inv))) return fail(rc);
    if (l >= 1) {
      const auto& pt = lh.pt;
      lc.n_patches = pt.n_patches; lc.maxl = pt.maxl; lc.n_colours = pt.n_colours;
      lc.colour_off = pt.colour_off; lc.n8 = pt.n8;
      if ((rc = upload_as(h, &lc.dofs, pt.dofs)) || (rc = upload_as(h, &lc.cls, pt.cls)) ||
          (rc = upload_as(h, &lc.nloc, pt.nloc)) || (rc = upload_as(h, &lc.d2p_off, pt.d2p_off)) ||
          (rc = upload_as(h, &lc.d2p_idx, pt.d2p_idx)))
        return fail(rc);
      max_delta = std::max(max_delta, (size_t)pt.n_patches * pt.maxl);
    }
  }
  h->ndof0 = h->host.ndof0;
  if ((rc = upload_typed<double>(h, h->d, max_delta))) return fail(rc);
  if (fp32_base(pr) && (rc = upload_typed<float>(h, h->f, max_delta))) return fail(rc);
  // the matrix-free advection tables live on the device from here on (w * beta alone is
  // 2 (n (p+2))^2 doubles on the host)
  for (auto* v : {&h->host.adv_bp, &h->host.adv_dp, &h->host.adv_bq, &h->host.adv_dq, &h->host.adv_beta})
    std::vector<double>().swap(*v);
  h->ndof0 = h->host.ndof0;
  long long nfine = h->lc[L - 1].sz.n_total;
  if ((rc = dmalloc(h, (void**)&h->part, 2 * sizeof(double) * (nblk(nfine) + 1)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->norm2, 2 * sizeof(double)))) return fail(rc);
  if (cudaMemset(h->norm2, 0, 2 * sizeof(double)) != cudaSuccess) return fail(IGAMG_ECUDA);
  h->sweep_err = (int*)(h->norm2 + 1);
  if ((rc = dmalloc(h, (void**)&h->divmax, sizeof(unsigned long long)))) return fail(rc);
  if ((rc = upload_as(h, &h->lv_p, h->host.lv_p)) || (rc = upload_as(h, &h->lv_q, h->host.lv_q))) return fail(rc);
  if ((rc = setup_sweep_forms(h))) return fail(rc);
  if ((rc = choose_adv_form<double>(h))) return fail(rc);
  if (fp32_base(pr) && (rc = choose_adv_form<float>(h))) return fail(rc);
  size_t nG = (size_t)pr.n_fine * (p + 2);
  if ((rc = dmalloc(h, (void**)&h->f_dev, 2 * nG * nG * sizeof(double)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->Fh, nfine * sizeof(double)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->Uh, nfine * sizeof(double)))) return fail(rc);
  size_t nint = (size_t)(pr.n_fine + p - 2);
  if ((rc = dmalloc(h, (void**)&h->psi, nint * nint * sizeof(double)))) return fail(rc);
  if (cudaMallocHost((void**)&h->h_pinned, 2 * sizeof(double)) != cudaSuccess) return fail(IGAMG_ECUDA);
  if (!h->host.jt.empty() && (rc = upload_as(h, &h->jt, h->host.jt))) return fail(rc);
  if ((rc = autotune_fused<double>(h, h->d))) return fail(rc);
  if (fp32_base(pr) && (rc = autotune_fused<float>(h, h->f))) return fail(rc);
  if (pr.precision >= IGAMG_FGMRES_FP64 &&
      (rc = krylov_alloc(h->kw, pr.restart > 0 ? pr.restart : 20, nfine, h->allocs)))
    return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->zeros, nfine * sizeof(double)))) return fail(rc);
  if (cudaMemset(h->zeros, 0, nfine * sizeof(double)) != cudaSuccess) return fail(IGAMG_ECUDA);
  if ((rc = dmalloc(h, (void**)&h->dots, (5 * kDotGrid + 8) * sizeof(double)))) return fail(rc);
  if (cudaStreamCreateWithFlags(&h->exec_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(IGAMG_ECUDA);
  if (cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess) return fail(IGAMG_ECUDA);
  *out = h;
  return IGAMG_OK;
#undef fail
}

void igamg_destroy(igamg_handle* h) {
  if (!h) return;
  if (h->d3) h3_destroy(h->d3);
  krylov_free_host(h->kw);
  for (auto& g : h->graph) if (g) cudaGraphExecDestroy(g);
  batch_cache_free(h->bc);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->exec_stream) cudaStreamDestroy(h->exec_stream);
  if (h->ev) cudaEventDestroy(h->ev);
  delete h;
}

int igamg_get_sizes(const igamg_handle* h, int level, igamg_sizes* out) {
  if (h && out && h->d3) return h3_sizes(h->d3, level, out);
  if (!h || !out || level < 0 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  *out = h->lc[level].sz;
  return IGAMG_OK;
}

int igamg_quad_points(const igamg_handle* h, double* x, size_t cap, size_t* n_out) {
  if (!h || !n_out) return IGAMG_EINVAL;
  const std::vector<double>& qx = h->d3 ? h3_quad_x(h->d3) : h->host.quad_x;
  *n_out = qx.size();
  if (x) {
    if (cap < qx.size()) return IGAMG_EINVAL;
    std::memcpy(x, qx.data(), qx.size() * sizeof(double));
  }
  return IGAMG_OK;
}

int igamg_load_vector(igamg_handle* h, const double* f_qp, double* F) {
  if (!h || !f_qp || !F) return IGAMG_EINVAL;
  if (h->d3) return h3_load_vector(h->d3, f_qp, F);
  auto& Lt = h->d.lev.back().L;
  if (h->jt) {                                       // mapped domain: load J^T f
    const int npts = h->prob.n_fine * (h->prob.p + 2) * h->prob.n_fine * (h->prob.p + 2);
    k_pullback<<<nblk(npts), kBlock, 0, h->stream>>>(npts, h->jt, f_qp, h->f_dev);
    f_qp = h->f_dev;
  }
  if (h->prob.p == 2) k_load<2><<<nblk(Lt.n_total), kBlock, 0, h->stream>>>(Lt, h->lv_p, h->lv_q, f_qp, F);
  else k_load<3><<<nblk(Lt.n_total), kBlock, 0, h->stream>>>(Lt, h->lv_p, h->lv_q, f_qp, F);
  return launch_check();
}

int igamg_quad_points_xy(const igamg_handle* h, double* xy, size_t cap, size_t* n_out) {
  if (!h || !n_out) return IGAMG_EINVAL;
  if (h->d3) {                                       // (3, nG, nG, nG) [x, y or z][z][y][x]
    const std::vector<double>& qx = h3_quad_x(h->d3);
    const std::vector<double>& q3 = h3_quad_xyz(h->d3);
    const size_t nG = qx.size(), np = nG * nG * nG;
    *n_out = 3 * np;
    if (!xy) return IGAMG_OK;
    if (cap < 3 * np) return IGAMG_EINVAL;
    if (!q3.empty()) { std::memcpy(xy, q3.data(), 3 * np * sizeof(double)); return IGAMG_OK; }
    for (size_t iz = 0; iz < nG; ++iz)
      for (size_t iy = 0; iy < nG; ++iy)
        for (size_t ix = 0; ix < nG; ++ix) {
          const size_t o = (iz * nG + iy) * nG + ix;
          xy[o] = qx[ix]; xy[np + o] = qx[iy]; xy[2 * np + o] = qx[iz];
        }
    return IGAMG_OK;
  }
  const std::vector<double>& qx = h->host.quad_x;
  const size_t nG = qx.size();
  *n_out = 2 * nG * nG;
  if (!xy) return IGAMG_OK;
  if (cap < 2 * nG * nG) return IGAMG_EINVAL;
  if (!h->host.quad_xy.empty()) {
    std::memcpy(xy, h->host.quad_xy.data(), 2 * nG * nG * sizeof(double));
  } else {
    for (size_t iy = 0; iy < nG; ++iy)
      for (size_t ix = 0; ix < nG; ++ix) { xy[iy * nG + ix] = qx[ix]; xy[nG * nG + iy * nG + ix] = qx[iy]; }
  }
  return IGAMG_OK;
}

int igamg_residual(igamg_handle* h, int level, const double* U, const double* F, double* R, double* norm_out) {
  if (h && U && F && R && h->d3) return h3_residual(h->d3, level, U, F, R, norm_out);
  if (!h || !U || !F || !R || level < 0 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  int rc = do_residual<double>(h, level, U, F, R, h->norm2, h->stream);
  if (rc) return rc;
  if (norm_out) return read_norm(h, norm_out);
  return IGAMG_OK;
}

int igamg_smooth(igamg_handle* h, int level, double* U, const double* F, int sweeps) {
  if (h && U && F && h->d3) return h3_smooth(h->d3, level, U, F, sweeps);
  if (!h || !U || !F || level < 1 || level >= (int)h->lc.size() || sweeps < 0) return IGAMG_EINVAL;
  return do_smooth_n<double>(h, level, U, F, sweeps, h->stream);
}

int igamg_level_form(const igamg_handle* h, int level, int* lanes, int* threads, int* tiles) {
  if (!h || level < 0) return IGAMG_EINVAL;
  if (h->d3) return IGAMG_EUNSUPPORTED;
  if (level >= (int)h->lc.size()) return IGAMG_EINVAL;
  const auto& lc = h->lc[level];
  const bool tiled = lc.ntx > 0;
  if (lanes) *lanes = tiled ? 1 : lc.lpr;
  if (threads) *threads = tiled ? (lc.ntx * lc.nty == 1 ? kSoloThreads : kTileThreads) : (lc.tpb > 0 ? lc.tpb : colour_block());
  if (tiles) *tiles = tiled ? lc.ntx * lc.nty : 0;
  return IGAMG_OK;
}

int igamg_residual_f32(igamg_handle* h, int level, const float* U, const float* F, float* R, double* norm_out) {
  if (!h || !U || !F || !R) return IGAMG_EINVAL;
  if (h->d3 || !fp32_base(h->prob)) return IGAMG_EUNSUPPORTED;
  if (level < 0 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  int rc = do_residual<float>(h, level, U, F, R, h->norm2, h->stream);
  if (rc) return rc;
  if (norm_out) return read_norm(h, norm_out);
  return IGAMG_OK;
}

int igamg_residual_form(const igamg_handle* h, int* form64, int* form32) {
  if (!h) return IGAMG_EINVAL;
  if (h->d3) return IGAMG_EUNSUPPORTED;
  if (form64) *form64 = h->d.adv.beta ? (h->d.adv_mf ? 2 : 1) : 0;
  if (form32) *form32 = !fp32_base(h->prob) ? -1 : (h->f.adv.beta ? (h->f.adv_mf ? 2 : 1) : 0);
  return IGAMG_OK;
}

int igamg_set_residual_form(igamg_handle* h, int form64, int form32) {
  if (!h || form64 < 0 || form64 > 2 || form32 < 0 || form32 > 2) return IGAMG_EINVAL;
  if (h->d3) return IGAMG_EUNSUPPORTED;
  if (form64 && !h->d.adv.beta) return IGAMG_EUNSUPPORTED;
  if (form32 && (!fp32_base(h->prob) || !h->f.adv.beta)) return IGAMG_EUNSUPPORTED;
  // the captured solve graphs hold the old form's launches: drop them (re-captured on use)
  CK(cudaStreamSynchronize(h->stream));
  if (h->exec_stream) CK(cudaStreamSynchronize(h->exec_stream));
  for (int k = 0; k < 3; ++k)
    if (h->graph[k]) { cudaGraphExecDestroy(h->graph[k]); h->graph[k] = nullptr; h->gU[k] = h->gF[k] = nullptr; }
  if (form64) h->d.adv_mf = form64 == 2 ? 1 : 0;
  if (form32) h->f.adv_mf = form32 == 2 ? 1 : 0;
  return IGAMG_OK;
}

int igamg_level_chains(const igamg_handle* h, int level, int* chains) {
  if (!h || level < 0 || !chains) return IGAMG_EINVAL;
  if (h->d3) return IGAMG_EUNSUPPORTED;
  if (level >= (int)h->lc.size()) return IGAMG_EINVAL;
  *chains = h->lc[level].ch;
  return IGAMG_OK;
}

int igamg_smooth_f32(igamg_handle* h, int level, float* U, const float* F, int sweeps) {
  if (!h || !U || !F || sweeps < 0) return IGAMG_EINVAL;
  if (h->d3 || !fp32_base(h->prob)) return IGAMG_EUNSUPPORTED;
  if (level < 1 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  return do_smooth_n<float>(h, level, U, F, sweeps, h->stream);
}

int igamg_restrict(igamg_handle* h, int level, const double* r_fine, double* g_coarse) {
  if (h && r_fine && g_coarse && h->d3) return h3_restrict(h->d3, level, r_fine, g_coarse);
  if (!h || !r_fine || !g_coarse || level < 1 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  return do_restrict<double>(h, level, r_fine, g_coarse, h->stream);
}

int igamg_prolong_add(igamg_handle* h, int level, const double* u_coarse, double* u_fine) {
  if (h && u_coarse && u_fine && h->d3) return h3_prolong_add(h->d3, level, u_coarse, u_fine);
  if (!h || !u_coarse || !u_fine || level < 1 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  return do_prolong<double>(h, level, u_coarse, u_fine, h->stream);
}

int igamg_coarse_solve(igamg_handle* h, const double* G, double* U) {
  if (!h || !G || !U) return IGAMG_EINVAL;
  if (h->d3) return h3_coarse_solve(h->d3, G, U);
  return do_coarse<double>(h, G, U, h->stream);
}

int igamg_vcycle(igamg_handle* h, double* U, const double* F) {
  if (!h || !U || !F) return IGAMG_EINVAL;
  if (h->d3) return h3_vcycle(h->d3, U, F);
  int rc = ensure_graph(h, 1, U, F);
  if (rc) return rc;
  CK(cudaGraphLaunch(h->graph[1], h->stream));
  return IGAMG_OK;
}

int igamg_solve(igamg_handle* h, double* U, const double* F, double rtol, int max_cycles, igamg_report* rep) {
  if (!h || !U || !F || !(rtol >= 0) || max_cycles < 0) return IGAMG_EINVAL;
  if (h->d3) return h3_solve(h->d3, U, F, rtol, max_cycles, rep, -1.0);
  return solve_impl(h, U, F, rtol, max_cycles, rep, -1.0);
}

int igamg_solve_host(igamg_handle* h, const double* f_qp_host, double* U_host, double rtol, int max_cycles,
                     igamg_report* rep) {
  if (!h || !f_qp_host || !U_host || !(rtol >= 0) || max_cycles < 0) return IGAMG_EINVAL;
  if (h->d3) return h3_solve_host(h->d3, f_qp_host, U_host, rtol, max_cycles, rep);
  size_t nG = (size_t)h->prob.n_fine * (h->prob.p + 2);
  size_t nt = (size_t)h->lc.back().sz.n_total;
  CK(cudaMemcpyAsync(h->f_dev, f_qp_host, 2 * nG * nG * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->Uh, U_host, nt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  int rc = igamg_load_vector(h, h->f_dev, h->Fh);
  if (rc) return rc;
  int st = solve_impl(h, h->Uh, h->Fh, rtol, max_cycles, rep, -1.0);
  if (st < 0) return st;
  CK(cudaMemcpyAsync(U_host, h->Uh, nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return st;
}

int igamg_solve_batch(int n, igamg_handle** handles, double** U, const double** F, double rtol, int max_cycles,
                      igamg_report* reports, int* status) {
  if (n < 0 || (n > 0 && (!handles || !U || !F)) || !(rtol >= 0) || max_cycles < 0) return IGAMG_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!handles[i] || !U[i] || !F[i]) return IGAMG_EINVAL;
    for (int j = 0; j < i; ++j) if (handles[j] == handles[i]) return IGAMG_EINVAL;
  }
  if (any_3d(n, handles)) return batch_3d(n, handles, U, F, rtol, nullptr, max_cycles, reports, status);
  return solve_batch_impl(n, handles, U, F, rtol, max_cycles, reports, status);
}

int igamg_solve_abs(igamg_handle* h, double* U, const double* F, double atol, int max_cycles, igamg_report* rep) {
  if (!h || !U || !F || !(atol >= 0) || max_cycles < 0) return IGAMG_EINVAL;
  if (h->d3) return h3_solve(h->d3, U, F, 0.0, max_cycles, rep, atol);
  return solve_impl(h, U, F, 0.0, max_cycles, rep, atol);
}

int igamg_solve_batch_abs(int n, igamg_handle** handles, double** U, const double** F, const double* atol,
                          int max_cycles, igamg_report* reports, int* status) {
  if (n < 0 || (n > 0 && (!handles || !U || !F || !atol)) || max_cycles < 0) return IGAMG_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!handles[i] || !U[i] || !F[i] || !(atol[i] >= 0)) return IGAMG_EINVAL;
    for (int j = 0; j < i; ++j) if (handles[j] == handles[i]) return IGAMG_EINVAL;
  }
  if (any_3d(n, handles)) return batch_3d(n, handles, U, F, 0.0, atol, max_cycles, reports, status);
  return solve_batch_impl(n, handles, U, F, 0.0, max_cycles, reports, status, atol);
}

int igamg_div_inf(igamg_handle* h, const double* U, double* out) {
  if (!h || !U || !out) return IGAMG_EINVAL;
  if (h->d3) return h3_div_inf(h->d3, U, out);
  return div_inf_impl(h, U, out);
}

int igamg_streamfunction(igamg_handle* h, const double* U, double* psi) {
  if (!h || !U || !psi) return IGAMG_EINVAL;
  if (h->d3) return IGAMG_EUNSUPPORTED;
  auto& Lt = h->d.lev.back().L;
  k_streamfunction<<<nblk((long long)Lt.nint * 32, 128), 128, 0, h->stream>>>(Lt.nint, Lt.nxu, h->lc.back().inv_dcoef, U, psi);
  return launch_check();
}

int igamg_warm_start(igamg_handle* h, const float* grid, double psi_scale, double p_scale, double* U) {
  if (!h || !grid || !U) return IGAMG_EINVAL;
  if (h->d3) return IGAMG_EUNSUPPORTED;
  auto& Lt = h->d.lev.back().L;
  k_grid_to_psi<<<nblk((long long)Lt.nint * Lt.nint), kBlock, 0, h->stream>>>(Lt.nint, grid, psi_scale, h->psi);
  CK(cudaMemsetAsync(U, 0, Lt.n_total * sizeof(double), h->stream));
  k_curl<<<nblk(Lt.n_ux + Lt.n_uy), kBlock, 0, h->stream>>>(Lt, h->lc.back().dcoef, h->psi, U);
  const int H = Lt.nint + 2;
  k_grid_to_pressure<<<nblk(Lt.n_p), kBlock, 0, h->stream>>>(Lt.npd, grid + (size_t)H * H, H, p_scale,
                                                              U + Lt.n_ux + Lt.n_uy);
  return launch_check();
}

int igamg_warm_start_minres(igamg_handle* h, const float* grid, double psi_scale, double p_scale, const double* F,
                            double* U, double* alpha_out, double* beta_out) {
  if (!h || !grid || !F || !U) return IGAMG_EINVAL;
  if (h->d3) return IGAMG_EUNSUPPORTED;
  const int L = (int)h->d.lev.size();
  auto& Lt = h->d.lev.back().L;
  cudaStream_t s = h->stream;
  const int n = Lt.n_total, nu = Lt.n_ux + Lt.n_uy;
  double* Z = h->Fh;                    // the predicted pressure as a vector (velocity 0)
  double* W1 = h->Uh;                   // -K u
  double* W2 = h->d.lev[L - 1].R;       // -K Z
  k_grid_to_psi<<<nblk((long long)Lt.nint * Lt.nint), kBlock, 0, s>>>(Lt.nint, grid, psi_scale, h->psi);
  CK(cudaMemsetAsync(U, 0, n * sizeof(double), s));
  k_curl<<<nblk(nu), kBlock, 0, s>>>(Lt, h->lc.back().dcoef, h->psi, U);
  CK(cudaMemsetAsync(Z, 0, n * sizeof(double), s));
  const int H = Lt.nint + 2;
  k_grid_to_pressure<<<nblk(Lt.n_p), kBlock, 0, s>>>(Lt.npd, grid + (size_t)H * H, H, p_scale, Z + nu);
  int rc = launch_check();
  if (rc) return rc;
  if ((rc = do_residual<double>(h, L - 1, U, h->zeros, W1, nullptr, s))) return rc;
  if ((rc = do_residual<double>(h, L - 1, Z, h->zeros, W2, nullptr, s))) return rc;
  k_dots5<<<kDotGrid, 256, 0, s>>>(n, F, W1, W1, W1, F, W2, W1, W2, W2, W2, h->dots);
  k_dots5_finish<<<1, 32, 0, s>>>(kDotGrid, h->dots, h->dots + 5 * kDotGrid);
  if ((rc = launch_check())) return rc;
  double d[5];
  CK(cudaMemcpyAsync(d, h->dots + 5 * kDotGrid, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // (alpha, beta) minimise |F + alpha W1 + beta W2|^2 = |F - K(alpha u + beta Z)|^2:
  // normal equations [W1.W1 W1.W2; W1.W2 W2.W2] (alpha, beta) = -(F.W1, F.W2).
  // alpha = beta = 0 is admissible, so the first residual is never larger than |F|.
  const double a11 = d[1], a12 = d[3], a22 = d[4], r1 = -d[0], r2 = -d[2];
  const double det = a11 * a22 - a12 * a12;
  double alpha = 0.0, beta = 0.0;
  if (det > 1e-14 * a11 * a22) {
    alpha = (r1 * a22 - r2 * a12) / det;
    beta = (a11 * r2 - a12 * r1) / det;
  } else if (a11 > 0.0) {               // the two directions are (nearly) parallel
    alpha = r1 / a11;
  }
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return IGAMG_ENONFINITE;
  k_axpby<<<nblk(n), kBlock, 0, s>>>(n, alpha, beta, Z, U);
  if ((rc = launch_check())) return rc;
  if (alpha_out) *alpha_out = alpha;
  if (beta_out) *beta_out = beta;
  return IGAMG_OK;
}

int igamg_curl(igamg_handle* h, const double* psi, double* U) {
  if (!h || !psi || !U) return IGAMG_EINVAL;
  if (h->d3) return h3_curl(h->d3, psi, U);
  auto& Lt = h->d.lev.back().L;
  k_curl<<<nblk(Lt.n_ux + Lt.n_uy), kBlock, 0, h->stream>>>(Lt, h->lc.back().dcoef, psi, U);
  return launch_check();
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Residual entry point that allocates no device memory.
//
// For callers that cannot call cudaMalloc (a host program whose allocations all go
// through its own pool or arena, or an embedding that owns the whole device memory
// budget): the scratch of the residual kernel -- its level operator tables and its
// per-block partial sums -- lives in one fixed array in device memory that the library
// declares statically.  Every GPU that loads the library holds that array (1 MiB) until
// the process exits.
// ---------------------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchDoubles = 131072;  // 1 MiB
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_static_ptr[kMaxDevices] = {};
std::mutex g_static_mutex;                        // guards the first lookup per device

}  // namespace

extern "C" int igamg_residual_static(const igamg_problem* prob, int level, const double* U,
                                     const double* F, double* R, double* norm_out,
                                     void* cuda_stream) {
  if (!prob || !U || !F || !R) return IGAMG_EINVAL;
  const igamg_problem& pr = *prob;
  if (pr.dim != 2 || (pr.p != 2 && pr.p != 3) || pr.beta_qp || pr.geometry != IGAMG_GEOM_SQUARE)
    return IGAMG_EUNSUPPORTED;                                // Stokes on the unit square only
  if (pr.n_levels < 1 || pr.n_levels > 16 || pr.n_fine < 1 || pr.n_fine > 8192) return IGAMG_EINVAL;
  if (pr.n_fine % (1 << (pr.n_levels - 1))) return IGAMG_EINVAL;
  if (level < 0 || level >= pr.n_levels || !(pr.sigma > 0) || !(pr.nu > 0)) return IGAMG_EINVAL;
  const int p = pr.p, n = pr.n_fine >> (pr.n_levels - 1 - level);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  {
    // the tables go up through a pageable host copy that is freed on return, and norm_out
    // synchronises the stream: neither is valid while the stream is being captured
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
      g_err = "igamg_residual_static: the stream is being captured";
      return IGAMG_EUNSUPPORTED;
    }
  }

  // size check before any work: class stencil tables + partials + the norm slot
  igamg_sizes sz = level_sizes(p, n);
  const int TC = 2 * p + 1, NC = 2 * TC + 1;
  const size_t RU = (size_t)(2 * p + 1) * (2 * p - 1) + (size_t)2 * p * (2 * p - 1) + 1;
  const size_t n_tab = (size_t)NC * NC * 3 * RU;
  const unsigned nb = nblk(sz.n_total - 1);
  const size_t need = n_tab + 2 * (size_t)nb + 1;
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
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mutex);
    if (!g_static_ptr[dev]) {
      double* ptr = nullptr;
      CK(cudaGetSymbolAddress((void**)&ptr, g_static_scratch));
      g_static_ptr[dev] = ptr;
    }
    scratch = g_static_ptr[dev];
  }

  // this level's class stencils (host), copied into the front of the static array
  Level1D f;
  const double cpen = pr.c_penalty > 0 ? pr.c_penalty : 4.0 * (p - 1);
  build_level1d(p, n, pr.sigma, pr.nu, cpen * pr.n_fine, f);
  Stencils st;
  build_stencils(p, f, sz, st);
  std::vector<double> tab;
  tab.reserve(n_tab);
  tab.insert(tab.end(), st.sx.begin(), st.sx.end());
  tab.insert(tab.end(), st.sy.begin(), st.sy.end());
  tab.insert(tab.end(), st.sp.begin(), st.sp.end());
  if (tab.size() != n_tab) return IGAMG_EINVAL;
  CK(cudaMemcpyAsync(scratch, tab.data(), n_tab * sizeof(double), cudaMemcpyHostToDevice, s));
  LevelTab<double> L = make_tab<double>(sz, p, scratch, scratch + st.sx.size(), scratch + st.sx.size() + st.sy.size());
  double* part = scratch + n_tab;         // fully rewritten by every call
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

// Host-only: K_l rebuilt column by column through the same row evaluation the kernels
// use (class stencils, clamped neighbour indices), for checking the tables on a CPU.
extern "C" int igamg_host_operator_rows(const igamg_problem* prob, int level, double* K, size_t cap,
                                        long long* n_out) {
  if (!prob) return IGAMG_EINVAL;
  if (prob->dim == 3) return host_operator_rows3(prob, level, K, cap, n_out);
  int rc = validate(*prob);
  if (rc) return rc;
  if (level < 0 || level >= prob->n_levels) return IGAMG_EINVAL;
  HierarchyHost H;
  std::string err;
  if ((rc = build_hierarchy(*prob, H, err))) return rc;
  const auto& lh = H.lev[level];
  LevelTab<double> L = make_tab<double>(lh.sz, prob->p, lh.st.sx.data(), lh.st.sy.data(), lh.st.sp.data(),
                                        lh.rows.empty() ? nullptr : lh.rows.data(),
                                        lh.ext.empty() ? nullptr : lh.ext.data());
  long long n = lh.sz.n_total;
  if (n_out) *n_out = n;
  if (!K) return IGAMG_OK;
  if (cap < (size_t)(n * n)) return IGAMG_EINVAL;
  std::vector<double> e(n, 0.0);
  for (long long j = 0; j < n; ++j) {
    e[j] = 1.0;
    for (long long i = 0; i + 1 < n; ++i)
      K[i * n + j] = prob->p == 2 ? row_KU<2, double>(L, e.data(), (int)i) : row_KU<3, double>(L, e.data(), (int)i);
    double lam = 0.0;  // lambda row: m . p
    for (long long i = lh.sz.n_ux + lh.sz.n_uy; i + 1 < n; ++i) {
      int r = (int)(i - lh.sz.n_ux - lh.sz.n_uy);
      int ky = r / L.npd, kx = r - ky * L.npd;
      lam += lh.f.mq[kx] * lh.f.mq[ky] * e[i];
    }
    K[(n - 1) * n + j] = lam;
    e[j] = 0.0;
  }
  return IGAMG_OK;
}

// Host-only: KV = K_l V through the same row evaluation the kernels use.
extern "C" int igamg_host_operator_apply(const igamg_problem* prob, int level, const double* V, double* KV,
                                         size_t n) {
  if (!prob || !V || !KV) return IGAMG_EINVAL;
  if (prob->dim == 3) return host_operator_apply3(prob, level, V, KV, n);
  int rc = validate(*prob);
  if (rc) return rc;
  if (level < 0 || level >= prob->n_levels) return IGAMG_EINVAL;
  HierarchyHost H;
  std::string err;
  if ((rc = build_hierarchy(*prob, H, err))) return rc;
  const auto& lh = H.lev[level];
  if (n != (size_t)lh.sz.n_total) return IGAMG_EINVAL;
  LevelTab<double> L = make_tab<double>(lh.sz, prob->p, lh.st.sx.data(), lh.st.sy.data(), lh.st.sp.data(),
                                        lh.rows.empty() ? nullptr : lh.rows.data(),
                                        lh.ext.empty() ? nullptr : lh.ext.data());
  double lam = 0.0;
  for (size_t i = 0; i + 1 < n; ++i) {
    KV[i] = prob->p == 2 ? row_KU<2, double>(L, V, (int)i) : row_KU<3, double>(L, V, (int)i);
    if ((long long)i >= lh.sz.n_ux + lh.sz.n_uy) {
      int r = (int)(i - lh.sz.n_ux - lh.sz.n_uy);
      int ky = r / L.npd, kx = r - ky * L.npd;
      lam += lh.f.mq[kx] * lh.f.mq[ky] * V[i];
    }
  }
  KV[n - 1] = lam;
  return IGAMG_OK;
}
