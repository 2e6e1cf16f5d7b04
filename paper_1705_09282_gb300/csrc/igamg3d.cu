// Launch orchestration of the 3D (unit cube) V-cycle: Algorithm 1 with the multiplicative
// Schwarz smoother over vector-potential supports (Sec. 5.2), one launch per patch
// colour (3 p (p+1)^2 colours: per family strides p along its own axis and p+1 across),
// captured into CUDA graphs like the 2D path.  The C-ABI entry points in igamg.cu forward
// here for handles built with dim = 3.
//
// FP32 mode: each FP64 refinement step runs an FP32 V-cycle on the FP64 residual and adds
// the exact FP64 curl of a vector potential of its velocity correction, so every iterate
// stays divergence-free to FP64 round-off.  The vector potential of a divergence-free e
// (Sec. 4.3 complex, curl onto the divergence-free velocities) is built by integration:
//   psi_x = int_0^z e_y dz,  psi_y = -int_0^z e_x dz  (vanishing on z = 0), and, to cancel
//   their values on z = 1 (where psi x n = 0 is required), psi_z on the top element layer
//   = the 2D streamfunction chi of the depth totals, chi = -int_0^y (int_0^1 e_x dz) dy.
// In coefficients every integral is a prefix sum divided by the derivative coefficients.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "igamg3d.h"
#include "igamg_internal.h"
#include "kernels3d.cuh"
#include "krylov.h"

using namespace igamg;
using namespace igamg::dev;

namespace {

constexpr int kBlock = 256;
inline unsigned nblk(long long n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

// F = (int v.f, 0, 0) on the finest level; f at the quadrature points, (3, nG, nG, nG).
template <int P>
__global__ void k_load3(LevelTab3<double> L, const double* __restrict__ lvp, const double* __restrict__ lvq,
                        const double* __restrict__ f, double* __restrict__ F) {
  constexpr int Q = P - 1, G = P + 2;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_total) return;
  if (g >= L.n_u) { F[g] = 0.0; return; }
  int kind, i[3];
  decode3(L, g, kind, i[0], i[1], i[2]);
  const int n = L.n, nG = n * G;
  const double* fc = f + (size_t)kind * nG * nG * nG;
  int d[3];
  const double* tb[3];
  for (int a = 0; a < 3; ++a) { d[a] = a == kind ? P : Q; tb[a] = a == kind ? lvp : lvq; }
  double acc = 0.0;
  for (int kz = 0; kz <= d[2]; ++kz) {
    int ez = i[2] - d[2] + kz;
    if (ez < 0 || ez >= n) continue;
    const double* wz = tb[2] + ((size_t)i[2] * (d[2] + 1) + kz) * G;
    for (int ky = 0; ky <= d[1]; ++ky) {
      int ey = i[1] - d[1] + ky;
      if (ey < 0 || ey >= n) continue;
      const double* wy = tb[1] + ((size_t)i[1] * (d[1] + 1) + ky) * G;
      for (int kx = 0; kx <= d[0]; ++kx) {
        int ex = i[0] - d[0] + kx;
        if (ex < 0 || ex >= n) continue;
        const double* wx = tb[0] + ((size_t)i[0] * (d[0] + 1) + kx) * G;
        double sz = 0.0;
        for (int gz = 0; gz < G; ++gz) {
          double sy = 0.0;
          for (int gy = 0; gy < G; ++gy) {
            const double* row = fc + ((size_t)(ez * G + gz) * nG + (ey * G + gy)) * nG + ex * G;
            double sx = 0.0;
            for (int gx = 0; gx < G; ++gx) sx = fma(wx[gx], row[gx], sx);
            sy = fma(wy[gy], sx, sy);
          }
          sz = fma(wz[gz], sy, sz);
        }
        acc += sz;
      }
    }
  }
  F[g] = acc;
}

// full-index value of velocity component c (zero on the boundary indices of its own axis)
__device__ __forceinline__ double uval(const LevelTab3<double>& L, const double* U, int c, int x, int y, int z) {
  int own = sel3(c, x, y, z);
  if (own < 1 || own > L.ni) return 0.0;
  int dx = c == 0 ? L.ni : L.nq, dy = c == 1 ? L.ni : L.nq;
  x -= c == 0; y -= c == 1; z -= c == 2;
  return U[(size_t)c * L.n_uc + ((size_t)z * dy + y) * dx + x];
}

// max over the nq^3 pressure-space coefficients of |div u| (order-free max via bits)
__global__ void k_div_inf3(LevelTab3<double> L, const double* __restrict__ dcoef, const double* __restrict__ U,
                           unsigned long long* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (k < L.n_p) {
    int x = k % L.nq, t = k / L.nq, y = t % L.nq, z = t / L.nq;
    double c = dcoef[x] * (uval(L, U, 0, x + 1, y, z) - uval(L, U, 0, x, y, z)) +
               dcoef[y] * (uval(L, U, 1, x, y + 1, z) - uval(L, U, 1, x, y, z)) +
               dcoef[z] * (uval(L, U, 2, x, y, z + 1) - uval(L, U, 2, x, y, z));
    v = fabs(c);
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// vector potential families on the constrained space (zero outside the free ranges):
//   x: (z 1..ni, y 1..ni, x 0..nq-1), y: (z 1..ni, y 0..nq-1, x 1..ni), z: (z 0..nq-1, y 1..ni, x 1..ni)
struct Psi3 {
  const double* p;
  int ni, nq;
  __device__ double fx(int x, int y, int z) const {
    if (y < 1 || y > ni || z < 1 || z > ni) return 0.0;
    return p[((size_t)(z - 1) * ni + (y - 1)) * nq + x];
  }
  __device__ double fy(int x, int y, int z) const {
    if (x < 1 || x > ni || z < 1 || z > ni) return 0.0;
    return p[(size_t)nq * ni * ni + ((size_t)(z - 1) * nq + y) * ni + (x - 1)];
  }
  __device__ double fz(int x, int y, int z) const {
    if (x < 1 || x > ni || y < 1 || y > ni) return 0.0;
    return p[(size_t)2 * nq * ni * ni + ((size_t)z * ni + (y - 1)) * ni + (x - 1)];
  }
};

// velocity = curl psi (ADD = false), or U += (curl psi, e_p, e_lambda) (ADD = true)
template <bool ADD>
__global__ void k_curl3(LevelTab3<double> L, const double* __restrict__ dcoef, const double* __restrict__ psi,
                        const float* __restrict__ e, double* __restrict__ U) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (ADD ? L.n_total : L.n_u)) return;
  if (g >= L.n_u) { U[g] += (double)e[g]; return; }
  int kind, x, y, z;
  decode3(L, g, kind, x, y, z);
  Psi3 S{psi, L.ni, L.nq};
  double v;
  if (kind == 0)       // d psi_z/dy - d psi_y/dz
    v = dcoef[y] * (S.fz(x, y + 1, z) - S.fz(x, y, z)) - dcoef[z] * (S.fy(x, y, z + 1) - S.fy(x, y, z));
  else if (kind == 1)  // d psi_x/dz - d psi_z/dx
    v = dcoef[z] * (S.fx(x, y, z + 1) - S.fx(x, y, z)) - dcoef[x] * (S.fz(x + 1, y, z) - S.fz(x, y, z));
  else                 // d psi_y/dx - d psi_x/dy
    v = dcoef[x] * (S.fy(x + 1, y, z) - S.fy(x, y, z)) - dcoef[y] * (S.fx(x, y + 1, z) - S.fx(x, y, z));
  if (ADD) U[g] += v; else U[g] = v;
}

// Vector potential of a divergence-free correction e (FP32 in, FP64 out), part 1: the
// z-integrals.  Threads [0, ni*nq): psi_x columns (y 1..ni, x 0..nq-1) from e_y; threads
// [ni*nq, 2 ni*nq): psi_y columns (y 0..nq-1, x 1..ni) from e_x, and their depth totals.
__global__ void k_lift3_z(LevelTab3<float> L, const double* __restrict__ inv_dcoef, const float* __restrict__ e,
                          double* __restrict__ psi, double* __restrict__ tot) {
  const int ni = L.ni, nq = L.nq, ncol = ni * nq;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * ncol) return;
  if (t < ncol) {
    int y = t / nq + 1, x = t - (y - 1) * nq;                       // psi_x column
    const float* ey = e + L.n_uc;                                   // (z nq, y ni, x nq)
    double* out = psi;
    double run = 0.0;
    for (int k = 0; k < ni; ++k) {                                  // psi_x(z = k+1) = sum_{j <= k}
      run = fma((double)ey[((size_t)k * ni + (y - 1)) * nq + x], inv_dcoef[k], run);
      out[((size_t)k * ni + (y - 1)) * nq + x] = run;
    }
  } else {
    t -= ncol;
    int y = t / ni, x = t - y * ni + 1;                             // psi_y column
    const float* ex = e;                                            // (z nq, y nq, x ni)
    double* out = psi + (size_t)nq * ni * ni;
    double run = 0.0;
    for (int k = 0; k < nq; ++k) {
      run = fma(-(double)ex[((size_t)k * nq + y) * ni + (x - 1)], inv_dcoef[k], run);
      if (k < ni) out[((size_t)k * nq + y) * ni + (x - 1)] = run;
    }
    tot[(size_t)y * ni + (x - 1)] = run;                            // psi_y on z = 1 (to cancel)
  }
}

// part 2: psi_z on the top element layer = dcoef_{nq-1} chi, chi(y) = -sum_{j<y} tot(j) / dcoef_j;
// psi_z is zero on every other layer.  One thread per x in 1..ni.
__global__ void k_lift3_chi(int ni, int nq, const double* __restrict__ dcoef, const double* __restrict__ inv_dcoef,
                            const double* __restrict__ tot, double* __restrict__ psi) {
  int x = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (x > ni) return;
  double* pz = psi + (size_t)2 * nq * ni * ni + (size_t)(nq - 1) * ni * ni;
  double chi = 0.0;
  for (int y = 1; y <= ni; ++y) {
    chi = fma(-tot[(size_t)(y - 1) * ni + (x - 1)], inv_dcoef[y - 1], chi);
    pz[(size_t)(y - 1) * ni + (x - 1)] = dcoef[nq - 1] * chi;
  }
}

template <typename T>
struct Lev3T {
  LevelTab3<T> L{};
  T *cinv = nullptr, *cinv8 = nullptr, *cinv_all = nullptr;
  Xfer<T> tp{}, tq{};
  T *U = nullptr, *F = nullptr, *R = nullptr;
};

template <typename T>
struct Typed3 {
  std::vector<Lev3T<T>> lev;
  T* coarse_inv = nullptr;
  int fused_lc = -1;                // levels 0..fused_lc run in one cluster launch, or -1
  int fused_kind = 8;               // cluster size (blocks)
  int cluster_max = -1;
  Cluster3Desc<T> cdesc{};
};

struct Lev3Common {
  int n_patches = 0, maxl = 0, n_colours = 0, row_slots = 0;
  std::vector<int> colour_off, n8, colour_blk;
  int* colour_blk_dev = nullptr;
  int *dofs = nullptr, *cls = nullptr, *nloc = nullptr;
  int *slot_g = nullptr, *slot_c = nullptr;
  unsigned* slot_kb = nullptr;
  long long* cinv_off = nullptr;
  double *dcoef = nullptr, *inv_dcoef = nullptr;
};

}  // namespace

struct igamg3d_handle {
  igamg_problem prob{};
  HierarchyHost3 host;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  std::vector<Lev3Common> lc;
  Typed3<double> d;
  Typed3<float> f;
  int ndof0 = 0;
  double *part = nullptr, *norm2 = nullptr;
  unsigned long long* divmax = nullptr;
  double *lv_p = nullptr, *lv_q = nullptr, *h_pinned = nullptr;
  double *f_dev = nullptr, *Fh = nullptr, *Uh = nullptr;
  double *psi = nullptr, *tot = nullptr;
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  const void* gU[3] = {nullptr, nullptr, nullptr};
  const void* gF[3] = {nullptr, nullptr, nullptr};
  std::vector<void*> allocs;
  KrylovWork kw;                    // FGMRES modes
  double* zeros = nullptr;
  double* jt = nullptr;              // mapped domains: J^T at the finest quadrature points
};

namespace {

#define CK3(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_error(std::string(#x) + ": " + cudaGetErrorString(e_)); return IGAMG_ECUDA; } } while (0)

int dmalloc(igamg3d_handle* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return IGAMG_ECUDA; }
  h->allocs.push_back(*p);
  return IGAMG_OK;
}

template <typename V, typename S>
int upload_as(igamg3d_handle* h, V** dst, const std::vector<S>& src) {
  std::vector<V> tmp(src.begin(), src.end());
  int rc = dmalloc(h, (void**)dst, tmp.size() * sizeof(V));
  if (rc) return rc;
  CK3(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(V), cudaMemcpyHostToDevice));
  return IGAMG_OK;
}

int launch_check() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return IGAMG_ECUDA; }
  return IGAMG_OK;
}

// colour kernel: row-parallel (default) or the patch-per-lane-group form (IGAMG_PATCH_KERNEL=lanes)
bool row_parallel() {
  static const bool rp = [] {
    const char* e = std::getenv("IGAMG_PATCH_KERNEL");
    return !(e && std::strcmp(e, "lanes") == 0);
  }();
  return rp;
}

// Split rows (k_mult_rows3x) where a colour has few rows: IGAMG_ROW_SPLIT = 0 (never),
// 1 (always), unset (levels whose colours average fewer than kSplitBelow slot blocks).
constexpr int kSplitBelow = 152;
bool split_rows(const Lev3Common& lc) {
  static const int mode = [] {
    const char* e = std::getenv("IGAMG_ROW_SPLIT");
    return e ? std::atoi(e) : -1;
  }();
  if (mode >= 0) return mode == 1;
  return (long long)lc.colour_blk[lc.n_colours] * lc.row_slots < 256LL * kSplitBelow * lc.n_colours;
}

bool fp32_base3(const igamg_problem& pr) {
  return pr.precision == IGAMG_FP32_IR || pr.precision == IGAMG_FGMRES_FP32;
}

template <typename T> Typed3<T>& typed(igamg3d_handle* h);
template <> Typed3<double>& typed<double>(igamg3d_handle* h) { return h->d; }
template <> Typed3<float>& typed<float>(igamg3d_handle* h) { return h->f; }

template <typename T>
int upload_typed(igamg3d_handle* h, Typed3<T>& ty) {
  const int L = (int)h->host.lev.size();
  ty.lev.resize(L);
  int rc;
  for (int l = 0; l < L; ++l) {
    auto& hl = h->host.lev[l];
    auto& tl = ty.lev[l];
    LevelTab3<T>& Lt = tl.L;
    Lt.n = hl.sz.n; Lt.ni = hl.sz.ni; Lt.nq = hl.sz.nq;
    Lt.n_uc = (int)hl.sz.n_uc; Lt.n_u = (int)hl.sz.n_u; Lt.n_p = (int)hl.sz.n_p; Lt.n_total = (int)hl.sz.n_total;
    int* cm[4];
    T* rc4[4];
    for (int k = 0; k < 4; ++k) {
      if ((rc = upload_as(h, &cm[k], hl.st.cmap[k])) || (rc = upload_as(h, &rc4[k], hl.st.rec[k]))) return rc;
    }
    Lt.cm0 = cm[0]; Lt.cm1 = cm[1]; Lt.cm2 = cm[2]; Lt.cm3 = cm[3];
    Lt.rc0 = rc4[0]; Lt.rc1 = rc4[1]; Lt.rc2 = rc4[2]; Lt.rc3 = rc4[3];
    Lt.srow = nullptr;
    Lt.sext = nullptr;
    if (!hl.rows.empty()) {
      T* sr = nullptr;
      if ((rc = upload_as(h, &sr, hl.rows))) return rc;
      Lt.srow = sr;
    }
    if (!hl.ext.empty()) {
      T* se = nullptr;
      if ((rc = upload_as(h, &se, hl.ext))) return rc;
      Lt.sext = se;
    }
    if (l >= 1) {
      // the lane-group kernel's tables (maxl-stride inverses) only for class-record levels
      if (hl.rows.empty() && ((rc = upload_as(h, &tl.cinv, hl.pt.cinv)) || (rc = upload_as(h, &tl.cinv8, hl.pt.cinv8))))
        return rc;
      if ((rc = upload_as(h, &tl.cinv_all, hl.pt.cinv_all))) return rc;
      auto up = [&](const Transfer1D& t, Xfer<T>& x) -> int {
        x.nf = t.nf; x.nc = t.nc;
        int r;
        if ((r = upload_as(h, (int**)&x.c0, t.c0)) || (r = upload_as(h, (int**)&x.f0, t.f0)) ||
            (r = upload_as(h, (T**)&x.pv, t.pv)) || (r = upload_as(h, (T**)&x.rv, t.rv)))
          return r;
        return IGAMG_OK;
      };
      if ((rc = up(h->host.tp_free[l], tl.tp)) || (rc = up(h->host.tq[l], tl.tq))) return rc;
    }
    size_t nt = (size_t)hl.sz.n_total;
    if ((rc = dmalloc(h, (void**)&tl.U, nt * sizeof(T))) || (rc = dmalloc(h, (void**)&tl.F, nt * sizeof(T))) ||
        (rc = dmalloc(h, (void**)&tl.R, nt * sizeof(T))))
      return rc;
  }
  return upload_as(h, &ty.coarse_inv, h->host.coarse_inv);
}

// ---- per-step launchers ------------------------------------------------------------------
template <typename T>
int do_residual(igamg3d_handle* h, int l, const T* U, const T* F, T* R, double* norm2, cudaStream_t s) {
  auto& L = typed<T>(h).lev[l].L;
  unsigned nb = nblk(L.n_total - 1);
  if (h->prob.p == 2) k_residual3<2, T><<<nb, kBlock, 0, s>>>(L, U, F, R, h->part);
  else k_residual3<3, T><<<nb, kBlock, 0, s>>>(L, U, F, R, h->part);
  k_residual_finish<T><<<1, 1024, 0, s>>>(L.n_total, F, R, h->part, (int)nb, norm2);
  return launch_check();
}

template <typename T>
int do_smooth(igamg3d_handle* h, int l, T* U, const T* F, cudaStream_t s) {
  auto& lc = h->lc[l];
  auto& tl = typed<T>(h).lev[l];
  if ((row_parallel() || tl.L.srow) && lc.row_slots) {
    const int S = lc.row_slots;
    const int* sg = lc.slot_g; const int* sc = lc.slot_c; const unsigned* sk = lc.slot_kb;
    if (S <= 256 && split_rows(lc)) {
      for (int c = 0; c < lc.n_colours; ++c) {
        int b0 = lc.colour_blk[c], nb = lc.colour_blk[c + 1] - b0;
        if (nb == 0) continue;
        if (h->prob.p == 2 && S == 128) k_mult_rows3x<2, 128, T><<<nb, 384, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
        else if (h->prob.p == 2) k_mult_rows3x<2, 256, T><<<nb, 768, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
        else if (S == 128) k_mult_rows3x<3, 128, T><<<nb, 384, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
        else k_mult_rows3x<3, 256, T><<<nb, 768, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
      }
      return launch_check();
    }
    for (int c = 0; c < lc.n_colours; ++c) {
      int b0 = lc.colour_blk[c], nb = lc.colour_blk[c + 1] - b0;
      if (nb == 0) continue;
      if (h->prob.p == 2 && S == 128) k_mult_rows3<2, 128, T><<<nb, 128, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
      else if (h->prob.p == 3 && S == 128) k_mult_rows3<3, 128, T><<<nb, 128, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
      else if (h->prob.p == 2 && S == 256) k_mult_rows3<2, 256, T><<<nb, 256, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
      else if (h->prob.p == 2) k_mult_rows3<2, 1024, T><<<nb, 1024, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
      else if (S == 256) k_mult_rows3<3, 256, T><<<nb, 256, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
      else k_mult_rows3<3, 1024, T><<<nb, 1024, 0, s>>>(tl.L, U, F, sg, sc, sk, tl.cinv_all, lc.cinv_off, b0 * S);
    }
    return launch_check();
  }
  size_t shm = (size_t)(kBlock / 32) * lc.maxl * sizeof(T);
  for (int c = 0; c < lc.n_colours; ++c) {
    int first = lc.colour_off[c], count = lc.colour_off[c + 1] - first;
    if (count == 0) continue;
    int n8 = lc.n8[c], ngen = count - n8;
    int nb8 = (n8 + 31) / 32, nbg = (ngen + 7) / 8;
    unsigned nb = (unsigned)(nb8 + nbg);
    if (h->prob.p == 2)
      k_mult_colour3<2, T><<<nb, kBlock, shm, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
    else
      k_mult_colour3<3, T><<<nb, kBlock, shm, s>>>(tl.L, U, F, lc.dofs, lc.cls, tl.cinv, tl.cinv8, lc.nloc, lc.maxl, first, n8, ngen, nb8);
  }
  return launch_check();
}

template <typename T>
int do_restrict(igamg3d_handle* h, int l, const T* rf, T* gc, cudaStream_t s) {
  auto& f = typed<T>(h).lev[l];
  auto& c = typed<T>(h).lev[l - 1];
  k_restrict3<T><<<nblk(c.L.n_total), kBlock, 0, s>>>(f.L, c.L, f.tp, f.tq, rf, gc);
  return launch_check();
}

template <typename T>
int do_prolong(igamg3d_handle* h, int l, const T* uc, T* uf, cudaStream_t s) {
  auto& f = typed<T>(h).lev[l];
  auto& c = typed<T>(h).lev[l - 1];
  k_prolong_add3<T><<<nblk(f.L.n_total), kBlock, 0, s>>>(f.L, c.L, f.tp, f.tq, uc, uf);
  return launch_check();
}

template <typename T>
int do_coarse(igamg3d_handle* h, const T* G, T* U, cudaStream_t s) {
  k_coarse<T><<<1, 1024, h->ndof0 * sizeof(T), s>>>(h->ndof0, typed<T>(h).coarse_inv, G, U);
  return launch_check();
}

template <typename T>
int do_cluster(igamg3d_handle* h, const T* Fin, T* Uio, int load_u, cudaStream_t s) {
  auto& ty = typed<T>(h);
  ty.cdesc.nlev = ty.fused_lc + 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ty.fused_kind);
  cfg.blockDim = dim3(1024);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ty.fused_kind; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = h->prob.p == 2 ? cudaLaunchKernelEx(&cfg, k_cluster3<2, T>, ty.cdesc, Fin, Uio, load_u)
                                 : cudaLaunchKernelEx(&cfg, k_cluster3<3, T>, ty.cdesc, Fin, Uio, load_u);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return IGAMG_ECUDA; }
  return IGAMG_OK;
}

// Algorithm 1 from level l, recursively, in place on Ul (zeroed first if zero), with gamma
// coarse cycles per level (gamma = 2: the W-cycle); per-level launches throughout.
template <typename T>
int do_cycle(igamg3d_handle* h, int l, T* Ul, const T* Fl, bool zero, cudaStream_t s) {
  auto& ty = typed<T>(h);
  if (l == 0) return do_coarse<T>(h, Fl, Ul, s);
  int rc;
  if (zero) CK3(cudaMemsetAsync(Ul, 0, ty.lev[l].L.n_total * sizeof(T), s));
  for (int k = 0; k < h->prob.nu1; ++k) if ((rc = do_smooth<T>(h, l, Ul, Fl, s))) return rc;
  if ((rc = do_residual<T>(h, l, Ul, Fl, ty.lev[l].R, nullptr, s))) return rc;
  if ((rc = do_restrict<T>(h, l, ty.lev[l].R, ty.lev[l - 1].F, s))) return rc;
  const int gamma = std::max(1, h->prob.gamma);
  for (int g = 0; g < gamma; ++g)
    if ((rc = do_cycle<T>(h, l - 1, ty.lev[l - 1].U, ty.lev[l - 1].F, g == 0, s))) return rc;
  if ((rc = do_prolong<T>(h, l, ty.lev[l - 1].U, Ul, s))) return rc;
  for (int k = 0; k < h->prob.nu2; ++k) if ((rc = do_smooth<T>(h, l, Ul, Fl, s))) return rc;
  return IGAMG_OK;
}

template <typename T>
int do_vcycle(igamg3d_handle* h, T* U, const T* F, cudaStream_t s) {
  auto& ty = typed<T>(h);
  const int L = (int)ty.lev.size();
  if (L == 1) return do_coarse<T>(h, F, U, s);
  if (h->prob.gamma > 1) return do_cycle<T>(h, L - 1, U, F, false, s);
  int rc;
  const int lc = ty.fused_lc;
  if (lc == L - 1) return do_cluster<T>(h, F, U, 1, s);
  if (lc >= 1) {
    for (int l = L - 1; l > lc; --l) {
      T* Ul = (l == L - 1) ? U : ty.lev[l].U;
      const T* Fl = (l == L - 1) ? F : ty.lev[l].F;
      if (l < L - 1) CK3(cudaMemsetAsync(Ul, 0, ty.lev[l].L.n_total * sizeof(T), s));
      for (int k = 0; k < h->prob.nu1; ++k) if ((rc = do_smooth<T>(h, l, Ul, Fl, s))) return rc;
      if ((rc = do_residual<T>(h, l, Ul, Fl, ty.lev[l].R, nullptr, s))) return rc;
      if ((rc = do_restrict<T>(h, l, ty.lev[l].R, ty.lev[l - 1].F, s))) return rc;
    }
    if ((rc = do_cluster<T>(h, ty.lev[lc].F, ty.lev[lc].U, 0, s))) return rc;
    for (int l = lc + 1; l <= L - 1; ++l) {
      T* Ul = (l == L - 1) ? U : ty.lev[l].U;
      const T* Fl = (l == L - 1) ? F : ty.lev[l].F;
      if ((rc = do_prolong<T>(h, l, ty.lev[l - 1].U, Ul, s))) return rc;
      for (int k = 0; k < h->prob.nu2; ++k) if ((rc = do_smooth<T>(h, l, Ul, Fl, s))) return rc;
    }
    return IGAMG_OK;
  }
  for (int l = L - 1; l >= 1; --l) {
    T* Ul = (l == L - 1) ? U : ty.lev[l].U;
    const T* Fl = (l == L - 1) ? F : ty.lev[l].F;
    if (l < L - 1) CK3(cudaMemsetAsync(Ul, 0, ty.lev[l].L.n_total * sizeof(T), s));
    for (int k = 0; k < h->prob.nu1; ++k) if ((rc = do_smooth<T>(h, l, Ul, Fl, s))) return rc;
    if ((rc = do_residual<T>(h, l, Ul, Fl, ty.lev[l].R, nullptr, s))) return rc;
    if ((rc = do_restrict<T>(h, l, ty.lev[l].R, ty.lev[l - 1].F, s))) return rc;
  }
  if ((rc = do_coarse<T>(h, ty.lev[0].F, ty.lev[0].U, s))) return rc;
  for (int l = 1; l <= L - 1; ++l) {
    T* Ul = (l == L - 1) ? U : ty.lev[l].U;
    const T* Fl = (l == L - 1) ? F : ty.lev[l].F;
    if ((rc = do_prolong<T>(h, l, ty.lev[l - 1].U, Ul, s))) return rc;
    for (int k = 0; k < h->prob.nu2; ++k) if ((rc = do_smooth<T>(h, l, Ul, Fl, s))) return rc;
  }
  return IGAMG_OK;
}

// Full multigrid (nested iteration) on K e = r, r in the finest level's F workspace, e
// written to its U workspace: r restricted to every level, the coarsest solved exactly, then
// on each finer level one cycle from the prolongated coarser solution.
template <typename T>
int do_fmg(igamg3d_handle* h, cudaStream_t s) {
  auto& ty = typed<T>(h);
  const int L = (int)ty.lev.size();
  int rc;
  for (int l = L - 1; l >= 1; --l)
    if ((rc = do_restrict<T>(h, l, ty.lev[l].F, ty.lev[l - 1].F, s))) return rc;
  if ((rc = do_coarse<T>(h, ty.lev[0].F, ty.lev[0].U, s))) return rc;
  for (int l = 1; l <= L - 1; ++l) {
    CK3(cudaMemsetAsync(ty.lev[l].U, 0, ty.lev[l].L.n_total * sizeof(T), s));
    if ((rc = do_prolong<T>(h, l, ty.lev[l - 1].U, ty.lev[l].U, s))) return rc;
    if ((rc = do_cycle<T>(h, l, ty.lev[l].U, ty.lev[l].F, false, s))) return rc;
  }
  return IGAMG_OK;
}

// mapped domains: the parametric load J^T f at every quadrature point (f and fh may alias)
static __global__ void k_pullback3(int npts, const double* __restrict__ jt, const double* f, double* fh) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const double fx = f[i], fy = f[(size_t)npts + i], fz = f[(size_t)2 * npts + i];
  const double* t = jt + (size_t)9 * i;              // t[3k + c] = dX_c / dxi_k
  fh[i] = t[0] * fx + t[1] * fy + t[2] * fz;
  fh[(size_t)npts + i] = t[3] * fx + t[4] * fy + t[5] * fz;
  fh[(size_t)2 * npts + i] = t[6] * fx + t[7] * fy + t[8] * fz;
}

static __global__ void k_add_to3(int n, const double* __restrict__ E, double* __restrict__ U) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) U[i] += E[i];
}

// FP32 mode, one refinement step (R64 = F - K U on entry): FP32 V-cycle (with fmg: an FP32
// full-multigrid pass) on K e = R64, then U += (curl psi(e), e_p, e_lambda) in FP64 and
// R64 = F - K U with its norm.
int do_ir_step(igamg3d_handle* h, double* U, const double* F, cudaStream_t s, bool fmg = false) {
  const int L = (int)h->d.lev.size();
  auto& top32 = h->f.lev[L - 1];
  double* R64 = h->d.lev[L - 1].R;
  const auto& Ld = h->d.lev[L - 1].L;
  const auto& lc = h->lc[L - 1];
  k_to_float<<<nblk(Ld.n_total), kBlock, 0, s>>>(Ld.n_total, R64, top32.F);
  int rc;
  if (fmg) {
    if ((rc = do_fmg<float>(h, s))) return rc;
  } else {
    CK3(cudaMemsetAsync(top32.U, 0, Ld.n_total * sizeof(float), s));
    if ((rc = do_vcycle<float>(h, top32.U, top32.F, s))) return rc;
  }
  const int ni = Ld.ni, nq = Ld.nq;
  CK3(cudaMemsetAsync(h->psi + (size_t)2 * nq * ni * ni, 0, (size_t)nq * ni * ni * sizeof(double), s));
  k_lift3_z<<<nblk(2LL * ni * nq), kBlock, 0, s>>>(top32.L, lc.inv_dcoef, top32.U, h->psi, h->tot);
  k_lift3_chi<<<nblk(ni, 128), 128, 0, s>>>(ni, nq, lc.dcoef, lc.inv_dcoef, h->tot, h->psi);
  k_curl3<true><<<nblk(Ld.n_total), kBlock, 0, s>>>(Ld, lc.dcoef, h->psi, top32.U, U);
  if ((rc = launch_check())) return rc;
  return do_residual<double>(h, L - 1, U, F, R64, h->norm2, s);
}

int do_step(igamg3d_handle* h, double* U, const double* F, cudaStream_t s) {
  const int L = (int)h->d.lev.size();
  if (fp32_base3(h->prob)) return do_ir_step(h, U, F, s);
  int rc = do_vcycle<double>(h, U, F, s);
  if (rc) return rc;
  return do_residual<double>(h, L - 1, U, F, h->d.lev[L - 1].R, h->norm2, s);
}

// first solve step with fmg (R64 = F - K U on entry): U += FMG(R64), then R64 and its norm.
int do_fmg_step(igamg3d_handle* h, double* U, const double* F, cudaStream_t s) {
  const int L = (int)h->d.lev.size();
  if (fp32_base3(h->prob)) return do_ir_step(h, U, F, s, true);
  auto& top = h->d.lev[L - 1];
  const int n = top.L.n_total;
  CK3(cudaMemcpyAsync(top.F, top.R, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int rc = do_fmg<double>(h, s);
  if (rc) return rc;
  k_add_to3<<<nblk(n), kBlock, 0, s>>>(n, top.U, U);
  if ((rc = launch_check())) return rc;
  return do_residual<double>(h, L - 1, U, F, top.R, h->norm2, s);
}

int ensure_graph(igamg3d_handle* h, int kind, double* U, const double* F) {
  if (h->graph[kind] && h->gU[kind] == U && h->gF[kind] == F) return IGAMG_OK;
  if (h->graph[kind]) { cudaGraphExecDestroy(h->graph[kind]); h->graph[kind] = nullptr; }
  cudaGraph_t g;
  CK3(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int L = (int)h->d.lev.size();
  int rc = IGAMG_OK;
  if (kind == 1 && fp32_base3(h->prob))
    rc = do_residual<double>(h, L - 1, U, F, h->d.lev[L - 1].R, nullptr, h->cap_stream);
  if (!rc) rc = kind == 2 ? do_fmg_step(h, U, F, h->cap_stream) : do_step(h, U, F, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc) { if (e == cudaSuccess) cudaGraphDestroy(g); return rc; }
  CK3(e);
  cudaError_t ei = cudaGraphInstantiate(&h->graph[kind], g, 0);
  cudaGraphDestroy(g);
  CK3(ei);
  h->gU[kind] = U; h->gF[kind] = F;
  return IGAMG_OK;
}

int read_norm(igamg3d_handle* h, double* out) {
  CK3(cudaMemcpyAsync(h->h_pinned, h->norm2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK3(cudaStreamSynchronize(h->stream));
  *out = std::sqrt(h->h_pinned[0]);
  return IGAMG_OK;
}

}  // namespace

// Descriptor of the cluster form of the coarse end (k_cluster3) and the choice of its
// depth and cluster size: every candidate V-cycle is captured into a graph and replayed, the
// fastest kept (IGAMG_FUSED_LEVELS / IGAMG_FUSED_CLUSTER fix the choice, IGAMG_NO_CLUSTER
// disables the cluster form).
template <typename T>
int setup_cluster3(igamg3d_handle* h, Typed3<T>& ty) {
  ty.fused_lc = -1;
  ty.cluster_max = -1;
  const int L = (int)ty.lev.size();
  if (L < 2 || std::getenv("IGAMG_NO_CLUSTER")) return IGAMG_OK;
  if (h->prob.gamma > 1) return IGAMG_OK;     // W-cycles run level by level
  int best = -1;
  for (int l = 1; l < L && l < kMaxFused3; ++l) best = l;
  if (best < 1) return IGAMG_OK;
  Cluster3Desc<T>& D = ty.cdesc;
  D = Cluster3Desc<T>{};
  D.nlev = best + 1; D.nu1 = h->prob.nu1; D.nu2 = h->prob.nu2; D.ndof0 = h->ndof0;
  D.coarse_inv = ty.coarse_inv;
  int rc = dmalloc(h, (void**)&D.part, 32 * sizeof(double));
  if (rc) return rc;
  for (int l = 0; l <= best; ++l) {
    Cluster3Level<T>& V = D.lev[l];
    const auto& lc = h->lc[l];
    V.L = ty.lev[l].L; V.tp = ty.lev[l].tp; V.tq = ty.lev[l].tq; V.cinv = ty.lev[l].cinv_all; V.cinv_off = lc.cinv_off;
    V.slot_g = lc.slot_g; V.slot_c = lc.slot_c; V.slot_kb = lc.slot_kb; V.colour_blk = lc.colour_blk_dev;
    V.n_colours = lc.n_colours; V.maxl = lc.maxl; V.row_slots = lc.row_slots;
    V.U = ty.lev[l].U; V.F = ty.lev[l].F; V.R = ty.lev[l].R;
    if (l >= 1 && lc.row_slots != 128 && lc.row_slots != 256 && lc.row_slots != 1024) { best = l - 1; break; }
  }
  if (best < 1) return IGAMG_OK;
  for (auto fn : {(const void*)k_cluster3<2, T>, (const void*)k_cluster3<3, T>})
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return IGAMG_OK;
    }
  ty.cluster_max = best;
  const char* env = std::getenv("IGAMG_FUSED_LEVELS");
  if (env) {
    const char* ec = std::getenv("IGAMG_FUSED_CLUSTER");
    ty.fused_kind = ec ? std::max(2, std::atoi(ec)) : 8;
    ty.fused_lc = std::min(std::atoi(env), best);
    if (ty.fused_lc < 1) ty.fused_lc = -1;
    return IGAMG_OK;
  }
  // time the candidates on zero vectors of the finest level
  T* U = ty.lev[L - 1].U;
  T* F = ty.lev[L - 1].F;
  size_t nb = (size_t)ty.lev[L - 1].L.n_total * sizeof(T);
  CK3(cudaMemsetAsync(U, 0, nb, h->stream));
  CK3(cudaMemsetAsync(F, 0, nb, h->stream));
  cudaEvent_t e0, e1;
  CK3(cudaEventCreate(&e0));
  CK3(cudaEventCreate(&e1));
  const bool verbose = std::getenv("IGAMG_VERBOSE") != nullptr;
  std::vector<std::pair<int, int>> cands{{-1, 8}};
  for (int C : {8, 16})
    for (int d = 1; d <= best; ++d) cands.push_back({d, C});
  float best_ms = 1e30f;
  int best_lc = -1, best_kind = 8;
  for (auto [cand, kind] : cands) {
    ty.fused_lc = cand;
    ty.fused_kind = kind;
    cudaGraph_t g;
    cudaGraphExec_t ge = nullptr;
    CK3(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int r = do_vcycle<T>(h, U, F, h->cap_stream);
    cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
    if (r || ec != cudaSuccess) {
      if (ec == cudaSuccess) cudaGraphDestroy(g);
      cudaGetLastError();
      if (cand < 0) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r ? r : IGAMG_ECUDA; }
      continue;
    }
    cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) { cudaGetLastError(); continue; }
    float ms = 0;
    cudaError_t e = cudaGraphLaunch(ge, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int rr = 0; rr < 3 && e == cudaSuccess; ++rr) e = cudaGraphLaunch(ge, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); set_error(cudaGetErrorString(e)); return IGAMG_ECUDA; }
    if (verbose) std::fprintf(stderr, "igamg3d: cluster levels %d (blocks %d): %.1f us per V-cycle\n", cand, kind, 1e3f * ms / 3);
    if (ms < best_ms) { best_ms = ms; best_lc = cand; best_kind = kind; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ty.fused_lc = best_lc;
  ty.fused_kind = best_kind;
  if (verbose) std::fprintf(stderr, "igamg3d: chose cluster levels %d (blocks %d)\n", best_lc, best_kind);
  return IGAMG_OK;
}

// ---- entry points used by igamg.cu -----------------------------------------------------
namespace igamg {

int validate3(const igamg_problem& pr) {
  if (pr.p != 2 && pr.p != 3) return IGAMG_EUNSUPPORTED;
  if (pr.n_levels < 1 || pr.n_levels > 12 || pr.n_fine < 1) return IGAMG_EINVAL;
  if (pr.n_fine % (1 << (pr.n_levels - 1))) return IGAMG_EINVAL;
  if (!(pr.sigma > 0) || !(pr.nu > 0) || pr.nu1 < 0 || pr.nu2 < 0) return IGAMG_EINVAL;
  if (pr.smoother != IGAMG_MULT) return IGAMG_EUNSUPPORTED;   // eq. ASM is not built in 3D
  if (pr.precision < IGAMG_FP64 || pr.precision > IGAMG_FGMRES_FP32) return IGAMG_EUNSUPPORTED;
  if (pr.gamma < 0 || pr.gamma > 4 || pr.fmg < 0 || pr.fmg > 1) return IGAMG_EINVAL;
  if (pr.geometry != IGAMG_GEOM_SQUARE && pr.geometry != IGAMG_GEOM_HOLLOW_CYLINDER) return IGAMG_EUNSUPPORTED;
  if (pr.geometry == IGAMG_GEOM_HOLLOW_CYLINDER) {
    if (pr.beta_qp) return IGAMG_EUNSUPPORTED;                          // generalized Stokes only
    const double ri = pr.r_inner > 0 ? pr.r_inner : 0.075, ro = pr.r_outer > 0 ? pr.r_outer : 0.225;
    if (!(ri > 0) || !(ro > ri) || !std::isfinite(ro)) return IGAMG_EINVAL;
  }
  if (pr.fmg && pr.precision >= IGAMG_FGMRES_FP64) return IGAMG_EUNSUPPORTED;
  if (sizes3(pr.p, pr.n_fine).n_total > (1LL << 30)) return IGAMG_EINVAL;   // 32-bit row indices
  if (sizes3(pr.p, pr.n_fine >> (pr.n_levels - 1)).n_total > 4096) return IGAMG_EINVAL;
  return IGAMG_OK;
}

int h3_create(const igamg_problem* prob, void* cuda_stream, igamg3d_handle** out) {
  *out = nullptr;
  const igamg_problem& pr = *prob;
  int rc = validate3(pr);
  if (rc) return rc;
  auto* h = new igamg3d_handle();
  h->prob = pr;
  h->stream = (cudaStream_t)cuda_stream;
  std::string err;
  rc = build_hierarchy3(pr, h->host, err);
  if (rc) { set_error(err); delete h; return rc; }
  auto fail = [&](int code) { h3_destroy(h); return code; };
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(IGAMG_ECUDA);
  const int L = pr.n_levels, p = pr.p;
  h->lc.resize(L);
  for (int l = 0; l < L; ++l) {
    auto& lh = h->host.lev[l];
    auto& lc = h->lc[l];
    if ((rc = upload_as(h, &lc.dcoef, lh.f.dcoef))) return fail(rc);
    std::vector<double> inv(lh.f.dcoef.size());
    for (size_t k = 0; k < inv.size(); ++k) inv[k] = 1.0 / lh.f.dcoef[k];
    if ((rc = upload_as(h, &lc.inv_dcoef, inv))) return fail(rc);
    if (l >= 1) {
      const auto& pt = lh.pt;
      lc.n_patches = pt.n_patches; lc.maxl = pt.maxl; lc.n_colours = pt.n_colours;
      lc.colour_off = pt.colour_off; lc.n8 = pt.n8; lc.colour_blk = pt.colour_blk; lc.row_slots = pt.row_slots;
      if ((rc = upload_as(h, &lc.dofs, pt.dofs)) || (rc = upload_as(h, &lc.cls, pt.cls)) ||
          (rc = upload_as(h, &lc.nloc, pt.nloc)) || (rc = upload_as(h, &lc.slot_g, pt.slot_g)) ||
          (rc = upload_as(h, &lc.slot_c, pt.slot_c)) || (rc = upload_as(h, &lc.slot_kb, pt.slot_kb)) ||
          (rc = upload_as(h, &lc.colour_blk_dev, pt.colour_blk)) || (rc = upload_as(h, &lc.cinv_off, pt.cinv_off)))
        return fail(rc);
    }
  }
  h->ndof0 = h->host.ndof0;
  if ((rc = upload_typed<double>(h, h->d))) return fail(rc);
  if (fp32_base3(pr) && (rc = upload_typed<float>(h, h->f))) return fail(rc);
  const auto& fs = h->host.lev[L - 1].sz;
  long long nfine = fs.n_total;
  if ((rc = dmalloc(h, (void**)&h->part, 2 * sizeof(double) * (nblk(nfine) + 1)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->norm2, sizeof(double)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->divmax, sizeof(unsigned long long)))) return fail(rc);
  if ((rc = upload_as(h, &h->lv_p, h->host.lv_p)) || (rc = upload_as(h, &h->lv_q, h->host.lv_q))) return fail(rc);
  size_t nG = (size_t)pr.n_fine * (p + 2);
  if ((rc = dmalloc(h, (void**)&h->f_dev, 3 * nG * nG * nG * sizeof(double)))) return fail(rc);
  if (!h->host.jt.empty() && (rc = upload_as(h, &h->jt, h->host.jt))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->Fh, nfine * sizeof(double)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->Uh, nfine * sizeof(double)))) return fail(rc);
  size_t npsi = (size_t)3 * fs.nq * fs.ni * fs.ni;
  if ((rc = dmalloc(h, (void**)&h->psi, npsi * sizeof(double)))) return fail(rc);
  if ((rc = dmalloc(h, (void**)&h->tot, (size_t)fs.nq * fs.ni * sizeof(double)))) return fail(rc);
  if (cudaMallocHost((void**)&h->h_pinned, 2 * sizeof(double)) != cudaSuccess) return fail(IGAMG_ECUDA);
  // the colour kernels' dynamic shared memory (one maxl-vector per warp for wall patches)
  for (int l = 1; l < L; ++l) {
    size_t shm = (size_t)(kBlock / 32) * h->lc[l].maxl * sizeof(double);
    if (shm > 48 * 1024) {
      cudaFuncSetAttribute(k_mult_colour3<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
      cudaFuncSetAttribute(k_mult_colour3<3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
      cudaFuncSetAttribute(k_mult_colour3<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
      cudaFuncSetAttribute(k_mult_colour3<3, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    }
  }
  if ((size_t)h->ndof0 * sizeof(double) > 48 * 1024) {
    cudaFuncSetAttribute(k_coarse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(h->ndof0 * sizeof(double)));
    cudaFuncSetAttribute(k_coarse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(h->ndof0 * sizeof(float)));
  }
  // the cluster tuner runs V-cycles: only once every workspace above exists
  if ((rc = setup_cluster3<double>(h, h->d))) return fail(rc);
  if (fp32_base3(pr) && (rc = setup_cluster3<float>(h, h->f))) return fail(rc);
  if (pr.precision >= IGAMG_FGMRES_FP64) {
    if ((rc = krylov_alloc(h->kw, pr.restart > 0 ? pr.restart : 20, nfine, h->allocs))) return fail(rc);
    if ((rc = dmalloc(h, (void**)&h->zeros, nfine * sizeof(double)))) return fail(rc);
    if (cudaMemset(h->zeros, 0, nfine * sizeof(double)) != cudaSuccess) return fail(IGAMG_ECUDA);
  }
  *out = h;
  return IGAMG_OK;
}

void h3_destroy(igamg3d_handle* h) {
  if (!h) return;
  krylov_free_host(h->kw);
  for (auto& g : h->graph) if (g) cudaGraphExecDestroy(g);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

int h3_levels(const igamg3d_handle* h) { return (int)h->lc.size(); }

int h3_sizes(const igamg3d_handle* h, int level, igamg_sizes* out) {
  if (level < 0 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  *out = h->host.lev[level].pub;
  return IGAMG_OK;
}

const std::vector<double>& h3_quad_x(const igamg3d_handle* h) { return h->host.quad_x; }
const std::vector<double>& h3_quad_xyz(const igamg3d_handle* h) { return h->host.quad_xyz; }

int h3_load_vector(igamg3d_handle* h, const double* f_qp, double* F) {
  auto& Lt = h->d.lev.back().L;
  if (h->jt) {                                      // mapped domain: load J^T f
    const int nG = h->prob.n_fine * (h->prob.p + 2);
    const int npts = nG * nG * nG;
    k_pullback3<<<nblk(npts), kBlock, 0, h->stream>>>(npts, h->jt, f_qp, h->f_dev);
    f_qp = h->f_dev;
  }
  if (h->prob.p == 2) k_load3<2><<<nblk(Lt.n_total), kBlock, 0, h->stream>>>(Lt, h->lv_p, h->lv_q, f_qp, F);
  else k_load3<3><<<nblk(Lt.n_total), kBlock, 0, h->stream>>>(Lt, h->lv_p, h->lv_q, f_qp, F);
  return launch_check();
}

int h3_residual(igamg3d_handle* h, int level, const double* U, const double* F, double* R, double* norm_out) {
  if (level < 0 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  int rc = do_residual<double>(h, level, U, F, R, h->norm2, h->stream);
  if (rc) return rc;
  if (norm_out) return read_norm(h, norm_out);
  return IGAMG_OK;
}

int h3_smooth(igamg3d_handle* h, int level, double* U, const double* F, int sweeps) {
  if (level < 1 || level >= (int)h->lc.size() || sweeps < 0) return IGAMG_EINVAL;
  for (int k = 0; k < sweeps; ++k) { int rc = do_smooth<double>(h, level, U, F, h->stream); if (rc) return rc; }
  return IGAMG_OK;
}

int h3_restrict(igamg3d_handle* h, int level, const double* r, double* g) {
  if (level < 1 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  return do_restrict<double>(h, level, r, g, h->stream);
}

int h3_prolong_add(igamg3d_handle* h, int level, const double* uc, double* uf) {
  if (level < 1 || level >= (int)h->lc.size()) return IGAMG_EINVAL;
  return do_prolong<double>(h, level, uc, uf, h->stream);
}

int h3_coarse_solve(igamg3d_handle* h, const double* G, double* U) { return do_coarse<double>(h, G, U, h->stream); }

int h3_vcycle(igamg3d_handle* h, double* U, const double* F) {
  int rc = ensure_graph(h, 1, U, F);
  if (rc) return rc;
  CK3(cudaGraphLaunch(h->graph[1], h->stream));
  return IGAMG_OK;
}

int h3_div_inf(igamg3d_handle* h, const double* U, double* out) {
  const int L = (int)h->d.lev.size();
  auto& Lt = h->d.lev[L - 1].L;
  CK3(cudaMemsetAsync(h->divmax, 0, sizeof(unsigned long long), h->stream));
  k_div_inf3<<<nblk(Lt.n_p), kBlock, 0, h->stream>>>(Lt, h->lc[L - 1].dcoef, U, h->divmax);
  int rc = launch_check();
  if (rc) return rc;
  CK3(cudaMemcpyAsync(h->h_pinned, h->divmax, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK3(cudaStreamSynchronize(h->stream));
  *out = h->h_pinned[0];
  return IGAMG_OK;
}

static int kr3_precond(void* ctx, const double* v, double* z) {
  auto* h = (igamg3d_handle*)ctx;
  cudaStream_t s = h->stream;
  const int L = (int)h->d.lev.size();
  const auto& Ld = h->d.lev[L - 1].L;
  const auto& lc = h->lc[L - 1];
  CK3(cudaMemsetAsync(z, 0, Ld.n_total * sizeof(double), s));
  if (h->prob.precision == IGAMG_FGMRES_FP64) return do_vcycle<double>(h, z, v, s);
  auto& top32 = h->f.lev[L - 1];
  k_to_float<<<nblk(Ld.n_total), kBlock, 0, s>>>(Ld.n_total, v, top32.F);
  CK3(cudaMemsetAsync(top32.U, 0, Ld.n_total * sizeof(float), s));
  int rc = do_vcycle<float>(h, top32.U, top32.F, s);
  if (rc) return rc;
  const int ni = Ld.ni, nq = Ld.nq;
  CK3(cudaMemsetAsync(h->psi + (size_t)2 * nq * ni * ni, 0, (size_t)nq * ni * ni * sizeof(double), s));
  k_lift3_z<<<nblk(2LL * ni * nq), kBlock, 0, s>>>(top32.L, lc.inv_dcoef, top32.U, h->psi, h->tot);
  k_lift3_chi<<<nblk(ni, 128), 128, 0, s>>>(ni, nq, lc.dcoef, lc.inv_dcoef, h->tot, h->psi);
  k_curl3<true><<<nblk(Ld.n_total), kBlock, 0, s>>>(Ld, lc.dcoef, h->psi, top32.U, z);
  return launch_check();
}

static int kr3_apply(void* ctx, const double* z, double* w) {
  auto* h = (igamg3d_handle*)ctx;
  const int L = (int)h->d.lev.size();
  int rc = do_residual<double>(h, L - 1, z, h->zeros, w, nullptr, h->stream);    // w = -K z
  if (rc) return rc;
  return krylov_negate(w, h->d.lev[L - 1].L.n_total, h->stream);
}

static int kr3_residual(void* ctx, const double* U, const double* F, double* R, double* norm) {
  auto* h = (igamg3d_handle*)ctx;
  const int L = (int)h->d.lev.size();
  int rc = do_residual<double>(h, L - 1, U, F, R, h->norm2, h->stream);
  if (rc) return rc;
  return read_norm(h, norm);
}

int h3_solve(igamg3d_handle* h, double* U, const double* F, double rtol, int max_cycles, igamg_report* rep,
             double atol) {
  if (h->prob.precision >= IGAMG_FGMRES_FP64) {
    KrylovOps ops;
    ops.ctx = h; ops.stream = h->stream;
    ops.precond = kr3_precond; ops.apply = kr3_apply; ops.residual = kr3_residual;
    int st = fgmres_solve(ops, h->kw, U, F, rtol, atol, max_cycles, rep);
    if (st < 0) return st;
    if (rep) {
      double dv = 0.0;
      int rc = h3_div_inf(h, U, &dv);
      if (rc) return rc;
      rep->div_inf = dv;
    }
    return st;
  }
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
    CK3(cudaGraphLaunch(h->graph[(k == 0 && h->prob.fmg) ? 2 : 0], h->stream));
    ++k;
    if ((rc = read_norm(h, &rk))) return rc;
    if (!std::isfinite(rk)) { status = IGAMG_ENONFINITE; break; }
    if (rep && rep->history && k - 1 < rep->history_cap) rep->history[k - 1] = rk / r0;
    if (rk <= (atol >= 0 ? atol : rtol * r0)) status = IGAMG_OK;
  }
  if (rep) {
    rep->cycles = k; rep->res0 = r0; rep->rel_residual = r0 > 0 ? rk / r0 : 0.0;
    double dv = 0.0;
    if ((rc = h3_div_inf(h, U, &dv))) return rc;
    rep->div_inf = dv;
  }
  return status;
}

int h3_solve_host(igamg3d_handle* h, const double* f_qp_host, double* U_host, double rtol, int max_cycles,
                  igamg_report* rep) {
  size_t nG = (size_t)h->prob.n_fine * (h->prob.p + 2);
  size_t nt = (size_t)h->host.lev.back().sz.n_total;
  CK3(cudaMemcpyAsync(h->f_dev, f_qp_host, 3 * nG * nG * nG * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK3(cudaMemcpyAsync(h->Uh, U_host, nt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  int rc = h3_load_vector(h, h->f_dev, h->Fh);
  if (rc) return rc;
  int st = h3_solve(h, h->Uh, h->Fh, rtol, max_cycles, rep, -1.0);
  if (st < 0) return st;
  CK3(cudaMemcpyAsync(U_host, h->Uh, nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK3(cudaStreamSynchronize(h->stream));
  return st;
}

int h3_curl(igamg3d_handle* h, const double* psi, double* U) {
  auto& Lt = h->d.lev.back().L;
  k_curl3<false><<<nblk(Lt.n_u), kBlock, 0, h->stream>>>(Lt, h->lc.back().dcoef, psi, nullptr, U);
  return launch_check();
}

}  // namespace igamg

namespace igamg {

int host_operator_rows3(const igamg_problem* prob, int level, double* K, size_t cap, long long* n_out) {
  int rc = validate3(*prob);
  if (rc) return rc;
  if (level < 0 || level >= prob->n_levels) return IGAMG_EINVAL;
  if (sizes3(prob->p, prob->n_fine >> (prob->n_levels - 1 - level)).n_total > 20000) return IGAMG_EINVAL;
  HierarchyHost3 H;
  std::string err;
  // only the level's row records are needed: build a one-level hierarchy of that mesh
  igamg_problem one = *prob;
  one.n_fine = prob->n_fine >> (prob->n_levels - 1 - level);
  one.n_levels = 1;
  one.c_penalty = prob->c_penalty > 0 ? prob->c_penalty : 4.0 * (prob->p - 1);
  one.c_penalty *= (double)prob->n_fine / one.n_fine;   // keep C_I / h_fine
  // Stokes: only this level's records (one-level build of this mesh); Oseen: the level of the
  // full operator hierarchy (coarse levels are Galerkin products)
  const bool whole = prob->beta_qp || prob->geometry == IGAMG_GEOM_HOLLOW_CYLINDER;
  if ((rc = whole ? build_operators3(*prob, H, err) : build_level_only3(one, H, err))) return rc;
  const auto& lh = whole ? H.lev[level] : H.lev[0];
  LevelTab3<double> L{};
  L.n = lh.sz.n; L.ni = lh.sz.ni; L.nq = lh.sz.nq;
  L.n_uc = (int)lh.sz.n_uc; L.n_u = (int)lh.sz.n_u; L.n_p = (int)lh.sz.n_p; L.n_total = (int)lh.sz.n_total;
  L.cm0 = lh.st.cmap[0].data(); L.cm1 = lh.st.cmap[1].data(); L.cm2 = lh.st.cmap[2].data(); L.cm3 = lh.st.cmap[3].data();
  L.rc0 = lh.st.rec[0].data(); L.rc1 = lh.st.rec[1].data(); L.rc2 = lh.st.rec[2].data(); L.rc3 = lh.st.rec[3].data();
  L.srow = lh.rows.empty() ? nullptr : lh.rows.data();
  L.sext = lh.ext.empty() ? nullptr : lh.ext.data();
  long long n = lh.sz.n_total;
  if (n_out) *n_out = n;
  if (!K) return IGAMG_OK;
  if (cap < (size_t)(n * n)) return IGAMG_EINVAL;
  std::vector<double> e(n, 0.0);
  for (long long j = 0; j < n; ++j) {
    e[j] = 1.0;
    double lam = 0.0;
    for (long long i = 0; i + 1 < n; ++i) {
      double m = 0.0;
      K[i * n + j] = prob->p == 2 ? row3<2, double>(L, e.data(), (int)i, &m) : row3<3, double>(L, e.data(), (int)i, &m);
      lam += m * e[i];
    }
    K[(n - 1) * n + j] = lam;   // lambda row: m . p
    e[j] = 0.0;
  }
  return IGAMG_OK;
}


int host_operator_apply3(const igamg_problem* prob, int level, const double* V, double* KV, size_t n) {
  int rc = validate3(*prob);
  if (rc) return rc;
  if (level < 0 || level >= prob->n_levels) return IGAMG_EINVAL;
  igamg_problem one = *prob;
  one.n_fine = prob->n_fine >> (prob->n_levels - 1 - level);
  one.n_levels = 1;
  one.c_penalty = (prob->c_penalty > 0 ? prob->c_penalty : 4.0 * (prob->p - 1)) * prob->n_fine / one.n_fine;
  HierarchyHost3 H;
  std::string err;
  // Stokes: only this level's records (one-level build of this mesh); Oseen: the level of the
  // full operator hierarchy (coarse levels are Galerkin products)
  const bool whole = prob->beta_qp || prob->geometry == IGAMG_GEOM_HOLLOW_CYLINDER;
  if ((rc = whole ? build_operators3(*prob, H, err) : build_level_only3(one, H, err))) return rc;
  const auto& lh = whole ? H.lev[level] : H.lev[0];
  if (n != (size_t)lh.sz.n_total) return IGAMG_EINVAL;
  LevelTab3<double> L{};
  L.n = lh.sz.n; L.ni = lh.sz.ni; L.nq = lh.sz.nq;
  L.n_uc = (int)lh.sz.n_uc; L.n_u = (int)lh.sz.n_u; L.n_p = (int)lh.sz.n_p; L.n_total = (int)lh.sz.n_total;
  L.cm0 = lh.st.cmap[0].data(); L.cm1 = lh.st.cmap[1].data(); L.cm2 = lh.st.cmap[2].data(); L.cm3 = lh.st.cmap[3].data();
  L.rc0 = lh.st.rec[0].data(); L.rc1 = lh.st.rec[1].data(); L.rc2 = lh.st.rec[2].data(); L.rc3 = lh.st.rec[3].data();
  L.srow = lh.rows.empty() ? nullptr : lh.rows.data();
  L.sext = lh.ext.empty() ? nullptr : lh.ext.data();
  double lam = 0.0;
  for (size_t i = 0; i + 1 < n; ++i) {
    double m = 0.0;
    KV[i] = prob->p == 2 ? row3<2, double>(L, V, (int)i, &m) : row3<3, double>(L, V, (int)i, &m);
    lam += m * V[i];
  }
  KV[n - 1] = lam;
  return IGAMG_OK;
}

}  // namespace igamg
