// Flexible GMRES(m) (Saad's right-preconditioned FGMRES) in FP64 around the multigrid
// V-cycle: the Krylov wrapper of the precision layer (the paper's method is the
// preconditioner; the wrapper only accelerates it).  The preconditioner is either an FP64
// V-cycle or an FP32 V-cycle whose velocity is replaced by the FP64 curl of a potential,
// so every preconditioned direction is divergence-free and so is every iterate.
//
// Vector kernels (dots with fixed-order reductions, so results are reproducible):
//   k_multidot:        part[i][block] = sum over the block's entries of w . V_i
//   k_multidot_finish: out[i] (+)= sum_b part[i][b]   (one block per vector, fixed order)
//   k_update:          w -= sum_i c_i V_i
//   k_scale:           v = w / sqrt(nrm2) (nrm2 on the device) or v = w * s
//   k_lincomb:         x += sum_j y_j Z_j
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "igamg3d.h"
#include "krylov.h"

namespace igamg {
namespace {

constexpr int kDotBlock = 256;
constexpr int kDotBlocks = 304;   // 2 per SM: enough to stream a vector, few partials

__global__ void __launch_bounds__(kDotBlock) k_multidot(long long n, const double* __restrict__ w,
                                                        const double* __restrict__ V, long long ld,
                                                        double* __restrict__ part) {
  __shared__ double sh[kDotBlock / 32];
  const int i = blockIdx.y;
  const double* v = V + (size_t)i * ld;
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)kDotBlock + threadIdx.x; k < n; k += (long long)gridDim.x * kDotBlock)
    s = fma(w[k], v[k], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kDotBlock / 32; ++k) t += sh[k];
    part[(size_t)i * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_multidot_finish(int nb, const double* __restrict__ part, double* __restrict__ out, int accumulate) {
  __shared__ double sh[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)i * nb + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    out[i] = accumulate ? out[i] + t : t;
  }
}

__global__ void k_update(long long n, double* __restrict__ w, const double* __restrict__ V, long long ld, int nv,
                         const double* __restrict__ c) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = w[k];
  for (int i = 0; i < nv; ++i) s = fma(-c[i], V[(size_t)i * ld + k], s);
  w[k] = s;
}

__global__ void k_scale(long long n, const double* __restrict__ w, const double* __restrict__ nrm2, double factor,
                        double* __restrict__ v) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double f = nrm2 ? 1.0 / sqrt(*nrm2) : factor;
  v[k] = w[k] * f;
}

__global__ void k_negate(long long n, double* __restrict__ w) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) w[k] = -w[k];
}

__global__ void k_lincomb(long long n, double* __restrict__ x, const double* __restrict__ Z, long long ld, int m,
                          const double* __restrict__ y) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = x[k];
  for (int j = 0; j < m; ++j) s = fma(y[j], Z[(size_t)j * ld + k], s);
  x[k] = s;
}

inline unsigned nblocks(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }

#define CKK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_error(std::string(#x) + ": " + cudaGetErrorString(e_)); return IGAMG_ECUDA; } } while (0)

int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return IGAMG_ECUDA; }
  return IGAMG_OK;
}

// hcol[0..nv) (+)= w . V_i
int multidot(const KrylovWork& W, long long n, const double* w, const double* V, int nv, double* out, int acc,
             cudaStream_t s) {
  k_multidot<<<dim3(kDotBlocks, nv), kDotBlock, 0, s>>>(n, w, V, W.ld, W.part);
  k_multidot_finish<<<nv, 256, 0, s>>>(kDotBlocks, W.part, out, acc);
  return check_launch();
}

}  // namespace

int krylov_alloc(KrylovWork& W, int m, long long n, std::vector<void*>& allocs) {
  W.m = m;
  W.n = n;
  W.ld = (n + 31) / 32 * 32;
  auto dm = [&](void** p, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return IGAMG_ECUDA; }
    allocs.push_back(*p);
    return IGAMG_OK;
  };
  int rc;
  if ((rc = dm((void**)&W.V, (size_t)(m + 1) * W.ld * sizeof(double))) ||
      (rc = dm((void**)&W.Z, (size_t)m * W.ld * sizeof(double))) ||
      (rc = dm((void**)&W.w, (size_t)W.ld * sizeof(double))) ||
      (rc = dm((void**)&W.hcol, (size_t)2 * (m + 2) * sizeof(double))) ||
      (rc = dm((void**)&W.y, (size_t)(m + 1) * sizeof(double))) ||
      (rc = dm((void**)&W.part, (size_t)(m + 2) * kDotBlocks * sizeof(double))))
    return rc;
  if (cudaMallocHost((void**)&W.hhost, (size_t)2 * (m + 2) * sizeof(double)) != cudaSuccess) return IGAMG_ECUDA;
  return IGAMG_OK;
}

void krylov_free_host(KrylovWork& W) {
  if (W.hhost) cudaFreeHost(W.hhost);
  W.hhost = nullptr;
}

// FGMRES(m): U in place; stops when ||F - K U|| <= target (true residual, checked at the end
// of every restart cycle).  rep->cycles counts preconditioner applications (V-cycles);
// rep->history holds the relative residual estimates after each of them.
int fgmres_solve(const KrylovOps& ops, KrylovWork& W, double* U, const double* F, double rtol, double atol,
                 int max_iters, igamg_report* rep) {
  const long long n = W.n;
  const int m = W.m;
  cudaStream_t s = ops.stream;
  double beta = 0.0;
  int rc = ops.residual(ops.ctx, U, F, W.w, &beta);
  if (rc) return rc;
  if (!std::isfinite(beta)) return IGAMG_ENONFINITE;
  const double r0 = beta;
  const double target = atol >= 0 ? atol : rtol * r0;
  int its = 0, status = IGAMG_NOT_CONVERGED;
  double est = beta;
  if (beta == 0.0 || beta <= target) status = IGAMG_OK;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), yv(m);
  while (status == IGAMG_NOT_CONVERGED && its < max_iters) {
    // V_0 = r / beta
    k_scale<<<nblocks(n), 256, 0, s>>>(n, W.w, nullptr, 1.0 / beta, W.V);
    if ((rc = check_launch())) return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    bool done = false;
    for (int j = 0; j < m && its < max_iters; ++j) {
      double* vj = W.V + (size_t)j * W.ld;
      double* zj = W.Z + (size_t)j * W.ld;
      if ((rc = ops.precond(ops.ctx, vj, zj))) return rc;
      if ((rc = ops.apply(ops.ctx, zj, W.w))) return rc;            // w = K z_j
      ++its;
      // classical Gram-Schmidt, twice: pass-1 coefficients in hcol[0..j], pass-2 ones in
      // hcol[m+2 ..]; the Hessenberg column is their sum
      double* h2 = W.hcol + (m + 2);
      if ((rc = multidot(W, n, W.w, W.V, j + 1, W.hcol, 0, s))) return rc;
      k_update<<<nblocks(n), 256, 0, s>>>(n, W.w, W.V, W.ld, j + 1, W.hcol);
      if ((rc = check_launch())) return rc;
      if ((rc = multidot(W, n, W.w, W.V, j + 1, h2, 0, s))) return rc;
      k_update<<<nblocks(n), 256, 0, s>>>(n, W.w, W.V, W.ld, j + 1, h2);
      if ((rc = check_launch())) return rc;
      // |w|^2 into hcol[j+1]; V_{j+1} = w / |w|
      if ((rc = multidot(W, n, W.w, W.w, 1, W.hcol + j + 1, 0, s))) return rc;
      k_scale<<<nblocks(n), 256, 0, s>>>(n, W.w, W.hcol + j + 1, 0.0, W.V + (size_t)(j + 1) * W.ld);
      if ((rc = check_launch())) return rc;
      CKK(cudaMemcpyAsync(W.hhost, W.hcol, (size_t)2 * (m + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
      CKK(cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = W.hhost[i] + W.hhost[m + 2 + i];
      double hn = std::sqrt(std::max(W.hhost[j + 1], 0.0));
      H[(size_t)(j + 1) * m + j] = hn;
      // apply the previous rotations, then a new one that zeroes H[j+1][j]
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
      }
      double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
      double r = std::hypot(a, b);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? b / r : 0.0;
      H[(size_t)j * m + j] = r;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      est = std::fabs(g[j + 1]);
      k = j + 1;
      if (rep && rep->history && its - 1 < rep->history_cap) rep->history[its - 1] = r0 > 0 ? est / r0 : 0.0;
      if (!std::isfinite(est)) return IGAMG_ENONFINITE;
      if (est <= target || hn == 0.0) { done = true; break; }
    }
    // y = R^{-1} g, U += Z y
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int c = i + 1; c < k; ++c) t -= H[(size_t)i * m + c] * yv[c];
      yv[i] = H[(size_t)i * m + i] != 0.0 ? t / H[(size_t)i * m + i] : 0.0;
    }
    CKK(cudaMemcpyAsync(W.y, yv.data(), (size_t)k * sizeof(double), cudaMemcpyHostToDevice, s));
    k_lincomb<<<nblocks(n), 256, 0, s>>>(n, U, W.Z, W.ld, k, W.y);
    if ((rc = check_launch())) return rc;
    // true residual for the stopping test and the next restart
    if ((rc = ops.residual(ops.ctx, U, F, W.w, &beta))) return rc;
    if (!std::isfinite(beta)) return IGAMG_ENONFINITE;
    est = beta;
    if (beta <= target) status = IGAMG_OK;
    (void)done;
  }
  if (rep) {
    rep->cycles = its;
    rep->res0 = r0;
    rep->rel_residual = r0 > 0 ? est / r0 : 0.0;
  }
  return status;
}

int krylov_negate(double* w, long long n, cudaStream_t s) {
  k_negate<<<nblocks(n), 256, 0, s>>>(n, w);
  return check_launch();
}

}  // namespace igamg
