// Internal interface of the FGMRES wrapper (krylov.cu), shared by the 2D and 3D drivers.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "igamg.h"

namespace igamg {

// Operations the wrapper needs from a handle (all enqueue on `stream`).
struct KrylovOps {
  void* ctx = nullptr;
  cudaStream_t stream = nullptr;
  int (*precond)(void* ctx, const double* v, double* z) = nullptr;   // z = M v
  int (*apply)(void* ctx, const double* z, double* w) = nullptr;     // w = K z
  // R = F - K U; *norm = ||R||_2 (synchronises)
  int (*residual)(void* ctx, const double* U, const double* F, double* R, double* norm) = nullptr;
};

struct KrylovWork {
  int m = 0;
  long long n = 0, ld = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *hcol = nullptr, *y = nullptr, *part = nullptr;
  double* hhost = nullptr;
};

int krylov_alloc(KrylovWork& W, int m, long long n, std::vector<void*>& allocs);
void krylov_free_host(KrylovWork& W);
int krylov_negate(double* w, long long n, cudaStream_t s);
int fgmres_solve(const KrylovOps& ops, KrylovWork& W, double* U, const double* F, double rtol, double atol,
                 int max_iters, igamg_report* rep);

}  // namespace igamg
