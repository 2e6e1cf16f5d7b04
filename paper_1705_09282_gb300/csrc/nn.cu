// The learned warm start: a small fully convolutional network (3x3 convolutions
// cin -> 32 -> 32 -> 32 -> 2, GELU after the first three) that maps the forcing sampled on
// the streamfunction control grid plus log10(sigma/nu) to a scaled streamfunction and a
// scaled pressure; the exact discrete curl of the first seeds the V-cycle with a
// divergence-free velocity, the second with a pressure.
//
// Weights are held in BF16 for every product (FP32 master copy for the optimizer);
// activations and accumulation are FP32.  Forward, backward (data and weights), the masked
// mean-squared loss and Adam are hand-written kernels; tiles of 16 x 16 pixels per block
// with the input tile (plus halo) and the layer's weights staged in shared memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "igamg.h"

namespace {

constexpr int TILE = 16;
constexpr int NT = TILE * TILE;       // threads per block
template <int DIL> struct Halo { static constexpr int value = TILE + 2 * DIL; };

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

enum Epi { EPI_GELU = 0, EPI_LINEAR = 1, EPI_DGELU = 2 };

// out[b,o,p] = bias[o] + sum_{c,tap} w[o,c,tap] in[b,c,p+DIL*tap] (zero padding; taps in
// {-1,0,1}^2, spread by the dilation DIL), then
//   EPI_GELU:   z = out, a = gelu(z)          (z -> outz, a -> outa)
//   EPI_LINEAR: z = out                        (-> outz)
//   EPI_DGELU:  out * gelu'(aux[b,o,p])        (-> outz; backward through an activation)
template <int CIN, int COUT, int DIL>
__global__ void __launch_bounds__(NT) k_conv(int H, int W, int tiles_x, int tiles_y, const float* __restrict__ in,
                                             const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                                             const float* __restrict__ aux, float* __restrict__ outz,
                                             float* __restrict__ outa, int epi) {
  constexpr int HALO = Halo<DIL>::value;
  extern __shared__ float smf[];
  float* tile = smf;                                // CIN * HALO * HALO
  float* ws = smf + CIN * HALO * HALO;              // COUT * CIN * 9
  const int tid = threadIdx.x;
  const int tpi = tiles_x * tiles_y;
  const int b = blockIdx.x / tpi, t = blockIdx.x - b * tpi;
  const int y0 = (t / tiles_x) * TILE, x0 = (t % tiles_x) * TILE;
  for (int i = tid; i < COUT * CIN * 9; i += NT) ws[i] = __bfloat162float(w[i]);
  const float* inb = in + (size_t)b * CIN * H * W;
  for (int i = tid; i < CIN * HALO * HALO; i += NT) {
    int c = i / (HALO * HALO), r = i - c * HALO * HALO;
    int yy = y0 + r / HALO - DIL, xx = x0 + r % HALO - DIL;
    tile[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? inb[((size_t)c * H + yy) * W + xx] : 0.0f;
  }
  __syncthreads();
  const int ty = tid / TILE, tx = tid % TILE;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = 0.0f;
  for (int c = 0; c < CIN; ++c) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      float v = tile[c * HALO * HALO + (ty + DIL * (tap / 3)) * HALO + tx + DIL * (tap % 3)];
#pragma unroll
      for (int o = 0; o < COUT; ++o) acc[o] = fmaf(ws[(o * CIN + c) * 9 + tap], v, acc[o]);
    }
  }
  const int y = y0 + ty, x = x0 + tx;
  if (y >= H || x >= W) return;
#pragma unroll
  for (int o = 0; o < COUT; ++o) {
    size_t idx = (((size_t)b * COUT + o) * H + y) * W + x;
    float z = acc[o] + (bias ? bias[o] : 0.0f);
    if (epi == EPI_GELU) { outz[idx] = z; outa[idx] = gelu_f(z); }
    else if (epi == EPI_LINEAR) outz[idx] = z;
    else outz[idx] = z * gelu_grad_f(aux[idx]);
  }
}

// ---- 32 -> 32 convolution on the tensor cores (tcgen05, inference) -----------------------
// An implicit GEMM per block: D (128 pixels x 32 output channels, FP32 in tensor memory) =
// A (128 pixels x K, BF16) * B^T (32 channels x K, BF16), K = 32 input channels x 9 taps = 288,
// as 18 tcgen05.mma instructions of 128 x 32 x 16 issued by one thread.  A (the dilated 3 x 3
// neighbourhoods of 128 consecutive pixels, zero outside the image) and B (the layer's BF16
// weights) are staged in shared memory in the no-swizzle K-major layout of 8-row x 16-byte
// core matrices: core matrix (r, k) of an operand at ((r * KC + k) * 128) bytes, KC = K / 8,
// so the descriptor's K-direction stride is 128 bytes and its row-group stride KC * 128.  The
// accumulator is read back per warp (32 pixels x 32 channels) with tcgen05.ld and the bias and
// GELU are applied on the way out.
constexpr int TC_M = 128, TC_N = 32, TC_K = 288, TC_KC = TC_K / 8;
constexpr int TC_A_BYTES = TC_M * TC_K * 2, TC_B_BYTES = TC_N * TC_K * 2;
constexpr size_t TC_SMEM = TC_A_BYTES + TC_B_BYTES + 64;
constexpr int TC_TMEM_COLS = 32;
constexpr long TC_SPIN = 1L << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, K-direction (leading) and row-group (stride)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M
constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int DIL>
__global__ void __launch_bounds__(128) k_conv32_tc(int H, int W, int tiles, const float* __restrict__ in,
                                                   const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                                                   float* __restrict__ outz, float* __restrict__ outa, int epi,
                                                   int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(smem + TC_A_BYTES);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + TC_A_BYTES + TC_B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + TC_A_BYTES + TC_B_BYTES + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x / tiles, t = blockIdx.x - b * tiles;
  const int HW = H * W, p0 = t * TC_M;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // A: thread m stages pixel p0 + m's 288 neighbourhood values (coalesced over m per (c, tap))
  {
    const int m = tid, pix = p0 + m;
    const int y = pix / W, x = pix - (pix / W) * W;
    const float* inb = in + (size_t)b * 32 * HW;
    __nv_bfloat16* arow = As + (m >> 3) * (TC_KC * 64) + (m & 7) * 8;
    for (int c = 0; c < 32; ++c) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int yy = y + DIL * (tap / 3 - 1), xx = x + DIL * (tap % 3 - 1);
        float v = 0.0f;
        if (pix < HW && yy >= 0 && yy < H && xx >= 0 && xx < W) v = inb[(size_t)c * HW + yy * W + xx];
        const int k = c * 9 + tap;
        arow[(k >> 3) * 64 + (k & 7)] = __float2bfloat16_rn(v);
      }
    }
  }
  // B: the weights w[o][k] (k = c * 9 + tap), o = output channel
  for (int i = tid; i < TC_N * TC_K; i += 128) {
    const int o = i / TC_K, k = i - o * TC_K;
    Bs[((o >> 3) * TC_KC + (k >> 3)) * 64 + (o & 7) * 8 + (k & 7)] = w[i];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
    constexpr uint32_t idesc = tc_idesc(TC_M, TC_N);
#pragma unroll 1
    for (int s = 0; s < TC_K / 16; ++s) {
      const uint64_t ad = tc_smem_desc(a0 + s * 256, 128, TC_KC * 128);
      const uint64_t bd = tc_smem_desc(b0 + s * 256, 128, TC_KC * 128);
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(idesc), "r"(s));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
  }
  // wait for the accumulator (bounded)
  uint32_t done = 0;
  for (long it = 0; it < TC_SPIN && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(mbar))
        : "memory");
  }
  if (!done && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done) {
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int pix = p0 + warp * 32 + lane;
    if (pix < HW) {
#pragma unroll
      for (int o = 0; o < 32; ++o) {
        const size_t idx = ((size_t)b * 32 + o) * HW + pix;
        const float z = __uint_as_float(r[o]) + (bias ? bias[o] : 0.0f);
        if (epi == EPI_GELU) { outz[idx] = z; outa[idx] = gelu_f(z); }
        else outz[idx] = z;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// dw[o,c,tap] += sum_{b,p} dz[b,o,p] in[b,c,p+tap], dbias[o] += sum dz[b,o,p]; blocks loop
// over tiles and add their partial sums atomically once at the end.
template <int CIN, int COUT, int DIL>
__global__ void __launch_bounds__(NT) k_conv_wgrad(int B, int H, int W, int tiles_x, int tiles_y,
                                                   const float* __restrict__ in, const float* __restrict__ dz,
                                                   float* __restrict__ dw, float* __restrict__ db) {
  constexpr int HALO = Halo<DIL>::value;
  constexpr int NO = COUT * CIN * 9 + COUT;
  constexpr int PER = (NO + NT - 1) / NT;
  extern __shared__ float smf[];
  float* tile = smf;                                // CIN * HALO * HALO
  float* dzs = smf + CIN * HALO * HALO;             // COUT * NT
  const int tid = threadIdx.x;
  float acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.0f;
  const int tpi = tiles_x * tiles_y, ntiles = B * tpi;
  for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const int b = tt / tpi, t = tt - b * tpi;
    const int y0 = (t / tiles_x) * TILE, x0 = (t % tiles_x) * TILE;
    __syncthreads();
    const float* inb = in + (size_t)b * CIN * H * W;
    for (int i = tid; i < CIN * HALO * HALO; i += NT) {
      int c = i / (HALO * HALO), r = i - c * HALO * HALO;
      int yy = y0 + r / HALO - DIL, xx = x0 + r % HALO - DIL;
      tile[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? inb[((size_t)c * H + yy) * W + xx] : 0.0f;
    }
    for (int i = tid; i < COUT * NT; i += NT) {
      int o = i / NT, pp = i - o * NT;
      int yy = y0 + pp / TILE, xx = x0 + pp % TILE;
      dzs[i] = (yy < H && xx < W) ? dz[(((size_t)b * COUT + o) * H + yy) * W + xx] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      int idx = tid + k * NT;
      if (idx >= NO) break;
      float s = acc[k];
      if (idx < COUT * CIN * 9) {
        int o = idx / (CIN * 9), rem = idx - o * CIN * 9, c = rem / 9, tap = rem - c * 9;
        const float* d = dzs + o * NT;
        const float* tl = tile + c * HALO * HALO + DIL * (tap / 3) * HALO + DIL * (tap % 3);
        for (int pp = 0; pp < NT; ++pp) s = fmaf(d[pp], tl[(pp / TILE) * HALO + pp % TILE], s);
      } else {
        const float* d = dzs + (idx - COUT * CIN * 9) * NT;
        for (int pp = 0; pp < NT; ++pp) s += d[pp];
      }
      acc[k] = s;
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    int idx = tid + k * NT;
    if (idx >= NO) break;
    if (idx < COUT * CIN * 9) atomicAdd(&dw[idx], acc[k]);
    else atomicAdd(&db[idx - COUT * CIN * 9], acc[k]);
  }
}

// masked mean-squared loss of the two output channels: channel 0 (streamfunction) over the
// interior points (the boundary ring, where psi = 0, excluded), channel 1 (pressure) over
// the leading (H-1) x (W-1) points; each channel's mean is over its own mask:
// dz = 2 (z - t) / M_c, loss += (z - t)^2 / M_c
__global__ void k_loss(int B, int H, int W, const float* __restrict__ z, const float* __restrict__ tgt,
                       float* __restrict__ dz, double* __restrict__ loss, float inv_m0, float inv_m1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < B * 2 * H * W) {
    int r = i % (H * W), ch = (i / (H * W)) % 2, y = r / W, x = r % W;
    bool in = ch == 0 ? (y > 0 && y < H - 1 && x > 0 && x < W - 1) : (y < H - 1 && x < W - 1);
    float inv_m = ch == 0 ? inv_m0 : inv_m1;
    float d = in ? z[i] - tgt[i] : 0.0f;
    dz[i] = 2.0f * d * inv_m;
    l = (double)d * d * inv_m;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.0f - b1) * gi;
  float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi; v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 copies of the weights: forward layout w[o,c,tap] and the flipped transpose
// wT[c,o,8-tap] used to propagate gradients back through a layer.
__global__ void k_refresh_bf16(int cout, int cin, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb,
                               __nv_bfloat16* __restrict__ wt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cout * cin * 9) return;
  int o = i / (cin * 9), rem = i - o * cin * 9, c = rem / 9, tap = rem - c * 9;
  __nv_bfloat16 v = __float2bfloat16_rn(w[i]);
  wb[i] = v;
  wt[(c * cout + o) * 9 + (8 - tap)] = v;
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

std::string g_nn_err;

}  // namespace

struct igamg_nn {
  int cin = 3, width = 32;
  int dil[4] = {1, 1, 1, 1};
  int off_w[4], off_b[4], cin_l[4], cout_l[4];
  int nparam = 0;
  float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr, *wt = nullptr;      // per-layer bf16 weights, same offsets as master
  int step = 0;
  cudaStream_t stream = nullptr;
  size_t cap = 0;                                   // B*H*W capacity of the workspaces
  float* z[4] = {nullptr, nullptr, nullptr, nullptr};
  float* a[3] = {nullptr, nullptr, nullptr};
  float *d0 = nullptr, *d1 = nullptr;
  double* loss = nullptr;
  double* h_loss = nullptr;
  int* tc_err = nullptr;                            // set by a tensor-core convolution whose wait gave up
  int* h_tc_err = nullptr;
};

namespace {

#define NCK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { g_nn_err = cudaGetErrorString(e_); return IGAMG_ECUDA; } } while (0)

// splitmix64 + Box-Muller (own counter-based generator) for the He initialisation
struct Rng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uni() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
  double normal() { double u1 = 1.0 - uni(), u2 = uni(); return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2); }
};

template <int CIN, int COUT, int DIL>
size_t conv_smem() { return (size_t)(CIN * Halo<DIL>::value * Halo<DIL>::value + COUT * CIN * 9) * sizeof(float); }
template <int CIN, int COUT, int DIL>
size_t wgrad_smem() { return (size_t)(CIN * Halo<DIL>::value * Halo<DIL>::value + COUT * NT) * sizeof(float); }

template <int CIN, int COUT, int DIL>
int set_smem_one() {
  NCK(cudaFuncSetAttribute(k_conv<CIN, COUT, DIL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<CIN, COUT, DIL>()));
  NCK(cudaFuncSetAttribute(k_conv_wgrad<CIN, COUT, DIL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)wgrad_smem<CIN, COUT, DIL>()));
  return IGAMG_OK;
}
template <int DIL>
int set_smem_tc() {
  NCK(cudaFuncSetAttribute(k_conv32_tc<DIL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
  return IGAMG_OK;
}

// Tensor-core forward of the 32 -> 32 layers (default) or the SIMT kernel (IGAMG_NN_TC=0).
bool nn_tc() {
  const char* e = std::getenv("IGAMG_NN_TC");
  return !e || std::atoi(e) != 0;
}

template <int DIL>
void conv32_tc_d(igamg_nn* nn, int B, int H, int W, const float* in, const __nv_bfloat16* w, const float* bias,
                 float* outz, float* outa, int epi) {
  const int tiles = (int)cdiv((long long)H * W, TC_M);
  k_conv32_tc<DIL><<<B * tiles, 128, TC_SMEM, nn->stream>>>(H, W, tiles, in, w, bias, outz, outa, epi, nn->tc_err);
}
void conv32_tc(igamg_nn* nn, int dil, int B, int H, int W, const float* in, const __nv_bfloat16* w, const float* bias,
               float* outz, float* outa, int epi) {
  switch (dil) {
    case 2: conv32_tc_d<2>(nn, B, H, W, in, w, bias, outz, outa, epi); break;
    case 4: conv32_tc_d<4>(nn, B, H, W, in, w, bias, outz, outa, epi); break;
    case 8: conv32_tc_d<8>(nn, B, H, W, in, w, bias, outz, outa, epi); break;
    default: conv32_tc_d<1>(nn, B, H, W, in, w, bias, outz, outa, epi);
  }
}

template <int CIN, int COUT>
int set_smem_all() {
  int rc;
  if ((rc = set_smem_one<CIN, COUT, 1>()) || (rc = set_smem_one<CIN, COUT, 2>()) || (rc = set_smem_one<CIN, COUT, 4>()) ||
      (rc = set_smem_one<CIN, COUT, 8>()))
    return rc;
  return IGAMG_OK;
}

template <int CIN, int COUT, int DIL>
void conv_d(igamg_nn* nn, int B, int H, int W, const float* in, const __nv_bfloat16* w, const float* bias,
            const float* aux, float* outz, float* outa, int epi) {
  int tx = cdiv(W, TILE), ty = cdiv(H, TILE);
  k_conv<CIN, COUT, DIL><<<B * tx * ty, NT, conv_smem<CIN, COUT, DIL>(), nn->stream>>>(H, W, tx, ty, in, w, bias, aux,
                                                                                       outz, outa, epi);
}
template <int CIN, int COUT>
void conv(igamg_nn* nn, int dil, int B, int H, int W, const float* in, const __nv_bfloat16* w, const float* bias,
          const float* aux, float* outz, float* outa, int epi) {
  switch (dil) {
    case 2: conv_d<CIN, COUT, 2>(nn, B, H, W, in, w, bias, aux, outz, outa, epi); break;
    case 4: conv_d<CIN, COUT, 4>(nn, B, H, W, in, w, bias, aux, outz, outa, epi); break;
    case 8: conv_d<CIN, COUT, 8>(nn, B, H, W, in, w, bias, aux, outz, outa, epi); break;
    default: conv_d<CIN, COUT, 1>(nn, B, H, W, in, w, bias, aux, outz, outa, epi);
  }
}

template <int CIN, int COUT, int DIL>
void wgrad_d(igamg_nn* nn, int B, int H, int W, const float* in, const float* dz, float* dw, float* db) {
  int tx = cdiv(W, TILE), ty = cdiv(H, TILE);
  int nt = B * tx * ty;
  int grid = nt < 2 * 152 ? nt : 2 * 152;
  k_conv_wgrad<CIN, COUT, DIL><<<grid, NT, wgrad_smem<CIN, COUT, DIL>(), nn->stream>>>(B, H, W, tx, ty, in, dz, dw, db);
}
template <int CIN, int COUT>
void wgrad(igamg_nn* nn, int dil, int B, int H, int W, const float* in, const float* dz, float* dw, float* db) {
  switch (dil) {
    case 2: wgrad_d<CIN, COUT, 2>(nn, B, H, W, in, dz, dw, db); break;
    case 4: wgrad_d<CIN, COUT, 4>(nn, B, H, W, in, dz, dw, db); break;
    case 8: wgrad_d<CIN, COUT, 8>(nn, B, H, W, in, dz, dw, db); break;
    default: wgrad_d<CIN, COUT, 1>(nn, B, H, W, in, dz, dw, db);
  }
}

int ensure_cap(igamg_nn* nn, size_t pix) {
  if (pix <= nn->cap) return IGAMG_OK;
  for (auto*& p : nn->z) { if (p) cudaFree(p); p = nullptr; }
  for (auto*& p : nn->a) { if (p) cudaFree(p); p = nullptr; }
  if (nn->d0) cudaFree(nn->d0);
  if (nn->d1) cudaFree(nn->d1);
  nn->d0 = nn->d1 = nullptr;
  size_t wpix = pix * nn->width * sizeof(float);
  for (int l = 0; l < 3; ++l) { NCK(cudaMalloc(&nn->z[l], wpix)); NCK(cudaMalloc(&nn->a[l], wpix)); }
  NCK(cudaMalloc(&nn->z[3], 2 * pix * sizeof(float)));
  NCK(cudaMalloc(&nn->d0, wpix));
  NCK(cudaMalloc(&nn->d1, wpix));
  nn->cap = pix;
  return IGAMG_OK;
}

int refresh(igamg_nn* nn) {
  for (int l = 0; l < 4; ++l) {
    int n = nn->cout_l[l] * nn->cin_l[l] * 9;
    k_refresh_bf16<<<cdiv(n, 256), 256, 0, nn->stream>>>(nn->cout_l[l], nn->cin_l[l], nn->master + nn->off_w[l],
                                                          nn->wb + nn->off_w[l], nn->wt + nn->off_w[l]);
  }
  NCK(cudaGetLastError());
  return IGAMG_OK;
}

// tc: the two 32 -> 32 layers on the tensor cores (BF16 activations and weights, FP32
// accumulation); training keeps the SIMT path (FP32 activations, used by the backward pass)
int forward(igamg_nn* nn, int B, int H, int W, const float* x, bool tc = false) {
  const float* P = nn->master;
  const int* d = nn->dil;
  conv<3, 32>(nn, d[0], B, H, W, x, nn->wb + nn->off_w[0], P + nn->off_b[0], nullptr, nn->z[0], nn->a[0], EPI_GELU);
  if (tc) {
    conv32_tc(nn, d[1], B, H, W, nn->a[0], nn->wb + nn->off_w[1], P + nn->off_b[1], nn->z[1], nn->a[1], EPI_GELU);
    conv32_tc(nn, d[2], B, H, W, nn->a[1], nn->wb + nn->off_w[2], P + nn->off_b[2], nn->z[2], nn->a[2], EPI_GELU);
  } else {
    conv<32, 32>(nn, d[1], B, H, W, nn->a[0], nn->wb + nn->off_w[1], P + nn->off_b[1], nullptr, nn->z[1], nn->a[1], EPI_GELU);
    conv<32, 32>(nn, d[2], B, H, W, nn->a[1], nn->wb + nn->off_w[2], P + nn->off_b[2], nullptr, nn->z[2], nn->a[2], EPI_GELU);
  }
  conv<32, 2>(nn, d[3], B, H, W, nn->a[2], nn->wb + nn->off_w[3], P + nn->off_b[3], nullptr, nn->z[3], nullptr, EPI_LINEAR);
  NCK(cudaGetLastError());
  return IGAMG_OK;
}

// loss and gradients into nn->grad (zeroed first); loss left in nn->loss (device)
int backward(igamg_nn* nn, int B, int H, int W, const float* x, const float* tgt) {
  long long pix = (long long)B * H * W;
  long long m0 = (long long)B * (H - 2) * (W - 2), m1 = (long long)B * (H - 1) * (W - 1);
  NCK(cudaMemsetAsync(nn->grad, 0, nn->nparam * sizeof(float), nn->stream));
  NCK(cudaMemsetAsync(nn->loss, 0, sizeof(double), nn->stream));
  float* dz4 = nn->d0;
  k_loss<<<cdiv(2 * pix, 256), 256, 0, nn->stream>>>(B, H, W, nn->z[3], tgt, dz4, nn->loss, 1.0f / (float)m0,
                                                       1.0f / (float)m1);
  float* G = nn->grad;
  const int* d = nn->dil;
  wgrad<32, 2>(nn, d[3], B, H, W, nn->a[2], dz4, G + nn->off_w[3], G + nn->off_b[3]);
  float* dz3 = nn->d1;
  conv<2, 32>(nn, d[3], B, H, W, dz4, nn->wt + nn->off_w[3], nullptr, nn->z[2], dz3, nullptr, EPI_DGELU);
  wgrad<32, 32>(nn, d[2], B, H, W, nn->a[1], dz3, G + nn->off_w[2], G + nn->off_b[2]);
  float* dz2 = nn->d0;
  conv<32, 32>(nn, d[2], B, H, W, dz3, nn->wt + nn->off_w[2], nullptr, nn->z[1], dz2, nullptr, EPI_DGELU);
  wgrad<32, 32>(nn, d[1], B, H, W, nn->a[0], dz2, G + nn->off_w[1], G + nn->off_b[1]);
  float* dz1 = nn->d1;
  conv<32, 32>(nn, d[1], B, H, W, dz2, nn->wt + nn->off_w[1], nullptr, nn->z[0], dz1, nullptr, EPI_DGELU);
  wgrad<3, 32>(nn, d[0], B, H, W, x, dz1, G + nn->off_w[0], G + nn->off_b[0]);
  NCK(cudaGetLastError());
  return IGAMG_OK;
}

int check_dims(igamg_nn* nn, int B, int H, int W) {
  if (!nn || B < 1 || H < 3 || W < 3 || (long long)B * H * W > (1LL << 31) / 64) return IGAMG_EINVAL;
  return ensure_cap(nn, (size_t)B * H * W);
}

}  // namespace

extern "C" {

int igamg_nn_create(int in_channels, int width, const int* dilations, unsigned long long seed, void* cuda_stream,
                    igamg_nn** out) {
  if (!out) return IGAMG_EINVAL;
  *out = nullptr;
  if (in_channels != 3 || width != 32) return IGAMG_EUNSUPPORTED;
  for (int l = 0; dilations && l < 4; ++l)
    if (dilations[l] != 1 && dilations[l] != 2 && dilations[l] != 4 && dilations[l] != 8) return IGAMG_EUNSUPPORTED;
  auto* nn = new igamg_nn();
  nn->stream = (cudaStream_t)cuda_stream;
  for (int l = 0; dilations && l < 4; ++l) nn->dil[l] = dilations[l];
  const int cins[4] = {3, 32, 32, 32}, couts[4] = {32, 32, 32, 2};
  int off = 0;
  for (int l = 0; l < 4; ++l) {
    nn->cin_l[l] = cins[l]; nn->cout_l[l] = couts[l];
    nn->off_w[l] = off; off += couts[l] * cins[l] * 9;
    nn->off_b[l] = off; off += couts[l];
  }
  nn->nparam = off;
  std::vector<float> h(off, 0.0f);
  Rng r{seed};
  for (int l = 0; l < 4; ++l) {
    double sd = std::sqrt(2.0 / (cins[l] * 9.0)) * (l == 3 ? 0.1 : 1.0);   // He; small last layer
    for (int i = 0; i < couts[l] * cins[l] * 9; ++i) h[nn->off_w[l] + i] = (float)(sd * r.normal());
  }
  auto fail = [&](int code) { igamg_nn_destroy(nn); return code; };
  size_t pb = off * sizeof(float);
  if (cudaMalloc(&nn->master, pb) || cudaMalloc(&nn->grad, pb) || cudaMalloc(&nn->m, pb) || cudaMalloc(&nn->v, pb) ||
      cudaMalloc(&nn->wb, off * sizeof(__nv_bfloat16)) || cudaMalloc(&nn->wt, off * sizeof(__nv_bfloat16)) ||
      cudaMalloc(&nn->loss, sizeof(double)) || cudaMallocHost(&nn->h_loss, sizeof(double)) ||
      cudaMalloc(&nn->tc_err, sizeof(int)) || cudaMallocHost(&nn->h_tc_err, sizeof(int)))
    return fail(IGAMG_ECUDA);
  if (cudaMemset(nn->tc_err, 0, sizeof(int))) return fail(IGAMG_ECUDA);
  if (cudaMemcpy(nn->master, h.data(), pb, cudaMemcpyHostToDevice) || cudaMemset(nn->m, 0, pb) ||
      cudaMemset(nn->v, 0, pb) || cudaMemset(nn->wt, 0, off * sizeof(__nv_bfloat16)))
    return fail(IGAMG_ECUDA);
  int rc;
  if ((rc = set_smem_all<3, 32>()) || (rc = set_smem_all<32, 32>()) || (rc = set_smem_all<32, 2>()) ||
      (rc = set_smem_all<2, 32>()) || (rc = set_smem_tc<1>()) || (rc = set_smem_tc<2>()) || (rc = set_smem_tc<4>()) ||
      (rc = set_smem_tc<8>()))
    return fail(rc);
  if ((rc = refresh(nn))) return fail(rc);
  if (cudaStreamSynchronize(nn->stream)) return fail(IGAMG_ECUDA);
  *out = nn;
  return IGAMG_OK;
}

void igamg_nn_destroy(igamg_nn* nn) {
  if (!nn) return;
  for (void* p : {(void*)nn->master, (void*)nn->grad, (void*)nn->m, (void*)nn->v, (void*)nn->wb, (void*)nn->wt,
                  (void*)nn->loss, (void*)nn->d0, (void*)nn->d1, (void*)nn->tc_err})
    if (p) cudaFree(p);
  if (nn->h_tc_err) cudaFreeHost(nn->h_tc_err);
  for (auto* p : nn->z) if (p) cudaFree(p);
  for (auto* p : nn->a) if (p) cudaFree(p);
  if (nn->h_loss) cudaFreeHost(nn->h_loss);
  delete nn;
}

int igamg_nn_num_params(const igamg_nn* nn) { return nn ? nn->nparam : 0; }

int igamg_nn_get_params(igamg_nn* nn, float* host, size_t cap) {
  if (!nn || !host || cap < (size_t)nn->nparam) return IGAMG_EINVAL;
  NCK(cudaMemcpyAsync(host, nn->master, nn->nparam * sizeof(float), cudaMemcpyDeviceToHost, nn->stream));
  NCK(cudaStreamSynchronize(nn->stream));
  return IGAMG_OK;
}

int igamg_nn_set_params(igamg_nn* nn, const float* host, size_t n) {
  if (!nn || !host || n != (size_t)nn->nparam) return IGAMG_EINVAL;
  NCK(cudaMemcpyAsync(nn->master, host, n * sizeof(float), cudaMemcpyHostToDevice, nn->stream));
  NCK(cudaMemsetAsync(nn->m, 0, n * sizeof(float), nn->stream));
  NCK(cudaMemsetAsync(nn->v, 0, n * sizeof(float), nn->stream));
  nn->step = 0;
  int rc = refresh(nn);
  if (rc) return rc;
  NCK(cudaStreamSynchronize(nn->stream));
  return IGAMG_OK;
}

int igamg_nn_forward(igamg_nn* nn, int B, int H, int W, const float* x, float* out) {
  int rc = check_dims(nn, B, H, W);
  if (rc) return rc;
  if (!x || !out) return IGAMG_EINVAL;
  const bool tc = nn_tc();
  if ((rc = forward(nn, B, H, W, x, tc))) return rc;
  NCK(cudaMemcpyAsync(out, nn->z[3], (size_t)B * 2 * H * W * sizeof(float), cudaMemcpyDeviceToDevice, nn->stream));
  if (tc) {                                   // a tensor-core wait that gave up is reported here
    NCK(cudaMemcpyAsync(nn->h_tc_err, nn->tc_err, sizeof(int), cudaMemcpyDeviceToHost, nn->stream));
    NCK(cudaStreamSynchronize(nn->stream));
    if (*nn->h_tc_err) {
      NCK(cudaMemset(nn->tc_err, 0, sizeof(int)));
      g_nn_err = "a tensor-core convolution gave up waiting for its accumulator";
      return IGAMG_ETIMEOUT;
    }
  }
  return IGAMG_OK;
}

int igamg_nn_loss_grad(igamg_nn* nn, int B, int H, int W, const float* x, const float* target, double* loss,
                       float* grad_host) {
  int rc = check_dims(nn, B, H, W);
  if (rc) return rc;
  if (!x || !target) return IGAMG_EINVAL;
  if ((rc = forward(nn, B, H, W, x)) || (rc = backward(nn, B, H, W, x, target))) return rc;
  NCK(cudaMemcpyAsync(nn->h_loss, nn->loss, sizeof(double), cudaMemcpyDeviceToHost, nn->stream));
  if (grad_host) NCK(cudaMemcpyAsync(grad_host, nn->grad, nn->nparam * sizeof(float), cudaMemcpyDeviceToHost, nn->stream));
  NCK(cudaStreamSynchronize(nn->stream));
  if (loss) *loss = *nn->h_loss;
  return IGAMG_OK;
}

int igamg_nn_train_step(igamg_nn* nn, int B, int H, int W, const float* x, const float* target, float lr,
                        double* loss) {
  int rc = check_dims(nn, B, H, W);
  if (rc) return rc;
  if (!x || !target || !(lr > 0)) return IGAMG_EINVAL;
  if ((rc = forward(nn, B, H, W, x)) || (rc = backward(nn, B, H, W, x, target))) return rc;
  nn->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.0f - std::pow(b1, (float)nn->step), c2 = 1.0f - std::pow(b2, (float)nn->step);
  k_adam<<<cdiv(nn->nparam, 256), 256, 0, nn->stream>>>(nn->nparam, nn->master, nn->grad, nn->m, nn->v, lr, b1, b2,
                                                         1e-8f, c1, c2);
  if ((rc = refresh(nn))) return rc;
  if (loss) {
    NCK(cudaMemcpyAsync(nn->h_loss, nn->loss, sizeof(double), cudaMemcpyDeviceToHost, nn->stream));
    NCK(cudaStreamSynchronize(nn->stream));
    *loss = *nn->h_loss;
  }
  return IGAMG_OK;
}

}  // extern "C"
