// mlp.cu -- the learned surrogate of Omega: a 4 -> 128 -> 128 -> 128 -> 1 MLP
// with SiLU activations over (q, h, T, Delta), trained on free energies the
// k-sum itself produced.  (The paper has no learned component; the surrogate
// only proposes where the exact k-sum should look.)
//
// Precision: the two 128 x 128 layers multiply BF16 activations by BF16
// weights on the tensor cores (mma.sync m16n8k16, FP32 accumulation); the
// 4-wide input layer, the 1-wide output layer, SiLU, its derivative and the
// loss are FP32.  Master weights and Adam moments are FP32.  Every reduction
// over samples is a fixed-order sum of per-block partials (deterministic).
//
// Flat parameter layout (33 793 floats): W1[4][128], b1[128], W2[128][128],
// b2[128], W3[128][128], b3[128], W4[128], b4[1]; W[i][o] maps input i to
// output o.  Inputs are normalised as x = (raw - shift) * scale; the network
// predicts the target divided by y_scale.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/ffe.h"
#include "plan.h"

namespace ffe {

constexpr int kW = 128;       // layer width
constexpr int kRows = 64;     // samples per block
constexpr int kLdA = 136;     // padded row stride (bf16) of [rows][128] tiles
constexpr int kLdT = 72;      // padded row stride (bf16) of transposed [128][64] tiles
constexpr int kOffW1 = 0, kOffB1 = 512, kOffW2 = 640, kOffB2 = 17024, kOffW3 = 17152, kOffB3 = 33536,
              kOffW4 = 33664, kOffB4 = 33792, kNParams = 33793;

struct MlpDev {
  const float* master;          // FP32 parameters (layout above)
  const __nv_bfloat16* w2t;     // W2 transposed [out][in]
  const __nv_bfloat16* w3t;     // W3 transposed [out][in]
  const __nv_bfloat16* w2n;     // W2 [in][out]
  const __nv_bfloat16* w3n;     // W3 [in][out]
  float shift[4], scale[4];
};

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + __expf(-z)); }
__device__ __forceinline__ float siluf_(float z) { return z * sigmoidf_(z); }
__device__ __forceinline__ float silu_primef_(float z) {
  const float s = sigmoidf_(z);
  return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Block-level C[M x 128] = A[M x K] * B[K x 128] with 4 warps; A stored [m][k]
// (stride lda), B stored transposed Bt[n][k] (stride ldb); M = 64 * MT.
// Warp w owns rows [16 MT w, 16 MT (w+1)).  acc[mt][nt][.] follows the
// m16n8 accumulator layout: rows g, g+8 of the tile, columns 2t, 2t+1.
template <int MT>
__device__ __forceinline__ void gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* Bt, int ldb, int K,
                                          float (&acc)[MT][16][4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[MT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int r = (warp * MT + mt) * 16 + g;
      a[mt][0] = ld32(A + r * lda + k0 + 2 * t);
      a[mt][1] = ld32(A + (r + 8) * lda + k0 + 2 * t);
      a[mt][2] = ld32(A + r * lda + k0 + 2 * t + 8);
      a[mt][3] = ld32(A + (r + 8) * lda + k0 + 2 * t + 8);
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int n = nt * 8 + g;
      const uint32_t b0 = ld32(Bt + n * ldb + k0 + 2 * t);
      const uint32_t b1 = ld32(Bt + n * ldb + k0 + 2 * t + 8);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) mma_bf16(acc[mt][nt], a[mt], b0, b1);
    }
  }
}

// Copy a [128][128] BF16 matrix from global into a padded shared tile.
__device__ __forceinline__ void load_w(__nv_bfloat16* dst, const __nv_bfloat16* src) {
  for (int i = threadIdx.x; i < kW * kW / 2; i += blockDim.x) {
    const int r = (2 * i) / kW, c = (2 * i) % kW;
    *reinterpret_cast<uint32_t*>(dst + r * kLdA + c) = reinterpret_cast<const uint32_t*>(src)[i];
  }
}

// Forward pass of up to 64 samples per block.  With Z/H non-NULL it also
// keeps the pre-activations z1..z3 (FP32) and activations h1, h2 (BF16) for
// the backward pass.
__global__ void __launch_bounds__(128) mlp_fwd_kernel(const MlpDev P, const float* __restrict__ xraw, int64_t n,
                                                      float* y, float* Z, __nv_bfloat16* H) {
  extern __shared__ __align__(16) unsigned char sm[];
  float* X = reinterpret_cast<float*>(sm);                                   // [64][4]
  __nv_bfloat16* Ha = reinterpret_cast<__nv_bfloat16*>(sm + 64 * 4 * 4);     // [64][136]
  __nv_bfloat16* Hb = Ha + kRows * kLdA;                                      // [64][136]
  __nv_bfloat16* Ws = Hb + kRows * kLdA;                                      // [128][136]
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  const int tid = threadIdx.x;
  for (int i = tid; i < kRows * 4; i += blockDim.x) {
    const int r = i / 4, f = i % 4;
    const int64_t row = row0 + r;
    X[i] = row < n ? (xraw[row * 4 + f] - P.shift[f]) * P.scale[f] : 0.0f;
  }
  __syncthreads();
  {  // layer 1 in FP32: thread = output column
    const int c = tid;
    const float w0 = P.master[kOffW1 + 0 * kW + c], w1 = P.master[kOffW1 + 1 * kW + c];
    const float w2 = P.master[kOffW1 + 2 * kW + c], w3 = P.master[kOffW1 + 3 * kW + c];
    const float b = P.master[kOffB1 + c];
    for (int r = 0; r < kRows; ++r) {
      const float z = fmaf(X[r * 4 + 0], w0, fmaf(X[r * 4 + 1], w1, fmaf(X[r * 4 + 2], w2, fmaf(X[r * 4 + 3], w3, b))));
      const __nv_bfloat16 hb = __float2bfloat16(siluf_(z));
      Ha[r * kLdA + c] = hb;
      const int64_t row = row0 + r;
      if (Z && row < n) {
        Z[(0 * n + row) * kW + c] = z;
        H[(0 * n + row) * kW + c] = hb;
      }
    }
  }
  load_w(Ws, P.w2t);
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  {  // layer 2: tensor cores
    float acc[1][16][4];
    gemm_bf16<1>(Ha, kLdA, Ws, kLdA, kW, acc);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = warp * 16 + g + (i >= 2 ? 8 : 0), c = nt * 8 + 2 * t + (i & 1);
        const float z = acc[0][nt][i] + P.master[kOffB2 + c];
        const __nv_bfloat16 hb = __float2bfloat16(siluf_(z));
        Hb[r * kLdA + c] = hb;
        const int64_t row = row0 + r;
        if (Z && row < n) {
          Z[(1 * n + row) * kW + c] = z;
          H[(1 * n + row) * kW + c] = hb;
        }
      }
  }
  __syncthreads();
  load_w(Ws, P.w3t);
  __syncthreads();
  {  // layer 3 and the output layer
    float acc[1][16][4];
    gemm_bf16<1>(Hb, kLdA, Ws, kLdA, kW, acc);
    float s0 = 0.0f, s1 = 0.0f;  // rows g and g + 8 of this warp's tile
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = warp * 16 + g + (i >= 2 ? 8 : 0), c = nt * 8 + 2 * t + (i & 1);
        const float z = acc[0][nt][i] + P.master[kOffB3 + c];
        const int64_t row = row0 + r;
        if (Z && row < n) Z[(2 * n + row) * kW + c] = z;
        const float hw = siluf_(z) * P.master[kOffW4 + c];
        if (i < 2)
          s0 += hw;
        else
          s1 += hw;
      }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    if (t == 0) {
      const int64_t ra = row0 + warp * 16 + g, rb = ra + 8;
      const float b4 = P.master[kOffB4];
      if (ra < n) y[ra] = s0 + b4;
      if (rb < n) y[rb] = s1 + b4;
    }
  }
}

// Backward pass through the layers (data gradients), 64 samples per block:
// dz3 = dy W4 s'(z3), dz2 = (dz3 W3^T) s'(z2), dz1 = (dz2 W2^T) s'(z1).
// dy = 2 (y - t) / B for the mean squared error over a batch of B samples.
__global__ void __launch_bounds__(128) mlp_bwd_data_kernel(const MlpDev P, const float* __restrict__ y,
                                                           const float* __restrict__ tgt, float inv_yscale, int64_t n,
                                                           float two_over_b, const float* __restrict__ Z, float* dZ,
                                                           float* dy_out, double* loss_part) {
  extern __shared__ __align__(16) unsigned char sm[];
  float* dy = reinterpret_cast<float*>(sm);                                  // [64]
  __nv_bfloat16* Da = reinterpret_cast<__nv_bfloat16*>(sm + 64 * 4);        // [64][136]
  __nv_bfloat16* Ws = Da + kRows * kLdA;                                     // [128][136]
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  const int tid = threadIdx.x;
  if (tid < kRows) {
    const int64_t row = row0 + tid;
    float r = 0.0f;
    if (row < n) r = y[row] - tgt[row] * inv_yscale;
    dy[tid] = two_over_b * r;
    if (row < n) dy_out[row] = two_over_b * r;
    // per-block sum of squared residuals (fixed order: thread 0 adds below)
    reinterpret_cast<float*>(Ws)[tid] = r * r;
  }
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < kRows; ++i) s += reinterpret_cast<float*>(Ws)[i];
    loss_part[blockIdx.x] = s;
  }
  __syncthreads();
  {  // dz3 = dy W4 s'(z3)
    const int c = tid;
    const float w4 = P.master[kOffW4 + c];
    for (int r = 0; r < kRows; ++r) {
      const int64_t row = row0 + r;
      float d = 0.0f;
      if (row < n) {
        d = dy[r] * w4 * silu_primef_(Z[(2 * n + row) * kW + c]);
        dZ[(2 * n + row) * kW + c] = d;
      }
      Da[r * kLdA + c] = __float2bfloat16(d);
    }
  }
  load_w(Ws, P.w3n);  // B[k = out][n = in] = W3[in][out]: the natural layout is Bt
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  for (int layer = 1; layer >= 0; --layer) {
    float acc[1][16][4];
    gemm_bf16<1>(Da, kLdA, Ws, kLdA, kW, acc);
    __syncthreads();
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = warp * 16 + g + (i >= 2 ? 8 : 0), c = nt * 8 + 2 * t + (i & 1);
        const int64_t row = row0 + r;
        float d = 0.0f;
        if (row < n) {
          d = acc[0][nt][i] * silu_primef_(Z[(layer * n + row) * kW + c]);
          dZ[(layer * n + row) * kW + c] = d;
        }
        Da[r * kLdA + c] = __float2bfloat16(d);
      }
    if (layer == 1) load_w(Ws, P.w2n);
    __syncthreads();
  }
}

// Weight gradients of the two 128 x 128 layers for 64 samples:
// dW2 = h1^T dz2 (blockIdx.y = 0), dW3 = h2^T dz3 (blockIdx.y = 1).
__global__ void __launch_bounds__(128) mlp_bwd_weight_kernel(const __nv_bfloat16* __restrict__ H,
                                                             const float* __restrict__ dZ, int64_t n, float* part) {
  extern __shared__ __align__(16) unsigned char sm[];
  __nv_bfloat16* At = reinterpret_cast<__nv_bfloat16*>(sm);  // [128][72]: h^T
  __nv_bfloat16* Bt = At + kW * kLdT;                         // [128][72]: dz^T
  const int L = blockIdx.y;
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  for (int i = threadIdx.x; i < kRows * kW; i += blockDim.x) {
    const int r = i / kW, c = i % kW;
    const int64_t row = row0 + r;
    const bool ok = row < n;
    At[c * kLdT + r] = ok ? H[((int64_t)L * n + row) * kW + c] : __float2bfloat16(0.0f);
    Bt[c * kLdT + r] = __float2bfloat16(ok ? dZ[((int64_t)(L + 1) * n + row) * kW + c] : 0.0f);
  }
  __syncthreads();
  float acc[2][16][4];
  gemm_bf16<2>(At, kLdT, Bt, kLdT, kRows, acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  float* dst = part + (int64_t)blockIdx.x * kNParams + (L == 0 ? kOffW2 : kOffW3);
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = (warp * 2 + mt) * 16 + g + (i >= 2 ? 8 : 0), c = nt * 8 + 2 * t + (i & 1);
        dst[m * kW + c] = acc[mt][nt][i];
      }
}

// The thin parts of the gradient for 64 samples: dW1 = x^T dz1, biases,
// dW4 = h3^T dy, db4 = sum dy (thread = column).
__global__ void __launch_bounds__(128) mlp_bwd_small_kernel(const MlpDev P, const float* __restrict__ xraw,
                                                            const float* __restrict__ Z, const float* __restrict__ dZ,
                                                            const float* __restrict__ dyv, int64_t n, float* part) {
  const int c = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  float gw1[4] = {0, 0, 0, 0}, gb1 = 0, gb2 = 0, gb3 = 0, gw4 = 0, gb4 = 0;
  for (int r = 0; r < kRows; ++r) {
    const int64_t row = row0 + r;
    if (row >= n) break;
    const float d1 = dZ[(0 * n + row) * kW + c];
#pragma unroll
    for (int f = 0; f < 4; ++f) gw1[f] += (xraw[row * 4 + f] - P.shift[f]) * P.scale[f] * d1;
    gb1 += d1;
    gb2 += dZ[(1 * n + row) * kW + c];
    gb3 += dZ[(2 * n + row) * kW + c];
    const float dy = dyv[row];
    gw4 += siluf_(Z[(2 * n + row) * kW + c]) * dy;
    gb4 += dy;
  }
  float* dst = part + (int64_t)blockIdx.x * kNParams;
#pragma unroll
  for (int f = 0; f < 4; ++f) dst[kOffW1 + f * kW + c] = gw1[f];
  dst[kOffB1 + c] = gb1;
  dst[kOffB2 + c] = gb2;
  dst[kOffB3 + c] = gb3;
  dst[kOffW4 + c] = gw4;
  if (c == 0) dst[kOffB4] = gb4;
}

// Sum the per-block partials (fixed order); optionally write the gradient;
// optionally take an Adam step and refresh the BF16 copies.
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int n_blocks, float* grad, float* master, float* m,
                                  float* v, float lr, float beta1, float beta2, float eps, float bc1, float bc2,
                                  int do_step, __nv_bfloat16* w2t, __nv_bfloat16* w3t, __nv_bfloat16* w2n,
                                  __nv_bfloat16* w3n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  float gsum = 0.0f;
  for (int b = 0; b < n_blocks; ++b) gsum += part[(int64_t)b * kNParams + i];
  if (grad) grad[i] = gsum;
  if (!do_step) return;
  const float mi = beta1 * m[i] + (1.0f - beta1) * gsum;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gsum * gsum;
  m[i] = mi;
  v[i] = vi;
  const float w = master[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  master[i] = w;
  if (i >= kOffW2 && i < kOffW2 + kW * kW) {
    const int j = i - kOffW2, in = j / kW, out = j % kW;
    w2n[in * kW + out] = __float2bfloat16(w);
    w2t[out * kW + in] = __float2bfloat16(w);
  } else if (i >= kOffW3 && i < kOffW3 + kW * kW) {
    const int j = i - kOffW3, in = j / kW, out = j % kW;
    w3n[in * kW + out] = __float2bfloat16(w);
    w3t[out * kW + in] = __float2bfloat16(w);
  }
}

// BF16 copies of W2 and W3 from the master weights.
__global__ void mlp_copies_kernel(const float* master, __nv_bfloat16* w2t, __nv_bfloat16* w3t, __nv_bfloat16* w2n,
                                  __nv_bfloat16* w3n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kW * kW) return;
  const int in = j / kW, out = j % kW;
  w2n[j] = __float2bfloat16(master[kOffW2 + j]);
  w3n[j] = __float2bfloat16(master[kOffW3 + j]);
  w2t[out * kW + in] = w2n[j];
  w3t[out * kW + in] = w3n[j];
}

constexpr size_t kSmemFwd = 64 * 4 * 4 + 2 * kRows * kLdA * 2 + kW * kLdA * 2;
constexpr size_t kSmemBwdData = 64 * 4 + kRows * kLdA * 2 + kW * kLdA * 2;
constexpr size_t kSmemBwdW = 2 * kW * kLdT * 2;

}  // namespace ffe

// --------------------------------------------------------------- host side
using namespace ffe;

struct ffe_surrogate {
  ffe_context* ctx = nullptr;
  ffe_surrogate_meta meta;
  float* master = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wcopies = nullptr;  // w2t, w3t, w2n, w3n
  int64_t adam_t = 0;
  // training scratch, sized for `cap` samples
  int64_t cap = 0;
  float *x = nullptr, *t = nullptr, *y = nullptr, *Z = nullptr, *dZ = nullptr, *dy = nullptr, *part = nullptr;
  double* loss_part = nullptr;
  __nv_bfloat16* H = nullptr;
  float* grad = nullptr;
  cudaStream_t stream = nullptr;
};

namespace {

MlpDev make_dev(const ffe_surrogate* s) {
  MlpDev P;
  P.master = s->master;
  P.w2t = s->wcopies;
  P.w3t = s->wcopies + kW * kW;
  P.w2n = s->wcopies + 2 * kW * kW;
  P.w3n = s->wcopies + 3 * kW * kW;
  for (int f = 0; f < 4; ++f) {
    P.shift[f] = s->meta.shift[f];
    P.scale[f] = s->meta.scale[f];
  }
  return P;
}

ffe_status sfail(ffe_surrogate* s, cudaError_t e, const char* what) { return cuda_fail(s->ctx, e, what); }

#define SUR_CU(call, what)                                \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return sfail(s, e_, what);     \
  } while (0)

void free_scratch(ffe_surrogate* s) {
  for (void* p : {(void*)s->x, (void*)s->t, (void*)s->y, (void*)s->Z, (void*)s->dZ, (void*)s->dy, (void*)s->part,
                  (void*)s->loss_part, (void*)s->H})
    if (p) cudaFree(p);
  s->x = s->t = s->y = s->Z = s->dZ = s->dy = s->part = nullptr;
  s->loss_part = nullptr;
  s->H = nullptr;
  s->cap = 0;
}

ffe_status ensure_scratch(ffe_surrogate* s, int64_t n) {
  if (n <= s->cap) return FFE_OK;
  free_scratch(s);
  const int64_t nb = (n + kRows - 1) / kRows;
  SUR_CU(cudaMalloc(&s->x, n * 4 * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->t, n * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->y, n * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->dy, n * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->Z, 3 * n * kW * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->dZ, 3 * n * kW * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->H, 2 * n * kW * sizeof(__nv_bfloat16)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->part, nb * kNParams * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->loss_part, nb * sizeof(double)), "cudaMalloc");
  s->cap = n;
  return FFE_OK;
}

ffe_status set_attrs(ffe_surrogate* s) {
  SUR_CU(cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemFwd), "attr");
  SUR_CU(cudaFuncSetAttribute(mlp_bwd_data_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBwdData),
         "attr");
  SUR_CU(cudaFuncSetAttribute(mlp_bwd_weight_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBwdW),
         "attr");
  return FFE_OK;
}

// One forward + backward over samples [0, n) of the device arrays x/t
// (offset already applied), gradient partials into s->part.
ffe_status fwd_bwd(ffe_surrogate* s, const float* x, const float* t, int64_t n, cudaStream_t st) {
  const MlpDev P = make_dev(s);
  const int nb = (int)((n + kRows - 1) / kRows);
  mlp_fwd_kernel<<<nb, 128, kSmemFwd, st>>>(P, x, n, s->y, s->Z, s->H);
  SUR_CU(cudaGetLastError(), "mlp_fwd");
  mlp_bwd_data_kernel<<<nb, 128, kSmemBwdData, st>>>(P, s->y, t, 1.0f / s->meta.y_scale, n, 2.0f / (float)n, s->Z,
                                                      s->dZ, s->dy, s->loss_part);
  SUR_CU(cudaGetLastError(), "mlp_bwd_data");
  mlp_bwd_weight_kernel<<<dim3(nb, 2), 128, kSmemBwdW, st>>>(s->H, s->dZ, n, s->part);
  SUR_CU(cudaGetLastError(), "mlp_bwd_weight");
  mlp_bwd_small_kernel<<<nb, 128, 0, st>>>(P, x, s->Z, s->dZ, s->dy, n, s->part);
  SUR_CU(cudaGetLastError(), "mlp_bwd_small");
  return FFE_OK;
}

}  // namespace

extern "C" {

ffe_status ffe_surrogate_create(ffe_context* ctx, const ffe_surrogate_meta* meta, const float* params,
                                ffe_surrogate** out) {
  if (!ctx || !meta || !out) return FFE_EINVAL;
  *out = nullptr;
  if (!(meta->y_scale > 0.0f)) return set_err(ctx, "y_scale must be > 0"), FFE_EINVAL;
  ffe_surrogate* s = new (std::nothrow) ffe_surrogate();
  if (!s) return FFE_ENOMEM;
  s->ctx = ctx;
  s->meta = *meta;
  cudaError_t e = cudaMalloc(&s->master, kNParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->m, kNParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->v, kNParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->wcopies, 4 * kW * kW * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&s->grad, kNParams * sizeof(float));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    ffe_status st = cuda_fail(ctx, e, "surrogate alloc");
    ffe_surrogate_destroy(s);
    return st;
  }
  ffe_status st = set_attrs(s);
  if (st == FFE_OK) st = ffe_surrogate_set_params(s, params);
  if (st != FFE_OK) {
    ffe_surrogate_destroy(s);
    return st;
  }
  *out = s;
  return FFE_OK;
}

void ffe_surrogate_destroy(ffe_surrogate* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_scratch(s);
  for (void* p : {(void*)s->master, (void*)s->m, (void*)s->v, (void*)s->wcopies, (void*)s->grad})
    if (p) cudaFree(p);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

ffe_status ffe_surrogate_set_params(ffe_surrogate* s, const float* params) {
  if (!s) return FFE_EINVAL;
  std::vector<float> zeros;
  if (!params) {
    zeros.assign(kNParams, 0.0f);
    params = zeros.data();
  }
  SUR_CU(cudaMemcpy(s->master, params, kNParams * sizeof(float), cudaMemcpyHostToDevice), "set params");
  SUR_CU(cudaMemset(s->m, 0, kNParams * sizeof(float)), "memset");
  SUR_CU(cudaMemset(s->v, 0, kNParams * sizeof(float)), "memset");
  s->adam_t = 0;
  mlp_copies_kernel<<<(kW * kW + 255) / 256, 256, 0, s->stream>>>(s->master, s->wcopies, s->wcopies + kW * kW,
                                                                   s->wcopies + 2 * kW * kW, s->wcopies + 3 * kW * kW);
  SUR_CU(cudaGetLastError(), "copies");
  SUR_CU(cudaStreamSynchronize(s->stream), "sync");
  return FFE_OK;
}

ffe_status ffe_surrogate_get_params(ffe_surrogate* s, float* params) {
  if (!s || !params) return FFE_EINVAL;
  SUR_CU(cudaStreamSynchronize(s->stream), "sync");
  SUR_CU(cudaMemcpy(params, s->master, kNParams * sizeof(float), cudaMemcpyDeviceToHost), "get params");
  return FFE_OK;
}

ffe_status ffe_surrogate_predict(ffe_surrogate* s, const float* xraw, int64_t n, float* y, void* stream) {
  if (!s || !xraw || !y || n < 1) return FFE_EINVAL;
  (void)stream;
  ffe_status st = ensure_scratch(s, n);
  if (st != FFE_OK) return st;
  cudaStream_t cs = s->stream;
  SUR_CU(cudaMemcpyAsync(s->x, xraw, n * 4 * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  const int nb = (int)((n + kRows - 1) / kRows);
  mlp_fwd_kernel<<<nb, 128, kSmemFwd, cs>>>(make_dev(s), s->x, n, s->y, nullptr, nullptr);
  SUR_CU(cudaGetLastError(), "mlp_fwd");
  std::vector<float> yn(n);
  SUR_CU(cudaMemcpyAsync(yn.data(), s->y, n * sizeof(float), cudaMemcpyDeviceToHost, cs), "download");
  SUR_CU(cudaStreamSynchronize(cs), "sync");
  for (int64_t i = 0; i < n; ++i) y[i] = yn[i] * s->meta.y_scale;
  return FFE_OK;
}

ffe_status ffe_surrogate_grad(ffe_surrogate* s, const float* xraw, const float* traw, int64_t n, float* grad,
                              double* loss, void* stream) {
  if (!s || !xraw || !traw || !grad || n < 1) return FFE_EINVAL;
  (void)stream;
  ffe_status st = ensure_scratch(s, n);
  if (st != FFE_OK) return st;
  cudaStream_t cs = s->stream;
  SUR_CU(cudaMemcpyAsync(s->x, xraw, n * 4 * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  SUR_CU(cudaMemcpyAsync(s->t, traw, n * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  if ((st = fwd_bwd(s, s->x, s->t, n, cs)) != FFE_OK) return st;
  const int nb = (int)((n + kRows - 1) / kRows);
  mlp_reduce_kernel<<<(kNParams + 255) / 256, 256, 0, cs>>>(s->part, nb, s->grad, nullptr, nullptr, nullptr, 0, 0, 0,
                                                             0, 1, 1, 0, nullptr, nullptr, nullptr, nullptr);
  SUR_CU(cudaGetLastError(), "reduce");
  std::vector<double> lp(nb);
  SUR_CU(cudaMemcpyAsync(grad, s->grad, kNParams * sizeof(float), cudaMemcpyDeviceToHost, cs), "download");
  SUR_CU(cudaMemcpyAsync(lp.data(), s->loss_part, nb * sizeof(double), cudaMemcpyDeviceToHost, cs), "download");
  SUR_CU(cudaStreamSynchronize(cs), "sync");
  if (loss) {
    double tot = 0.0;
    for (double v : lp) tot += v;
    *loss = tot / (double)n;
  }
  return FFE_OK;
}

ffe_status ffe_surrogate_train(ffe_surrogate* s, const float* xraw, const float* traw, int64_t n, int32_t epochs,
                               int32_t batch, float lr, float* loss_per_epoch, void* stream) {
  if (!s || !xraw || !traw || n < 1 || epochs < 1 || batch < kRows || batch % kRows != 0 || !(lr > 0.0f))
    return s ? (set_err(s->ctx, "train: bad arguments (batch a multiple of 64)"), FFE_EINVAL) : FFE_EINVAL;
  (void)stream;
  ffe_status st = ensure_scratch(s, std::max<int64_t>(n, batch));
  if (st != FFE_OK) return st;
  cudaStream_t cs = s->stream;
  SUR_CU(cudaMemcpyAsync(s->x, xraw, n * 4 * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  SUR_CU(cudaMemcpyAsync(s->t, traw, n * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int64_t steps = n / batch;  // the tail that does not fill a batch is left out of the epoch
  if (steps < 1) return set_err(s->ctx, "train: fewer samples than one batch"), FFE_EINVAL;
  std::vector<double> lp((batch + kRows - 1) / kRows);
  for (int ep = 0; ep < epochs; ++ep) {
    double ep_loss = 0.0;
    for (int64_t k = 0; k < steps; ++k) {
      const int64_t off = k * batch;
      if ((st = fwd_bwd(s, s->x + off * 4, s->t + off, batch, cs)) != FFE_OK) return st;
      ++s->adam_t;
      const float bc1 = 1.0f - powf(b1, (float)s->adam_t), bc2 = 1.0f - powf(b2, (float)s->adam_t);
      mlp_reduce_kernel<<<(kNParams + 255) / 256, 256, 0, cs>>>(
          s->part, batch / kRows, nullptr, s->master, s->m, s->v, lr, b1, b2, eps, bc1, bc2, 1, s->wcopies,
          s->wcopies + kW * kW, s->wcopies + 2 * kW * kW, s->wcopies + 3 * kW * kW);
      SUR_CU(cudaGetLastError(), "adam");
      if (loss_per_epoch) {
        SUR_CU(cudaMemcpyAsync(lp.data(), s->loss_part, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, cs),
               "download");
        SUR_CU(cudaStreamSynchronize(cs), "sync");
        for (double v : lp) ep_loss += v;
      }
    }
    if (loss_per_epoch) loss_per_epoch[ep] = (float)(ep_loss / (double)(steps * batch));
  }
  SUR_CU(cudaStreamSynchronize(cs), "sync");
  return FFE_OK;
}

}  // extern "C"

namespace ffe {

ffe_status surrogate_infer_device(ffe_surrogate* s, const float* x, int64_t n, float* y, cudaStream_t st) {
  if (n < 1) return FFE_OK;
  const int nb = (int)((n + kRows - 1) / kRows);
  mlp_fwd_kernel<<<nb, 128, kSmemFwd, st>>>(make_dev(s), x, n, y, nullptr, nullptr);
  SUR_CU(cudaGetLastError(), "mlp_fwd");
  return FFE_OK;
}

float surrogate_y_scale(const ffe_surrogate* s) { return s->meta.y_scale; }

}  // namespace ffe
