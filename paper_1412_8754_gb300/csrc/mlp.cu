// mlp.cu -- the learned surrogate of Omega: a 4 -> 128 -> 128 -> 128 -> 1 MLP
// with SiLU activations over (q, h, T, Delta), trained on free energies the
// k-sum itself produced.  (The paper has no learned component; the surrogate
// only proposes where the exact k-sum should look.)
//
// Precision: the two 128 x 128 layers multiply BF16 activations by BF16
// weights on the 5th-generation tensor cores (tcgen05.mma, kind::f16, FP32
// accumulators in tensor memory); the 4-wide input layer, the 1-wide output
// layer, SiLU, its derivative and the loss are FP32.  Master weights and Adam
// moments are FP32.  Every reduction over samples is a fixed-order sum of
// per-block partials (deterministic).
//
// One CTA owns 128 samples (the MMA's M) with kSplit threads per sample:
// thread t works on sample t mod 128, which is TMEM lane t mod 128 of the
// accumulator (warp w reads lanes 32 (w mod 4) .. 32 (w mod 4) + 31), and on
// kCols consecutive columns of it, so every SIMT epilogue is kCols deep.
// Each 128 x 128 product is eight K = 16 MMAs issued by one thread from two
// shared-memory tiles (the activations and the weights) and committed to an
// mbarrier; the weights' tiles arrive by one bulk asynchronous copy (TMA)
// each.  Tiles are in the canonical K-major layout without swizzle: 8 x 16-byte
// core matrices, 128 B apart along K and 2048 B apart along M/N.
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
constexpr int kRows = 128;    // samples per block (the MMA's M)
constexpr int kTile = kW * kW;  // bf16 elements of one 128 x 128 tile
constexpr int kTileBytes = kTile * 2;
constexpr int kOffW1 = 0, kOffB1 = 512, kOffW2 = 640, kOffB2 = 17024, kOffW3 = 17152, kOffB3 = 33536,
              kOffW4 = 33664, kOffB4 = 33792, kNParams = 33793;
constexpr int kPartStride = 33796;  // floats per block of gradient partials (16-byte rows)
// Threads of the forward and data-gradient kernels: kSplit per sample, each
// owning kW / kSplit consecutive columns of its sample's row.
constexpr int kSplit = 8, kThreads = kSplit * kRows, kCols = kW / kSplit;
// BF16 weight tiles (global, each in the MMA layout): the B operands of the
// forward products (n = out, k = in) and of the data-gradient products
// (n = in, k = out)
enum { kT2f = 0, kT3f = 1, kT2b = 2, kT3b = 3 };
constexpr unsigned kWaitLimit = 1u << 26;  // polls of an mbarrier before giving up
constexpr int kMaxEpochs = 1000000;         // epochs of one training call

struct MlpDev {
  const float* master;          // FP32 parameters (layout above)
  const __nv_bfloat16* tiles;   // the four weight tiles
  float shift[4], scale[4];
  int32_t* status;              // set to 1 when a wait gave up
};

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + __expf(-z)); }
__device__ __forceinline__ float siluf_(float z) { return z * sigmoidf_(z); }
__device__ __forceinline__ float silu_primef_(float z) {
  const float s = sigmoidf_(z);
  return s * (1.0f + z * (1.0f - s));
}

// Byte offset of element (r, k) of a 128 x 128 BF16 tile in the K-major
// no-swizzle layout: core matrix (r / 8, k / 8), 16-byte rows inside it.
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)((((r >> 3) << 4) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

// ---- tcgen05 / mbarrier helpers (inline PTX) ---------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) byte offset 128,
// stride (M/N) byte offset 2048, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tile_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(2048 >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

// Bounded wait on a phase of an mbarrier; false when it gave up (status set).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int32_t* status) {
  uint32_t done = 0;
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity));
    if (done) return true;
  }
  atomicOr(status, 1);
  return false;
}

// One 32 KB weight tile from global memory by the bulk copy engine, completing
// on bar (whose expected transaction bytes the caller has set).
__device__ __forceinline__ void tile_load_async(void* dst, const void* src, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(kTileBytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes));
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {  // one warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_addr(slot)));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t tmem) {  // the same warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// Generic-proxy writes of shared memory made visible to the tensor cores.
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[128 x 128] (TMEM) = A[128 x 128] * B[128 x 128]^T from two K-major tiles;
// one thread issues, the commit arrives on bar when the products are done.
__device__ __forceinline__ void mma_tile(uint32_t tmem, const void* a, const void* b, uint64_t* bar) {
  const uint32_t a0 = smem_addr(a), b0 = smem_addr(b);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint64_t ad = tile_desc(a0 + k * 256), bd = tile_desc(b0 + k * 256);  // K = 16: two core matrices
    const uint32_t acc = k > 0 ? 1u : 0u;
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar)));
}

// NC (16 or 32) consecutive FP32 accumulator columns of this thread's TMEM
// lane (warp w reads lanes 32 (w mod 4) .. 32 (w mod 4) + 31).
template <int NC>
__device__ __forceinline__ void tmem_row(uint32_t tmem, int c0, float (&v)[NC]) {
  static_assert(NC == 16 || NC == 32, "16 or 32 columns");
  const uint32_t ta = tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + (uint32_t)c0;
  uint32_t r[NC];
  if constexpr (NC == 32) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta));
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < NC; ++j) v[j] = __uint_as_float(r[j]);
}

// Eight values of row r, columns c0..c0+7 (c0 % 8 == 0), into a tile: one 16-byte store.
__device__ __forceinline__ void tile_store8(unsigned char* tile, int r, int c0, const float* v) {
  __align__(16) __nv_bfloat162 p[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) p[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
  *reinterpret_cast<uint4*>(tile + tile_off(r, c0)) = *reinterpret_cast<const uint4*>(p);
}

// The MMA of one layer and the wait for it, with the fences that order it
// after the threads' tile writes and TMEM reads.  Returns false if the wait
// gave up.
__device__ __forceinline__ bool layer_mma(uint32_t tmem, const void* a, const void* b, uint64_t* bar,
                                          uint32_t parity, int32_t* status) {
  proxy_fence();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (threadIdx.x == 0) mma_tile(tmem, a, b, bar);
  const bool ok = mbar_wait(bar, parity, status);
  tc_after_sync();
  return ok;
}

// Shared-memory plan of the kernels: up to three tiles, then the barriers, the
// TMEM address and small FP32 parameters.
constexpr size_t kSmemTiles3 = 3 * (size_t)kTileBytes;
constexpr size_t kSmemExtra = 64 + 4 * 1088 + 4 * kSplit * kRows;
constexpr size_t kSmemFwd = kSmemTiles3 + kSmemExtra;
constexpr size_t kSmemBwdData = kSmemTiles3 + kSmemExtra;
constexpr size_t kSmemBwdW = 2 * (size_t)kTileBytes + kSmemExtra;

struct Bars {
  uint64_t w, mma;
  uint32_t tmem;
  int32_t ok;
};

// Forward pass of up to 128 samples per block, kSplit threads per sample
// (thread t: sample t mod 128, columns kCols (t / 128) onwards).  With Z/H
// non-NULL it also keeps the pre-activations z1..z3 (FP32) and activations
// h1, h2 (BF16), each as [layer][feature][ld] (ld >= the rows of every block,
// a multiple of 128) for the backward pass; rows of the block at or beyond n
// are computed from x = 0 and kept too (the backward pass gives them zero
// weight).
__global__ void __launch_bounds__(kThreads, 1) mlp_fwd_kernel(const MlpDev P, const float* __restrict__ xraw,
                                                              int64_t n, float* __restrict__ y, float* __restrict__ Z,
                                                              __nv_bfloat16* __restrict__ H, int64_t ld) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* T2 = sm;
  unsigned char* T3 = sm + kTileBytes;
  unsigned char* Ht = sm + 2 * kTileBytes;
  Bars* bars = reinterpret_cast<Bars*>(sm + kSmemTiles3);
  float* prm = reinterpret_cast<float*>(sm + kSmemTiles3 + 64);  // W1 (512), b1, b2, b3, W4 (128 each), b4
  float* outp = prm + 1088;                                        // [kSplit][128] output-layer partials
  const int tid = threadIdx.x, rl = tid & (kRows - 1), cb = (tid / kRows) * kCols;
  if (tid == 0) {
    mbar_init(&bars->w, 1);
    mbar_init(&bars->mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    expect_tx(&bars->w, 2 * kTileBytes);
    tile_load_async(T2, P.tiles + kT2f * kTile, &bars->w);
    tile_load_async(T3, P.tiles + kT3f * kTile, &bars->w);
  }
  if (tid < 32) tmem_alloc(&bars->tmem);
  for (int i = tid; i < 512; i += kThreads) prm[i] = P.master[kOffW1 + i];
  for (int i = tid; i < kW; i += kThreads) {
    prm[512 + i] = P.master[kOffB1 + i];
    prm[640 + i] = P.master[kOffB2 + i];
    prm[768 + i] = P.master[kOffB3 + i];
    prm[896 + i] = P.master[kOffW4 + i];
  }
  if (tid == 0) prm[1024] = P.master[kOffB4];
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = bars->tmem;
  const int64_t row = (int64_t)blockIdx.x * kRows + rl;
  const bool live = row < n;
  float x[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) x[f] = live ? (xraw[row * 4 + f] - P.shift[f]) * P.scale[f] : 0.0f;
  // layer 1 in FP32
  for (int c0 = cb; c0 < cb + kCols; c0 += 8) {
    float h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + j;
      const float z = fmaf(x[0], prm[c], fmaf(x[1], prm[128 + c], fmaf(x[2], prm[256 + c],
                                                                         fmaf(x[3], prm[384 + c], prm[512 + c]))));
      h[j] = siluf_(z);
      if (Z) {
        Z[(0 * kW + c) * ld + row] = z;
        H[(0 * kW + c) * ld + row] = __float2bfloat16(h[j]);
      }
    }
    tile_store8(Ht, rl, c0, h);
  }
  if (tid == 0) bars->ok = mbar_wait(&bars->w, 0, P.status) ? 1 : 0;  // the weight tiles are in
  bool ok = layer_mma(tmem, Ht, T2, &bars->mma, 0, P.status) && bars->ok;
  {  // layer 2 epilogue: bias, SiLU, next layer's A tile
    float v[kCols];
    tmem_row<kCols>(tmem, cb, v);
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      const int c = cb + j;
      const float z = v[j] + prm[640 + c];
      v[j] = siluf_(z);
      if (Z) {
        Z[(1 * kW + c) * ld + row] = z;
        H[(1 * kW + c) * ld + row] = __float2bfloat16(v[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kCols; j += 8) tile_store8(Ht, rl, cb + j, v + j);
  }
  ok = layer_mma(tmem, Ht, T3, &bars->mma, 1, P.status) && ok;
  {  // layer 3 epilogue and this thread's share of the output layer
    float v[kCols];
    tmem_row<kCols>(tmem, cb, v);
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      const int c = cb + j;
      const float z = v[j] + prm[768 + c];
      if (Z) Z[(2 * kW + c) * ld + row] = z;
      acc = fmaf(siluf_(z), prm[896 + c], acc);
    }
    outp[tid] = acc;
  }
  tc_before_sync();
  __syncthreads();
  if (tid < kRows && live) {  // the shares of sample tid in a fixed order
    float acc = outp[tid];
#pragma unroll
    for (int p = 1; p < kSplit; ++p) acc += outp[p * kRows + tid];
    y[row] = ok ? acc + prm[1024] : NAN;
  }
  if (tid < 32) tmem_free(tmem);
}

// Backward pass through the layers (data gradients), 128 samples per block,
// kSplit threads per sample as in the forward pass:
// dz3 = dy W4 s'(z3), dz2 = (dz3 W3^T) s'(z2), dz1 = (dz2 W2^T) s'(z1).
// dy = 2 (y - t) / B for the mean squared error over a batch of B samples.
// dZ is written for every row of the block (zero at and beyond n).
__global__ void __launch_bounds__(kThreads, 1) mlp_bwd_data_kernel(const MlpDev P, const float* __restrict__ y,
                                                                   const float* __restrict__ tgt, float inv_yscale,
                                                                   int64_t n, float two_over_b,
                                                                   const float* __restrict__ Z, float* __restrict__ dZ,
                                                                   float* __restrict__ dy_out,
                                                                   double* __restrict__ loss_part, int64_t ld) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* T3 = sm;                    // B of dz2 = dz3 W3^T: (n = in, k = out)
  unsigned char* T2 = sm + kTileBytes;       // B of dz1 = dz2 W2^T
  unsigned char* Dt = sm + 2 * kTileBytes;   // the data gradient of the current layer, A
  Bars* bars = reinterpret_cast<Bars*>(sm + kSmemTiles3);
  float* red = reinterpret_cast<float*>(sm + kSmemTiles3 + 64);  // [128] squared residuals
  float* w4 = red + kRows;                                        // [128] W4
  const int tid = threadIdx.x, rl = tid & (kRows - 1), cb = (tid / kRows) * kCols;
  if (tid == 0) {
    mbar_init(&bars->w, 1);
    mbar_init(&bars->mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    expect_tx(&bars->w, 2 * kTileBytes);
    tile_load_async(T3, P.tiles + kT3b * kTile, &bars->w);
    tile_load_async(T2, P.tiles + kT2b * kTile, &bars->w);
  }
  if (tid < 32) tmem_alloc(&bars->tmem);
  for (int i = tid; i < kW; i += kThreads) w4[i] = P.master[kOffW4 + i];
  const int64_t row = (int64_t)blockIdx.x * kRows + rl;
  const bool live = row < n;
  const float r = live ? y[row] - tgt[row] * inv_yscale : 0.0f;
  const float dy = two_over_b * r;
  if (tid < kRows) {
    if (live) dy_out[row] = dy;
    red[tid] = r * r;
  }
  // this thread's columns of the saved pre-activations, loaded before any store
  float z[kCols];
#pragma unroll
  for (int j = 0; j < kCols; ++j) z[j] = live ? Z[(2 * kW + cb + j) * ld + row] : 0.0f;
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (tid < 32) {  // per-block sum of squared residuals: four per lane, then a fixed butterfly
    double s = ((double)red[tid] + (double)red[tid + 32]) + ((double)red[tid + 64] + (double)red[tid + 96]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) loss_part[blockIdx.x] = s;
  }
  const uint32_t tmem = bars->tmem;
#pragma unroll
  for (int j = 0; j < kCols; ++j) {  // dz3 = dy W4 s'(z3)
    z[j] = live ? dy * w4[cb + j] * silu_primef_(z[j]) : 0.0f;
    dZ[(2 * kW + cb + j) * ld + row] = z[j];
  }
#pragma unroll
  for (int j = 0; j < kCols; j += 8) tile_store8(Dt, rl, cb + j, z + j);
  if (tid == 0) bars->ok = mbar_wait(&bars->w, 0, P.status) ? 1 : 0;
  bool ok = true;
  for (int layer = 1; layer >= 0; --layer) {
#pragma unroll
    for (int j = 0; j < kCols; ++j) z[j] = live ? Z[(layer * kW + cb + j) * ld + row] : 0.0f;
    ok = layer_mma(tmem, Dt, layer == 1 ? T3 : T2, &bars->mma, layer == 1 ? 0 : 1, P.status) && bars->ok && ok;
    float v[kCols];
    tmem_row<kCols>(tmem, cb, v);
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      v[j] = live ? (ok ? v[j] : NAN) * silu_primef_(z[j]) : 0.0f;
      dZ[(layer * kW + cb + j) * ld + row] = v[j];
    }
    if (layer == 1) {
      // every thread's reads of the layer's TMEM result and of the A tile are
      // done before the tile is overwritten (the MMA that read it has completed)
#pragma unroll
      for (int j = 0; j < kCols; j += 8) tile_store8(Dt, rl, cb + j, v + j);
    }
  }
  tc_before_sync();
  __syncthreads();
  if (tid < 32) tmem_free(tmem);
}

// The thin parts of the gradient for 128 samples: dW1 = x^T dz1, biases,
// dW4 = h3^T dy, db4 = sum dy.  Thread t sums column t mod 128 over the 32
// rows 32 (t / 128) .. 32 (t / 128) + 31 (each column's rows are contiguous in
// the feature-major arrays and read four at a time; rows at or beyond n have
// zero data gradients); the kSplit row-segment sums are then added in a fixed
// order.  sh: (5 + 9 kSplit) 128 floats of shared memory.
__device__ __forceinline__ void bwd_small_block(const MlpDev& P, const float* __restrict__ xraw,
                                                const float* __restrict__ Z, const float* __restrict__ dZ,
                                                const float* __restrict__ dyv, int64_t n, float* __restrict__ part,
                                                int64_t ld, float* sh) {
  constexpr int kSeg = kRows / kSplit, kNv = 9;  // rows per thread, sums per column
  float(*xs)[4] = reinterpret_cast<float(*)[4]>(sh);
  float* dys = sh + 4 * kRows;
  float* psum = dys + kRows;  // [kNv][kSplit][128]
  const int tid = threadIdx.x, c = tid & (kRows - 1), seg = tid / kRows;
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  if (tid < kRows) {
    const int64_t row = row0 + tid;
    const bool live = row < n;
#pragma unroll
    for (int f = 0; f < 4; ++f) xs[tid][f] = live ? (xraw[row * 4 + f] - P.shift[f]) * P.scale[f] : 0.0f;
    dys[tid] = live ? dyv[row] : 0.0f;
  }
  __syncthreads();
  const int64_t rs = row0 + seg * kSeg;
  const float4* d1 = reinterpret_cast<const float4*>(dZ + (0 * kW + c) * ld + rs);
  const float4* d2 = reinterpret_cast<const float4*>(dZ + (1 * kW + c) * ld + rs);
  const float4* d3 = reinterpret_cast<const float4*>(dZ + (2 * kW + c) * ld + rs);
  const float4* z3 = reinterpret_cast<const float4*>(Z + (2 * kW + c) * ld + rs);
  float g[kNv] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // dW1 (4), db1, db2, db3, dW4, db4
#pragma unroll 1
  for (int r4 = 0; r4 < kSeg / 4; ++r4) {
    const float4 a = d1[r4], b = d2[r4], e = d3[r4], z = z3[r4];
    const float av[4] = {a.x, a.y, a.z, a.w}, zv[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = seg * kSeg + 4 * r4 + i;
#pragma unroll
      for (int f = 0; f < 4; ++f) g[f] += xs[r][f] * av[i];
      g[7] += siluf_(zv[i]) * dys[r];
      g[8] += dys[r];
    }
    g[4] += (a.x + a.y) + (a.z + a.w);
    g[5] += (b.x + b.y) + (b.z + b.w);
    g[6] += (e.x + e.y) + (e.z + e.w);
  }
#pragma unroll
  for (int k = 0; k < kNv; ++k) psum[(k * kSplit + seg) * kRows + c] = g[k];
  __syncthreads();
  if (tid >= kRows) return;
#pragma unroll
  for (int k = 0; k < kNv; ++k) {
    float t = psum[(k * kSplit) * kRows + c];
#pragma unroll
    for (int q = 1; q < kSplit; ++q) t += psum[(k * kSplit + q) * kRows + c];
    g[k] = t;
  }
  float* dst = part + (int64_t)blockIdx.x * kPartStride;
#pragma unroll
  for (int f = 0; f < 4; ++f) dst[kOffW1 + f * kW + c] = g[f];
  dst[kOffB1 + c] = g[4];
  dst[kOffB2 + c] = g[5];
  dst[kOffB3 + c] = g[6];
  dst[kOffW4 + c] = g[7];
  if (c == 0) dst[kOffB4] = g[8];
}

// Weight gradients for 128 samples: dW2 = h1^T dz2 (blockIdx.y = 0),
// dW3 = h2^T dz3 (blockIdx.y = 1), as D[i][o] = sum_s A[i][s] B[o][s] with
// A = h^T, B = dz^T (both K-major in s) on the tensor cores, thread t reading
// out columns kCols (t / 128) onwards of row t mod 128; the thin parts
// (blockIdx.y = 2) on the FP32 pipe.
__global__ void __launch_bounds__(kThreads, 1) mlp_bwd_weight_kernel(const MlpDev P,
                                                                     const __nv_bfloat16* __restrict__ H,
                                                                     const float* __restrict__ dZ,
                                                                     float* __restrict__ part, int64_t ld,
                                                                     const float* __restrict__ xraw,
                                                                     const float* __restrict__ Z,
                                                                     const float* __restrict__ dyv, int64_t n) {
  extern __shared__ __align__(1024) unsigned char sm[];
  if (blockIdx.y == 2) {
    bwd_small_block(P, xraw, Z, dZ, dyv, n, part, ld, reinterpret_cast<float*>(sm));
    return;
  }
  unsigned char* At = sm;
  unsigned char* Bt = sm + kTileBytes;
  Bars* bars = reinterpret_cast<Bars*>(sm + 2 * kTileBytes);
  const int L = blockIdx.y, tid = threadIdx.x, rl = tid & (kRows - 1), cb = (tid / kRows) * kCols;
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  if (tid == 0) {
    mbar_init(&bars->mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < 32) tmem_alloc(&bars->tmem);
  // rows i of A (features) and o of B: 8 consecutive samples per 16-byte store
  for (int e = tid; e < kW * (kRows / 8); e += kThreads) {
    const int f = e / (kRows / 8), s0 = (e % (kRows / 8)) * 8;
    *reinterpret_cast<uint4*>(At + tile_off(f, s0)) =
        *reinterpret_cast<const uint4*>(H + ((int64_t)L * kW + f) * ld + row0 + s0);
    const float4 a = *reinterpret_cast<const float4*>(dZ + ((int64_t)(L + 1) * kW + f) * ld + row0 + s0);
    const float4 b = *reinterpret_cast<const float4*>(dZ + ((int64_t)(L + 1) * kW + f) * ld + row0 + s0 + 4);
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    tile_store8(Bt, f, s0, v);
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = bars->tmem;
  const bool ok = layer_mma(tmem, At, Bt, &bars->mma, 0, P.status);
  float* dst = part + (int64_t)blockIdx.x * kPartStride + (L == 0 ? kOffW2 : kOffW3) + (int64_t)rl * kW + cb;
  {
    float v[kCols];
    tmem_row<kCols>(tmem, cb, v);
#pragma unroll
    for (int j = 0; j < kCols; j += 4)
      *reinterpret_cast<float4*>(dst + j) =
          ok ? make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]) : make_float4(NAN, NAN, NAN, NAN);
  }
  tc_before_sync();
  __syncthreads();
  if (tid < 32) tmem_free(tmem);
}

// The weight tiles of W2 / W3 element (in, out) in the MMA layout.
__device__ __forceinline__ void put_weight(__nv_bfloat16* tiles, int layer3, int in, int out, float w) {
  const __nv_bfloat16 b = __float2bfloat16(w);
  tiles[(layer3 ? kT3f : kT2f) * kTile + tile_off(out, in) / 2] = b;  // forward: n = out, k = in
  tiles[(layer3 ? kT3b : kT2b) * kTile + tile_off(in, out) / 2] = b;  // backward: n = in, k = out
}

// Sum the per-block partials (fixed order); optionally write the gradient;
// optionally take an Adam step and refresh the BF16 tiles.  With loss_total
// non-NULL the grid has one more block, whose first thread adds the step's
// loss partials (fixed order) to *loss_total.
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int n_blocks, float* grad, float* master, float* m,
                                  float* v, float lr, float beta1, float beta2, float eps, float bc1, float bc2,
                                  int do_step, __nv_bfloat16* tiles, const double* __restrict__ loss_part,
                                  double* loss_total) {
  if (loss_total && blockIdx.x == gridDim.x - 1) {
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int b = 0; b < n_blocks; ++b) s += loss_part[b];
      *loss_total += s;
    }
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  float gsum = 0.0f;
  for (int b = 0; b < n_blocks; ++b) gsum += part[(int64_t)b * kPartStride + i];
  if (grad) grad[i] = gsum;
  if (!do_step) return;
  const float mi = beta1 * m[i] + (1.0f - beta1) * gsum;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gsum * gsum;
  m[i] = mi;
  v[i] = vi;
  const float w = master[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  master[i] = w;
  if (i >= kOffW2 && i < kOffW2 + kW * kW) {
    const int j = i - kOffW2;
    put_weight(tiles, 0, j / kW, j % kW, w);
  } else if (i >= kOffW3 && i < kOffW3 + kW * kW) {
    const int j = i - kOffW3;
    put_weight(tiles, 1, j / kW, j % kW, w);
  }
}

// BF16 tiles of W2 and W3 from the master weights.
__global__ void mlp_copies_kernel(const float* master, __nv_bfloat16* tiles) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kW * kW) return;
  put_weight(tiles, 0, j / kW, j % kW, master[kOffW2 + j]);
  put_weight(tiles, 1, j / kW, j % kW, master[kOffW3 + j]);
}

// Training targets: y = (omega - omega of the line's first value) / N^2, one thread per value.
__global__ void targets_kernel(const double* __restrict__ omega, int64_t n_values, int32_t n_per_line,
                               double n2, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_values;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ref = i - i % n_per_line;
    y[i] = (float)((omega[i] - omega[ref]) / n2);
  }
}

}  // namespace ffe

// --------------------------------------------------------------- host side
using namespace ffe;

struct ffe_surrogate {
  ffe_context* ctx = nullptr;
  ffe_surrogate_meta meta;
  float* master = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* tiles = nullptr;  // the BF16 weight tiles in the MMA layout (kT2f, kT3f, kT2b, kT3b)
  int32_t* status = nullptr;       // device word: a kernel's wait gave up
  double* epoch_loss = nullptr;    // device: per-epoch loss totals of a training call
  int32_t epoch_cap = 0;
  int64_t adam_t = 0;
  // training scratch, sized for `cap` samples; per-sample arrays [layer][feature][ld]
  int64_t cap = 0, ld = 0;
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
  P.tiles = s->tiles;
  P.status = s->status;
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
  s->ld = 0;
}

// Scratch for n samples of input, target and output, and for the activations
// and gradient partials of n_act samples at once (0: inference only).
ffe_status ensure_scratch(ffe_surrogate* s, int64_t n, int64_t n_act) {
  const int64_t nb = (n_act + kRows - 1) / kRows;
  const int64_t ld = nb * kRows;  // rows of the per-sample arrays: every block's, padded
  if (n <= s->cap && ld <= s->ld) return FFE_OK;
  const int64_t cap = std::max(n, s->cap), ldn = std::max(ld, s->ld);
  free_scratch(s);
  SUR_CU(cudaMalloc(&s->x, cap * 4 * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->t, cap * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->y, cap * sizeof(float)), "cudaMalloc");
  SUR_CU(cudaMalloc(&s->dy, cap * sizeof(float)), "cudaMalloc");
  s->cap = cap;
  if (ldn > 0) {
    SUR_CU(cudaMalloc(&s->Z, 3 * ldn * kW * sizeof(float)), "cudaMalloc");
    SUR_CU(cudaMalloc(&s->dZ, 3 * ldn * kW * sizeof(float)), "cudaMalloc");
    SUR_CU(cudaMalloc(&s->H, 2 * ldn * kW * sizeof(__nv_bfloat16)), "cudaMalloc");
    SUR_CU(cudaMalloc(&s->part, (ldn / kRows) * kPartStride * sizeof(float)), "cudaMalloc");
    SUR_CU(cudaMalloc(&s->loss_part, (ldn / kRows) * sizeof(double)), "cudaMalloc");
  }
  s->ld = ldn;
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
  if ((int64_t)nb * kRows > s->ld) return set_err(s->ctx, "surrogate scratch too small"), FFE_EINTERNAL;
  mlp_fwd_kernel<<<nb, kThreads, kSmemFwd, st>>>(P, x, n, s->y, s->Z, s->H, s->ld);
  SUR_CU(cudaGetLastError(), "mlp_fwd");
  mlp_bwd_data_kernel<<<nb, kThreads, kSmemBwdData, st>>>(P, s->y, t, 1.0f / s->meta.y_scale, n, 2.0f / (float)n, s->Z,
                                                      s->dZ, s->dy, s->loss_part, s->ld);
  SUR_CU(cudaGetLastError(), "mlp_bwd_data");
  mlp_bwd_weight_kernel<<<dim3(nb, 3), kThreads, kSmemBwdW, st>>>(P, s->H, s->dZ, s->part, s->ld, x, s->Z, s->dy, n);
  SUR_CU(cudaGetLastError(), "mlp_bwd_weight");
  return FFE_OK;
}

// Waits for the surrogate's stream and reports a kernel whose wait gave up.
ffe_status check_status(ffe_surrogate* s) {
  int32_t st = 0;
  SUR_CU(cudaMemcpyAsync(&st, s->status, sizeof st, cudaMemcpyDeviceToHost, s->stream), "status");
  SUR_CU(cudaStreamSynchronize(s->stream), "sync");
  if (st != 0) {
    set_err(s->ctx, "surrogate kernel: a tensor-core wait gave up");
    return FFE_ETIMEOUT;
  }
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
  if (e == cudaSuccess) e = cudaMalloc(&s->tiles, 4 * (size_t)kTileBytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(s->status, 0, sizeof(int32_t));
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
  for (void* p : {(void*)s->master, (void*)s->m, (void*)s->v, (void*)s->tiles, (void*)s->grad, (void*)s->status,
                  (void*)s->epoch_loss})
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
  mlp_copies_kernel<<<(kW * kW + 255) / 256, 256, 0, s->stream>>>(s->master, s->tiles);
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

// Checkpoint layout (host bytes, little-endian as the machine writes it):
// header {magic "FFESUR01", parameter count, Adam step, meta}, then the FP32
// master weights, Adam first and second moments (kNParams floats each).
struct SurCheckpointHeader {
  char magic[8];
  int64_t n_params;
  int64_t adam_t;
  ffe_surrogate_meta meta;
};
constexpr char kSurMagic[8] = {'F', 'F', 'E', 'S', 'U', 'R', '0', '1'};

ffe_status ffe_surrogate_save(ffe_surrogate* s, void* buf, size_t* bytes) {
  if (!s || !bytes) return FFE_EINVAL;
  const size_t need = sizeof(SurCheckpointHeader) + 3 * (size_t)kNParams * sizeof(float);
  if (!buf) {
    *bytes = need;
    return FFE_OK;
  }
  if (*bytes < need) return set_err(s->ctx, "surrogate checkpoint: buffer of %zu bytes, %zu needed", *bytes, need),
                            FFE_EINVAL;
  SUR_CU(cudaStreamSynchronize(s->stream), "sync");
  SurCheckpointHeader h;
  std::memset(&h, 0, sizeof h);
  std::memcpy(h.magic, kSurMagic, 8);
  h.n_params = kNParams;
  h.adam_t = s->adam_t;
  h.meta = s->meta;
  unsigned char* b = static_cast<unsigned char*>(buf);
  std::memcpy(b, &h, sizeof h);
  float* f = reinterpret_cast<float*>(b + sizeof h);
  SUR_CU(cudaMemcpy(f, s->master, kNParams * sizeof(float), cudaMemcpyDeviceToHost), "save");
  SUR_CU(cudaMemcpy(f + kNParams, s->m, kNParams * sizeof(float), cudaMemcpyDeviceToHost), "save");
  SUR_CU(cudaMemcpy(f + 2 * kNParams, s->v, kNParams * sizeof(float), cudaMemcpyDeviceToHost), "save");
  *bytes = need;
  return FFE_OK;
}

ffe_status ffe_surrogate_load(ffe_surrogate* s, const void* buf, size_t bytes) {
  if (!s || !buf) return FFE_EINVAL;
  const size_t need = sizeof(SurCheckpointHeader) + 3 * (size_t)kNParams * sizeof(float);
  SurCheckpointHeader h;
  if (bytes < sizeof h) return set_err(s->ctx, "surrogate checkpoint: truncated"), FFE_EINVAL;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, kSurMagic, 8) != 0 || h.n_params != kNParams || bytes < need || h.adam_t < 0 ||
      !(h.meta.y_scale > 0.0f))
    return set_err(s->ctx, "surrogate checkpoint: not a checkpoint of this network"), FFE_EINVAL;
  const float* f = reinterpret_cast<const float*>(static_cast<const unsigned char*>(buf) + sizeof h);
  SUR_CU(cudaStreamSynchronize(s->stream), "sync");
  SUR_CU(cudaMemcpy(s->master, f, kNParams * sizeof(float), cudaMemcpyHostToDevice), "load");
  SUR_CU(cudaMemcpy(s->m, f + kNParams, kNParams * sizeof(float), cudaMemcpyHostToDevice), "load");
  SUR_CU(cudaMemcpy(s->v, f + 2 * kNParams, kNParams * sizeof(float), cudaMemcpyHostToDevice), "load");
  s->adam_t = h.adam_t;
  s->meta = h.meta;
  mlp_copies_kernel<<<(kW * kW + 255) / 256, 256, 0, s->stream>>>(s->master, s->tiles);
  SUR_CU(cudaGetLastError(), "copies");
  SUR_CU(cudaStreamSynchronize(s->stream), "sync");
  return FFE_OK;
}

ffe_status ffe_surrogate_targets(ffe_context* ctx, const double* omega, int64_t n_lines, int32_t n_per_line,
                                 int32_t N, float* y) {
  if (!ctx || !omega || !y || n_lines < 1 || n_per_line < 1 || N < 1) return FFE_EINVAL;
  const int64_t n = n_lines * (int64_t)n_per_line;
  double* d_om = nullptr;
  float* d_y = nullptr;
  cudaError_t e = cudaMalloc(&d_om, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_y, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(d_om, omega, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 65535);
    targets_kernel<<<blocks, 256>>>(d_om, n, n_per_line, (double)N * (double)N, d_y);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(y, d_y, n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(d_om);
  cudaFree(d_y);
  if (e != cudaSuccess) {
    set_err(ctx, "surrogate targets: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FFE_ENOMEM : FFE_ECUDA;
  }
  return FFE_OK;
}

ffe_status ffe_surrogate_predict(ffe_surrogate* s, const float* xraw, int64_t n, float* y, void* stream) {
  if (!s || !xraw || !y || n < 1) return FFE_EINVAL;
  (void)stream;
  ffe_status st = ensure_scratch(s, n, 0);
  if (st != FFE_OK) return st;
  cudaStream_t cs = s->stream;
  SUR_CU(cudaMemcpyAsync(s->x, xraw, n * 4 * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  const int nb = (int)((n + kRows - 1) / kRows);
  mlp_fwd_kernel<<<nb, kThreads, kSmemFwd, cs>>>(make_dev(s), s->x, n, s->y, nullptr, nullptr, 0);
  SUR_CU(cudaGetLastError(), "mlp_fwd");
  std::vector<float> yn(n);
  SUR_CU(cudaMemcpyAsync(yn.data(), s->y, n * sizeof(float), cudaMemcpyDeviceToHost, cs), "download");
  if ((st = check_status(s)) != FFE_OK) return st;
  for (int64_t i = 0; i < n; ++i) y[i] = yn[i] * s->meta.y_scale;
  return FFE_OK;
}

ffe_status ffe_surrogate_grad(ffe_surrogate* s, const float* xraw, const float* traw, int64_t n, float* grad,
                              double* loss, void* stream) {
  if (!s || !xraw || !traw || !grad || n < 1) return FFE_EINVAL;
  (void)stream;
  ffe_status st = ensure_scratch(s, n, n);
  if (st != FFE_OK) return st;
  cudaStream_t cs = s->stream;
  SUR_CU(cudaMemcpyAsync(s->x, xraw, n * 4 * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  SUR_CU(cudaMemcpyAsync(s->t, traw, n * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  if ((st = fwd_bwd(s, s->x, s->t, n, cs)) != FFE_OK) return st;
  const int nb = (int)((n + kRows - 1) / kRows);
  mlp_reduce_kernel<<<(kNParams + 255) / 256, 256, 0, cs>>>(s->part, nb, s->grad, nullptr, nullptr, nullptr, 0, 0, 0,
                                                             0, 1, 1, 0, nullptr, nullptr, nullptr);
  SUR_CU(cudaGetLastError(), "reduce");
  std::vector<double> lp(nb);
  SUR_CU(cudaMemcpyAsync(grad, s->grad, kNParams * sizeof(float), cudaMemcpyDeviceToHost, cs), "download");
  SUR_CU(cudaMemcpyAsync(lp.data(), s->loss_part, nb * sizeof(double), cudaMemcpyDeviceToHost, cs), "download");
  if ((st = check_status(s)) != FFE_OK) return st;
  if (loss) {
    double tot = 0.0;
    for (double v : lp) tot += v;
    *loss = tot / (double)n;
  }
  return FFE_OK;
}

ffe_status ffe_surrogate_train_schedule(ffe_surrogate* s, const float* xraw, const float* traw, int64_t n,
                                        int32_t epochs, int32_t batch, const float* lr_per_epoch,
                                        float* loss_per_epoch, void* stream) {
  if (!s || !xraw || !traw || !lr_per_epoch || n < 1 || epochs < 1 || epochs > kMaxEpochs || batch < 64 ||
      batch % 64 != 0)
    return s ? (set_err(s->ctx, "train: bad arguments (epochs in [1, %d], batch a multiple of 64)", kMaxEpochs),
                FFE_EINVAL)
             : FFE_EINVAL;
  for (int ep = 0; ep < epochs; ++ep)
    if (!(lr_per_epoch[ep] > 0.0f)) return set_err(s->ctx, "train: learning rates must be > 0"), FFE_EINVAL;
  (void)stream;
  ffe_status st = ensure_scratch(s, std::max<int64_t>(n, batch), batch);
  if (st != FFE_OK) return st;
  cudaStream_t cs = s->stream;
  if (epochs > s->epoch_cap) {
    if (s->epoch_loss) cudaFree(s->epoch_loss);
    s->epoch_loss = nullptr;
    s->epoch_cap = 0;
    SUR_CU(cudaMalloc(&s->epoch_loss, epochs * sizeof(double)), "cudaMalloc");
    s->epoch_cap = epochs;
  }
  SUR_CU(cudaMemsetAsync(s->epoch_loss, 0, epochs * sizeof(double), cs), "memset");
  SUR_CU(cudaMemcpyAsync(s->x, xraw, n * 4 * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  SUR_CU(cudaMemcpyAsync(s->t, traw, n * sizeof(float), cudaMemcpyHostToDevice, cs), "upload");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int64_t steps = n / batch;  // the tail that does not fill a batch is left out of the epoch
  if (steps < 1) return set_err(s->ctx, "train: fewer samples than one batch"), FFE_EINVAL;
  const int nb = (batch + kRows - 1) / kRows;
  for (int ep = 0; ep < epochs; ++ep) {
    const float lr = lr_per_epoch[ep];
    for (int64_t k = 0; k < steps; ++k) {
      const int64_t off = k * batch;
      if ((st = fwd_bwd(s, s->x + off * 4, s->t + off, batch, cs)) != FFE_OK) return st;
      ++s->adam_t;
      const float bc1 = 1.0f - powf(b1, (float)s->adam_t), bc2 = 1.0f - powf(b2, (float)s->adam_t);
      double* loss_total = loss_per_epoch ? s->epoch_loss + ep : nullptr;
      mlp_reduce_kernel<<<(kNParams + 255) / 256 + (loss_total ? 1 : 0), 256, 0, cs>>>(
          s->part, nb, nullptr, s->master, s->m, s->v, lr, b1, b2, eps, bc1, bc2, 1, s->tiles, s->loss_part,
          loss_total);
      SUR_CU(cudaGetLastError(), "adam");
    }
  }
  std::vector<double> el(epochs);
  if (loss_per_epoch)
    SUR_CU(cudaMemcpyAsync(el.data(), s->epoch_loss, epochs * sizeof(double), cudaMemcpyDeviceToHost, cs), "download");
  if ((st = check_status(s)) != FFE_OK) return st;
  if (loss_per_epoch)
    for (int ep = 0; ep < epochs; ++ep) loss_per_epoch[ep] = (float)(el[ep] / (double)(steps * batch));
  return FFE_OK;
}

ffe_status ffe_surrogate_train(ffe_surrogate* s, const float* xraw, const float* traw, int64_t n, int32_t epochs,
                               int32_t batch, float lr, float* loss_per_epoch, void* stream) {
  if (!s || epochs < 1 || epochs > kMaxEpochs || !(lr > 0.0f))
    return s ? (set_err(s->ctx, "train: bad arguments (epochs in [1, %d], lr > 0)", kMaxEpochs), FFE_EINVAL)
             : FFE_EINVAL;
  std::vector<float> lrs(epochs, lr);
  return ffe_surrogate_train_schedule(s, xraw, traw, n, epochs, batch, lrs.data(), loss_per_epoch, stream);
}

}  // extern "C"

namespace ffe {

ffe_status surrogate_infer_device(ffe_surrogate* s, const float* x, int64_t n, float* y, cudaStream_t st) {
  if (n < 1) return FFE_OK;
  const int nb = (int)((n + kRows - 1) / kRows);
  mlp_fwd_kernel<<<nb, kThreads, kSmemFwd, st>>>(make_dev(s), x, n, y, nullptr, nullptr, 0);
  SUR_CU(cudaGetLastError(), "mlp_fwd");
  return FFE_OK;
}

float surrogate_y_scale(const ffe_surrogate* s) { return s->meta.y_scale; }

}  // namespace ffe
