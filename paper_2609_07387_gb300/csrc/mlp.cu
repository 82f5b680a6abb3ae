// Troubled-cell indicator network 32 -> 64 -> 64 -> 1 on the 5th-generation
// tensor cores (tcgen05): BF16 operands staged in shared memory, FP32
// accumulators in tensor memory, one elected thread issuing the MMAs and
// committing them to an mbarrier, every wait bounded.
//
// Forward:  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3.
// Training: class-weighted binary cross-entropy, L = (1/n) sum c(y)[softplus(z) - y z];
// backward products dH1 = dH2 W2, dW2 = dH2^T H1, dW1 = dH1^T X on the tensor
// cores (all operands staged K-major, padded to M = 128), bias and last-layer
// gradients on the CUDA cores; per-CTA partial gradients are reduced in a
// fixed order (deterministic); Adam with FP32 master weights and BF16 copies.
// BF16 rounding points: x, W1, W2, w3, h1 (input of layer 2), dH2 and dH1
// (inputs of the gradient products).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mlp_internal.hpp"
#include "ucns.h"

namespace ucns {
int fail(int code, const std::string& msg);
}

namespace ucnsnet {

using bf16 = __nv_bfloat16;

constexpr int kThreads = 128;  // one thread per tile row, 4 warps = 4 TMEM lane quarters
constexpr long long kMbarCycles = 1ll << 30;  // ~0.5 s at 2 GHz: a wait gives up after this

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of a K-major BF16 tile with K columns: 8x8
// core matrices of 128 contiguous bytes, ordered K-fastest, so the leading
// (K) core-matrix stride is 128 B and the stride (8-row) one is K/8 * 128 B
__device__ __forceinline__ uint32_t kmaj(int r, int k, int K) {
  return (uint32_t)(((((r >> 3) * (K >> 3)) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t K) {
  const uint32_t lbo = 128, sbo = (K >> 3) * 128;
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// bounded wait for the phase with the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kMbarCycles) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; it++) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63u) == 63u && clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// D (TMEM, M = 128 rows) [+]= A (128 x K) * B (N x K)^T, K in steps of 16
__device__ __forceinline__ void gemm(uint32_t d, uint32_t a, uint32_t b, int K, int N, bool accumulate) {
  const uint32_t id = idesc(128, N);
  for (int k = 0; k < K; k += 16) {
    const uint32_t off = (uint32_t)(k >> 3) << 7;  // two core matrices per K step
    mma(d, sdesc(a + off, K), sdesc(b + off, K), id, (accumulate || k > 0) ? 1u : 0u);
  }
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// 8 floats -> 8 BF16 packed in 16 bytes
__device__ __forceinline__ uint4 pack8(const float* f) {
  uint4 u;
  __nv_bfloat162 p0 = __floats2bfloat162_rn(f[0], f[1]), p1 = __floats2bfloat162_rn(f[2], f[3]),
                 p2 = __floats2bfloat162_rn(f[4], f[5]), p3 = __floats2bfloat162_rn(f[6], f[7]);
  u.x = *reinterpret_cast<uint32_t*>(&p0);
  u.y = *reinterpret_cast<uint32_t*>(&p1);
  u.z = *reinterpret_cast<uint32_t*>(&p2);
  u.w = *reinterpret_cast<uint32_t*>(&p3);
  return u;
}

// ------------------------------------------------------- shared layouts
// forward
constexpr uint32_t kOffX = 0;                    // 128 x 32  bf16   8192
constexpr uint32_t kOffW1s = 8192;               //  64 x 32  bf16   4096
constexpr uint32_t kOffH1 = 12288;               // 128 x 64  bf16  16384
constexpr uint32_t kOffW2s = 28672;              //  64 x 64  bf16   8192
constexpr uint32_t kOffPar = 36864;              // b1, b2, w3 (bf16-rounded), b3: f32
constexpr uint32_t kOffBar = kOffPar + 1024;     // mbarrier, TMEM address slot
constexpr uint32_t kFwdSmem = kOffBar + 64;
// training (after the forward block); operand tiles on 1024-byte boundaries
__host__ __device__ constexpr uint32_t al1k(uint32_t x) { return (x + 1023u) & ~1023u; }
constexpr uint32_t kOffW2T = al1k(kFwdSmem);     //  64 x 64   bf16  W2^T
constexpr uint32_t kOffDH2 = kOffW2T + 8192;     // 128 x 64   bf16  dH2
constexpr uint32_t kOffA4 = kOffDH2 + 16384;     // 128 x 128  bf16  dH2^T (rows >= 64 zero)
constexpr uint32_t kOffB4 = kOffA4 + 32768;      //  64 x 128  bf16  H1^T
constexpr uint32_t kOffA5 = kOffB4 + 16384;      // 128 x 128  bf16  dH1^T (rows >= 64 zero)
constexpr uint32_t kOffB5 = kOffA5 + 32768;      //  32 x 128  bf16  X^T
constexpr uint32_t kOffRed = kOffB5 + 8192;      // 128 x 64   f32   column-sum scratch
constexpr uint32_t kOffAcc = kOffRed + 32768;    // gb1, gb2, gw3, gb3: f32
constexpr uint32_t kTrainSmem = kOffAcc + 1024;

static_assert(kOffW2T >= kFwdSmem, "training layout overlaps the forward block");
static_assert(kTrainSmem <= 227 * 1024, "shared memory budget");

struct FwdArgs {
  const bf16* __restrict__ X;  // [n][32]
  const bf16* __restrict__ W;  // W1 [64][32] then W2 [64][64]
  const float* __restrict__ theta;
  const float* __restrict__ w3r;
  float* __restrict__ z;        // [n] logits (may be null)
  uint8_t* __restrict__ flag;   // [n] z > threshold (may be null)
  bf16* __restrict__ h1;        // [n][64] first hidden layer as fed to layer 2 (may be null)
  float threshold;
  int64_t n;
  int* err;
};

struct GradArgs {
  const bf16* __restrict__ X;
  const float* __restrict__ y;  // [n] labels 0/1
  const bf16* __restrict__ W;
  const float* __restrict__ theta;
  const float* __restrict__ w3r;
  float* __restrict__ partial;  // [gridDim.x][kParams]
  int64_t n;
  float inv_n, w_pos, w_neg;
  int* err;
};

// stage the weights and the small parameter vectors into shared memory
__device__ __forceinline__ void stage_params(uint8_t* sm, const bf16* W, const float* theta, const float* w3r,
                                             bool transposed_w2) {
  const int tid = threadIdx.x;
  for (int e = tid; e < 64 * 32; e += kThreads)
    *reinterpret_cast<bf16*>(sm + kOffW1s + kmaj(e >> 5, e & 31, 32)) = W[e];
  for (int e = tid; e < 64 * 64; e += kThreads) {
    const int j = e >> 6, k = e & 63;
    *reinterpret_cast<bf16*>(sm + kOffW2s + kmaj(j, k, 64)) = W[2048 + e];
    if (transposed_w2) *reinterpret_cast<bf16*>(sm + kOffW2T + kmaj(k, j, 64)) = W[2048 + e];
  }
  float* par = reinterpret_cast<float*>(sm + kOffPar);
  for (int e = tid; e < 64; e += kThreads) {
    par[e] = theta[kOffB1 + e];
    par[64 + e] = theta[kOffB2 + e];
    par[128 + e] = w3r[e];
  }
  if (tid == 0) par[192] = theta[kOffB3];
}

// forward of one 128-row tile up to z; leaves h1 (bf16) in shared memory and
// returns per thread: z, and (for training) a1 > 0 / a2 > 0 masks and h2.
// Returns false if a wait gave up.
template <bool TRAIN>
__device__ __forceinline__ bool forward_tile(uint8_t* sm, uint32_t tmem, uint32_t lane, const bf16* X, int64_t n,
                                             int64_t row, uint64_t* bar, uint32_t& phase, float* h2out,
                                             uint64_t& m1, uint64_t& m2, float& z, bf16* h1out = nullptr) {
  const int tid = threadIdx.x;
  const uint32_t sbase = smem_u32(sm);
  const float* par = reinterpret_cast<const float*>(sm + kOffPar);
  // x row -> K-major tile (and X^T for the dW1 product)
  uint4 xr[4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
  if (row < n) {
    const uint4* src = reinterpret_cast<const uint4*>(X + row * 32);
#pragma unroll
    for (int c = 0; c < 4; c++) xr[c] = src[c];
  }
#pragma unroll
  for (int c = 0; c < 4; c++) *reinterpret_cast<uint4*>(sm + kOffX + kmaj(tid, 8 * c, 32)) = xr[c];
  if (TRAIN) {
    const bf16* xb = reinterpret_cast<const bf16*>(xr);
#pragma unroll
    for (int i = 0; i < 32; i++) *reinterpret_cast<bf16*>(sm + kOffB5 + kmaj(i, tid, 128)) = xb[i];
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  if (tid == 0) {
    fence_after();
    gemm(tmem, sbase + kOffX, sbase + kOffW1s, 32, 64, false);
    mma_commit(bar);
  }
  bool ok = mbar_wait(bar, phase);
  phase ^= 1u;
  fence_after();
  float h[64];
#pragma unroll
  for (int q = 0; q < 4; q++) tmem_ld16(tmem + lane + 16 * q, h + 16 * q);
  m1 = 0;
#pragma unroll
  for (int j = 0; j < 64; j++) {
    const float a = h[j] + par[j];
    if (a > 0.f) m1 |= (1ull << j);
    h[j] = fmaxf(a, 0.f);
  }
#pragma unroll
  for (int c = 0; c < 8; c++) {
    const uint4 hp = pack8(h + 8 * c);
    *reinterpret_cast<uint4*>(sm + kOffH1 + kmaj(tid, 8 * c, 64)) = hp;
    if (h1out && row < n) reinterpret_cast<uint4*>(h1out + row * 64)[c] = hp;
  }
  if (TRAIN) {
#pragma unroll
    for (int j = 0; j < 64; j++) *reinterpret_cast<bf16*>(sm + kOffB4 + kmaj(j, tid, 128)) = __float2bfloat16_rn(h[j]);
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  if (tid == 0) {
    fence_after();
    gemm(tmem + 64, sbase + kOffH1, sbase + kOffW2s, 64, 64, false);
    mma_commit(bar);
  }
  ok = mbar_wait(bar, phase) && ok;
  phase ^= 1u;
  fence_after();
#pragma unroll
  for (int q = 0; q < 4; q++) tmem_ld16(tmem + 64 + lane + 16 * q, h + 16 * q);
  m2 = 0;
  float acc = par[192];
#pragma unroll
  for (int j = 0; j < 64; j++) {
    const float a = h[j] + par[64 + j];
    if (a > 0.f) m2 |= (1ull << j);
    const float v = fmaxf(a, 0.f);
    if (TRAIN) h2out[j] = v;
    acc = fmaf(par[128 + j], v, acc);
  }
  z = acc;
  return ok;
}

__global__ void __launch_bounds__(kThreads, 1) k_mlp_forward(FwdArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kOffBar + 8);
  stage_params(sm, a.W, a.theta, a.w3r, false);
  if (tid == 0) mbar_init(bar);
  if (warp == 0) tmem_alloc(slot, 128);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *slot;
  const uint32_t lane = (uint32_t)(warp * 32) << 16;
  uint32_t phase = 0;
  bool ok = true;
  const int64_t ntiles = (a.n + 127) / 128;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t row = t * 128 + tid;
    uint64_t m1, m2;
    float z;
    ok = forward_tile<false>(sm, tmem, lane, a.X, a.n, row, bar, phase, nullptr, m1, m2, z, a.h1) && ok;
    if (row < a.n) {
      if (a.z) a.z[row] = z;
      if (a.flag) a.flag[row] = z > a.threshold ? 1 : 0;
    }
    fence_before();
    if (!__syncthreads_and(ok)) break;
  }
  if (!ok && tid == 0) atomicOr(a.err, 2);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// The give-up path of mbar_wait, exercised on its own: one thread waits, with
// a short limit, for a phase of a fresh mbarrier that no MMA commit and no
// thread arrives on (no MMA is issued, no TMEM is allocated), then reports
// it as the network's kernels do (bit 1 of the network's error word).
__global__ void k_mlp_wait_probe(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar);
  if (!mbar_wait(&bar, 0, limit)) atomicOr(err, 2);
}

// per-CTA partial gradients of the class-weighted BCE over its tiles
__global__ void __launch_bounds__(kThreads, 1) k_mlp_grad(GradArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sbase = smem_u32(sm);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kOffBar + 8);
  float* red = reinterpret_cast<float*>(sm + kOffRed);
  float* acc = reinterpret_cast<float*>(sm + kOffAcc);  // gb1[64] gb2[64] gw3[64] gb3
  const float* par = reinterpret_cast<const float*>(sm + kOffPar);
  stage_params(sm, a.W, a.theta, a.w3r, true);
  // the padding rows 64..127 of the transposed gradient operands stay zero
  for (uint32_t e = tid; e < 32768 / 16; e += kThreads) {
    reinterpret_cast<uint4*>(sm + kOffA4)[e] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(sm + kOffA5)[e] = make_uint4(0, 0, 0, 0);
  }
  for (int e = tid; e < 193; e += kThreads) acc[e] = 0.f;
  if (tid == 0) mbar_init(bar);
  if (warp == 0) tmem_alloc(slot, 512);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *slot;
  // TMEM columns: D1 [0,64) D2 [64,128) D3 [128,192) dW2 [192,256) dW1 [256,288)
  const uint32_t tD3 = tmem + 128, tW2 = tmem + 192, tW1 = tmem + 256;
  const uint32_t lane = (uint32_t)(warp * 32) << 16;
  uint32_t phase = 0;
  bool ok = true, first = true;
  const int64_t ntiles = (a.n + 127) / 128;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t row = t * 128 + tid;
    const bool live = row < a.n;
    uint64_t m1, m2;
    float z, h2[64];
    ok = forward_tile<true>(sm, tmem, lane, a.X, a.n, row, bar, phase, h2, m1, m2, z) && ok;
    // dL/dz = c(y) (sigmoid(z) - y) / n
    float dz = 0.f;
    if (live) {
      const float y = a.y[row];
      const float s = 1.f / (1.f + __expf(-z));
      dz = (y > 0.5f ? a.w_pos : a.w_neg) * (s - y) * a.inv_n;
    }
    // dH2 = dz w3 * [a2 > 0]  -> dH2 (K-major), dH2^T, and the FP32 rows for db2
    float d[64];
#pragma unroll
    for (int j = 0; j < 64; j++) d[j] = ((m2 >> j) & 1ull) ? dz * par[128 + j] : 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) *reinterpret_cast<uint4*>(sm + kOffDH2 + kmaj(tid, 8 * c, 64)) = pack8(d + 8 * c);
#pragma unroll
    for (int j = 0; j < 64; j++) {
      *reinterpret_cast<bf16*>(sm + kOffA4 + kmaj(j, tid, 128)) = __float2bfloat16_rn(d[j]);
      red[tid * 64 + j] = d[j];
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      gemm(tD3, sbase + kOffDH2, sbase + kOffW2T, 64, 64, false);          // dH1pre = dH2 W2
      gemm(tW2, sbase + kOffA4, sbase + kOffB4, 128, 64, !first);          // dW2 += dH2^T H1
      mma_commit(bar);
    }
    // column sums while the tensor cores run: db2, dw3, db3
    if (tid < 64) {
      float s2 = 0.f;
      for (int r = 0; r < 128; r++) s2 += red[r * 64 + tid];
      acc[64 + tid] += s2;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 64; j++) red[tid * 64 + j] = dz * h2[j];
    __syncthreads();
    if (tid < 64) {
      float s3 = 0.f;
      for (int r = 0; r < 128; r++) s3 += red[r * 64 + tid];
      acc[128 + tid] += s3;
    }
    __syncthreads();
    red[tid] = dz;
    __syncthreads();
    if (tid == 0) {
      float s4 = 0.f;
      for (int r = 0; r < 128; r++) s4 += red[r];
      acc[192] += s4;
    }
    ok = mbar_wait(bar, phase) && ok;
    phase ^= 1u;
    fence_after();
    // dH1 = dH1pre * [a1 > 0] -> dH1^T and the FP32 rows for db1
    float g[64];
#pragma unroll
    for (int q = 0; q < 4; q++) tmem_ld16(tD3 + lane + 16 * q, g + 16 * q);
    __syncthreads();  // the scalar column sum above is done with red
#pragma unroll
    for (int k = 0; k < 64; k++) {
      const float v = ((m1 >> k) & 1ull) ? g[k] : 0.f;
      *reinterpret_cast<bf16*>(sm + kOffA5 + kmaj(k, tid, 128)) = __float2bfloat16_rn(v);
      red[tid * 64 + k] = v;
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      gemm(tW1, sbase + kOffA5, sbase + kOffB5, 128, 32, !first);  // dW1 += dH1^T X
      mma_commit(bar);
    }
    if (tid < 64) {
      float s1 = 0.f;
      for (int r = 0; r < 128; r++) s1 += red[r * 64 + tid];
      acc[tid] += s1;
    }
    ok = mbar_wait(bar, phase) && ok;
    phase ^= 1u;
    fence_after();
    first = false;
    fence_before();
    if (!__syncthreads_and(ok)) break;
  }
  // write this CTA's partial gradient
  float* out = a.partial + (size_t)blockIdx.x * kParams;
  if (tid < 64) {
    float w[64];
    if (!first) {
#pragma unroll
      for (int q = 0; q < 4; q++) tmem_ld16(tW2 + lane + 16 * q, w + 16 * q);
    } else {
#pragma unroll
      for (int q = 0; q < 64; q++) w[q] = 0.f;
    }
    for (int k = 0; k < 64; k++) out[kOffW2 + tid * 64 + k] = w[k];
    if (!first) {
#pragma unroll
      for (int q = 0; q < 2; q++) tmem_ld16(tW1 + lane + 16 * q, w + 16 * q);
    }
    for (int i = 0; i < 32; i++) out[kOffW1 + tid * 32 + i] = w[i];
  } else {
    // warps 2-3 take part in the (warp-collective) loads of their own lanes, unused
    float w[64];
    if (!first) {
#pragma unroll
      for (int q = 0; q < 4; q++) tmem_ld16(tW2 + lane + 16 * q, w + 16 * q);
#pragma unroll
      for (int q = 0; q < 2; q++) tmem_ld16(tW1 + lane + 16 * q, w + 16 * q);
    }
  }
  __syncthreads();
  for (int e = tid; e < 64; e += kThreads) {
    out[kOffB1 + e] = acc[e];
    out[kOffB2 + e] = acc[64 + e];
    out[kOffW3 + e] = acc[128 + e];
  }
  if (tid == 0) out[kOffB3] = acc[192];
  if (!ok && tid == 0) atomicOr(a.err, 2);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// grad[p] = sum over CTAs in order of partial[c][p]
__global__ void k_mlp_reduce(const float* __restrict__ partial, int nctas, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float s = 0.f;
  for (int c = 0; c < nctas; c++) s += partial[(size_t)c * kParams + p];
  grad[p] = s;
}

// One training step after the per-CTA partial gradients: per parameter, the
// gradient summed over the CTAs in order (as k_mlp_reduce), the Adam update
// (beta 0.9 / 0.999, bias corrections c1, c2) and the rounded copies (as
// k_mlp_cast), in one launch
__global__ void k_mlp_step(const float* __restrict__ partial, int nctas, float* __restrict__ theta,
                           float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                           float c1, float c2, bf16* __restrict__ W, float* __restrict__ w3r) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float gp = 0.f;
  for (int c = 0; c < nctas; c++) gp += partial[(size_t)c * kParams + p];
  const float mp = b1 * m[p] + (1.f - b1) * gp;
  const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float th = theta[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
  theta[p] = th;
  if (p >= kOffW1 && p < kOffW1 + 2048) W[p - kOffW1] = __float2bfloat16_rn(th);
  if (p >= kOffW2 && p < kOffW2 + 4096) W[2048 + (p - kOffW2)] = __float2bfloat16_rn(th);
  if (p >= kOffW3 && p < kOffW3 + 64) w3r[p - kOffW3] = bf16r(th);
}

__global__ void k_mlp_cast(const float* __restrict__ theta, bf16* __restrict__ W, float* __restrict__ w3r) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < 2048) W[p] = __float2bfloat16_rn(theta[kOffW1 + p]);
  if (p < 4096) W[2048 + p] = __float2bfloat16_rn(theta[kOffW2 + p]);
  if (p < 64) w3r[p] = bf16r(theta[kOffW3 + p]);
}

}  // namespace ucnsnet

// ------------------------------------------------------------------ host
using namespace ucnsnet;

struct ucns_mlp {
  float* theta = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  bf16* W = nullptr;
  float* w3r = nullptr;
  float* partial = nullptr;
  float* grad = nullptr;
  int* err = nullptr;
  int64_t t = 0;
  int nsm = 0;
};

namespace {

#define MLP_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return ucns::fail(UCNS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int mlp_setup_attrs() {
  static bool done = false;
  if (done) return UCNS_OK;
  MLP_CUDA(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem));
  MLP_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem));
  done = true;
  return UCNS_OK;
}

// splitmix64 + Box-Muller for the He-normal initial weights
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double normal(uint64_t& s) {
  const double u1 = ((splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
  const double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

int cast(ucns_mlp* m, cudaStream_t s) {
  k_mlp_cast<<<(4096 + 255) / 256, 256, 0, s>>>(m->theta, m->W, m->w3r);
  MLP_CUDA(cudaGetLastError());
  return UCNS_OK;
}

// the per-CTA partial gradients of n rows into m->partial; returns the CTA count in *nctas
int grad_partials(ucns_mlp* m, const bf16* X, const float* y, int64_t n, float w_pos, float w_neg, int* nctas,
                  cudaStream_t s) {
  GradArgs a;
  a.X = X;
  a.y = y;
  a.W = m->W;
  a.theta = m->theta;
  a.w3r = m->w3r;
  a.partial = m->partial;
  a.n = n;
  a.inv_n = 1.f / (float)n;
  a.w_pos = w_pos;
  a.w_neg = w_neg;
  a.err = m->err;
  const int64_t ntiles = (n + 127) / 128;
  const int grid = (int)std::min<int64_t>(ntiles, m->nsm);
  k_mlp_grad<<<grid, kThreads, kTrainSmem, s>>>(a);
  MLP_CUDA(cudaGetLastError());
  *nctas = grid;
  return UCNS_OK;
}

int grad_into(ucns_mlp* m, const bf16* X, const float* y, int64_t n, float w_pos, float w_neg, float* grad,
              cudaStream_t s) {
  int nctas = 0;
  int rc = grad_partials(m, X, y, n, w_pos, w_neg, &nctas, s);
  if (rc) return rc;
  k_mlp_reduce<<<(kParams + 255) / 256, 256, 0, s>>>(m->partial, nctas, grad);
  MLP_CUDA(cudaGetLastError());
  return UCNS_OK;
}

}  // namespace

namespace ucnsnet {
// forward used by the gated residual (mesh side): logits and flags of n rows
int forward(ucns_mlp* m, const void* X, int64_t n, float* z, uint8_t* flag, float threshold, void* stream,
            void* h1) {
  int rc = mlp_setup_attrs();
  if (rc) return rc;
  FwdArgs a;
  a.h1 = reinterpret_cast<bf16*>(h1);
  a.X = reinterpret_cast<const bf16*>(X);
  a.W = m->W;
  a.theta = m->theta;
  a.w3r = m->w3r;
  a.z = z;
  a.flag = flag;
  a.threshold = threshold;
  a.n = n;
  a.err = m->err;
  const int64_t ntiles = (n + 127) / 128;
  const int grid = (int)std::min<int64_t>(ntiles, 4 * (int64_t)m->nsm);
  if (grid > 0) k_mlp_forward<<<grid, kThreads, kFwdSmem, (cudaStream_t)stream>>>(a);
  MLP_CUDA(cudaGetLastError());
  return UCNS_OK;
}
}  // namespace ucnsnet

extern "C" {

int ucns_mlp_create(uint64_t seed, ucns_mlp** out) {
  if (!out) return ucns::fail(UCNS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int rc = mlp_setup_attrs();
  if (rc) return rc;
  ucns_mlp* m = new (std::nothrow) ucns_mlp();
  if (!m) return ucns::fail(UCNS_ERR_NOMEM, "out of host memory");
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (m->nsm <= 0) m->nsm = 1;
  std::vector<float> th(kParams, 0.f);
  uint64_t st = seed;
  for (int p = 0; p < 2048; p++) th[kOffW1 + p] = (float)(normal(st) * std::sqrt(2.0 / 32));
  for (int p = 0; p < 4096; p++) th[kOffW2 + p] = (float)(normal(st) * std::sqrt(2.0 / 64));
  for (int p = 0; p < 64; p++) th[kOffW3 + p] = (float)(normal(st) * std::sqrt(1.0 / 64));
  bool okm = cudaMalloc(&m->theta, kParams * 4) == cudaSuccess && cudaMalloc(&m->m, kParams * 4) == cudaSuccess &&
             cudaMalloc(&m->v, kParams * 4) == cudaSuccess && cudaMalloc(&m->W, 6144 * 2) == cudaSuccess &&
             cudaMalloc(&m->w3r, 64 * 4) == cudaSuccess &&
             cudaMalloc(&m->partial, (size_t)m->nsm * kParams * 4) == cudaSuccess &&
             cudaMalloc(&m->grad, kParams * 4) == cudaSuccess && cudaMalloc(&m->err, sizeof(int)) == cudaSuccess;
  if (!okm) {
    ucns_mlp_destroy(m);
    return ucns::fail(UCNS_ERR_NOMEM, "cudaMalloc failed for the indicator network");
  }
  if (cudaMemcpy(m->theta, th.data(), kParams * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->m, 0, kParams * 4) != cudaSuccess || cudaMemset(m->v, 0, kParams * 4) != cudaSuccess ||
      cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess || cast(m, nullptr) != UCNS_OK ||
      cudaDeviceSynchronize() != cudaSuccess) {
    ucns_mlp_destroy(m);
    return ucns::fail(UCNS_ERR_CUDA, "initialising the indicator network failed");
  }
  *out = m;
  return UCNS_OK;
}

void ucns_mlp_destroy(ucns_mlp* m) {
  if (!m) return;
  void* p[] = {m->theta, m->m, m->v, m->W, m->w3r, m->partial, m->grad, m->err};
  for (void* q : p)
    if (q) cudaFree(q);
  delete m;
}

int ucns_mlp_get_params(const ucns_mlp* m, float* theta) {
  if (!m || !theta) return ucns::fail(UCNS_ERR_INVALID_ARG, "NULL argument");
  MLP_CUDA(cudaMemcpy(theta, m->theta, kParams * 4, cudaMemcpyDeviceToHost));
  return UCNS_OK;
}

int ucns_mlp_set_params(ucns_mlp* m, const float* theta) {
  if (!m || !theta) return ucns::fail(UCNS_ERR_INVALID_ARG, "NULL argument");
  MLP_CUDA(cudaMemcpy(m->theta, theta, kParams * 4, cudaMemcpyHostToDevice));
  MLP_CUDA(cudaMemset(m->m, 0, kParams * 4));
  MLP_CUDA(cudaMemset(m->v, 0, kParams * 4));
  m->t = 0;
  int rc = cast(m, nullptr);
  if (rc) return rc;
  MLP_CUDA(cudaDeviceSynchronize());
  return UCNS_OK;
}

int ucns_mlp_forward(ucns_mlp* m, const void* X, int64_t n, float* z, void* stream) {
  if (!m || !X || !z || n < 0) return ucns::fail(UCNS_ERR_INVALID_ARG, "bad argument");
  if (((uintptr_t)X & 15) != 0) return ucns::fail(UCNS_ERR_INVALID_ARG, "X must be 16-byte aligned");
  return ucnsnet::forward(m, X, n, z, nullptr, 0.f, stream);
}

int ucns_mlp_hidden(ucns_mlp* m, const void* X, int64_t n, void* h1, float* z, void* stream) {
  if (!m || !X || !h1 || !z || n < 0) return ucns::fail(UCNS_ERR_INVALID_ARG, "bad argument");
  if (((uintptr_t)X & 15) != 0 || ((uintptr_t)h1 & 15) != 0)
    return ucns::fail(UCNS_ERR_INVALID_ARG, "X and h1 must be 16-byte aligned");
  return ucnsnet::forward(m, X, n, z, nullptr, 0.f, stream, h1);
}

int ucns_mlp_grad(ucns_mlp* m, const void* X, const float* y, int64_t n, float w_pos, float w_neg, float* grad,
                  void* stream) {
  if (!m || !X || !y || !grad || n <= 0) return ucns::fail(UCNS_ERR_INVALID_ARG, "bad argument");
  if (((uintptr_t)X & 15) != 0) return ucns::fail(UCNS_ERR_INVALID_ARG, "X must be 16-byte aligned");
  return grad_into(m, reinterpret_cast<const bf16*>(X), y, n, w_pos, w_neg, grad, (cudaStream_t)stream);
}

int ucns_mlp_train(ucns_mlp* m, const void* X, const float* y, int64_t n, int64_t batch, float lr, float w_pos,
                   float w_neg, void* stream) {
  if (!m || !X || !y || n <= 0 || batch <= 0 || batch % 8 != 0 || !(lr > 0.f))
    return ucns::fail(UCNS_ERR_INVALID_ARG, "bad argument (batch must be a positive multiple of 8)");
  if (((uintptr_t)X & 15) != 0) return ucns::fail(UCNS_ERR_INVALID_ARG, "X must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const bf16* Xb = reinterpret_cast<const bf16*>(X);
  for (int64_t b0 = 0; b0 < n; b0 += batch) {
    const int64_t nb = std::min(batch, n - b0);
    int nctas = 0;
    int rc = grad_partials(m, Xb + b0 * 32, y + b0, nb, w_pos, w_neg, &nctas, s);
    if (rc) return rc;
    m->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)m->t)), c2 = (float)(1.0 - std::pow(0.999, (double)m->t));
    // the summed gradient, Adam and the BF16 copies in one launch
    k_mlp_step<<<(kParams + 255) / 256, 256, 0, s>>>(m->partial, nctas, m->theta, m->m, m->v, lr, b1, b2, 1e-8f,
                                                      c1, c2, m->W, m->w3r);
  }
  MLP_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int ucns_mlp_probe_bounded_wait(ucns_mlp* m, void* stream) {
  if (!m) return ucns::fail(UCNS_ERR_INVALID_ARG, "NULL argument");
  k_mlp_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(m->err, 1ll << 21);
  MLP_CUDA(cudaGetLastError());
  return ucns_mlp_check(m, stream);
}

int ucns_mlp_check(ucns_mlp* m, void* stream) {
  if (!m) return ucns::fail(UCNS_ERR_INVALID_ARG, "NULL argument");
  int h = 0;
  MLP_CUDA(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  MLP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (h) {
    MLP_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    return ucns::fail(UCNS_ERR_TIMEOUT, "a tensor-core wait gave up in the indicator network");
  }
  return UCNS_OK;
}

}  // extern "C"
