// Features of the learned troubled-cell indicator, one thread per cell:
// density and pressure jumps over the central stencil, normalised smoothness
// indicators of the optimal central polynomial p_opt (Eq. 4, Eq. 6 reading),
// and three scale-free flow measures from p_opt's gradient at the centroid.
#pragma once

#include <cuda_bf16.h>

#include "kernels_mixed.cuh"

namespace ucns {

struct FeatArgs {
  const double* __restrict__ U;    // [5][N] (FP64 form)
  const float* __restrict__ Uhl;   // [N][5][2] float pairs of U (mixed form)
  const int32_t* __restrict__ sc;  // [18][N] (FP64 form) or pair-blocked (mixed form)
  const void* __restrict__ Pc;     // [9][18][N] double (FP64 form) or pair-blocked float (mixed form)
  const double* __restrict__ mom;    // [6][N] (FP64 form)
  const double* __restrict__ inv_h;  // [N] (FP64 form)
  const float* __restrict__ cell;    // blocked [tiles][kCellRows][kTC] (mixed form)
  __nv_bfloat16* __restrict__ X;  // [N][32]
  float* __restrict__ Xf;         // [N][32] or null
  int N;
  float gam;
};

// features 24-31 from the central coefficients ao[v][k] (xi units) of the
// five variables, then the BF16 row (and the FP32 row when asked for)
__device__ __forceinline__ void features_finish(float F[32], const float (&ao)[5][9], const float S[6], float rf,
                                                float c, const float u[3], float ih, const FeatArgs& a, int i) {
  const float sc5[5] = {rf, rf * c, rf * c, rf * c, rf * c * c};
#pragma unroll
  for (int v = 0; v < 5; v++) {
    const float* o = ao[v];
    auto quad = [&](float x0, float x1, float x2) {
      return S[0] * x0 * x0 + S[1] * x1 * x1 + S[2] * x2 * x2 + 2.f * (S[3] * x0 * x1 + S[4] * x0 * x2 + S[5] * x1 * x2);
    };
    const float SI = o[0] * o[0] + o[1] * o[1] + o[2] * o[2] + quad(2.f * o[3], o[6], o[7]) +
                     quad(o[6], 2.f * o[4], o[8]) + quad(o[7], o[8], 2.f * o[5]) +
                     4.f * (o[3] * o[3] + o[4] * o[4] + o[5] * o[5]) + o[6] * o[6] + o[7] * o[7] + o[8] * o[8];
    const float q = 0.1f * sc5[v];
    F[24 + v] = SI / (SI + q * q);
  }
  // p_opt gradient at the centroid: linear coefficients / h
  const float h = 1.f / ih;
  float gu[3][3];
#pragma unroll
  for (int q = 0; q < 3; q++)
#pragma unroll
    for (int j = 0; j < 3; j++) gu[q][j] = (ao[1 + q][j] - u[q] * ao[0][j]) * ih / rf;
  const float wx = gu[2][1] - gu[1][2], wy = gu[0][2] - gu[2][0], wz = gu[1][0] - gu[0][1];
  F[29] = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / c;
  F[30] = h * fabsf(gu[0][0] + gu[1][1] + gu[2][2]) / c;
  F[31] = h * sqrtf(wx * wx + wy * wy + wz * wz) / c;
  uint4* dst = reinterpret_cast<uint4*>(a.X + (size_t)i * 32);
#pragma unroll
  for (int q = 0; q < 4; q++) {
    uint4 w;
    __nv_bfloat162 b0 = __floats2bfloat162_rn(F[8 * q + 0], F[8 * q + 1]);
    __nv_bfloat162 b1 = __floats2bfloat162_rn(F[8 * q + 2], F[8 * q + 3]);
    __nv_bfloat162 b2 = __floats2bfloat162_rn(F[8 * q + 4], F[8 * q + 5]);
    __nv_bfloat162 b3 = __floats2bfloat162_rn(F[8 * q + 6], F[8 * q + 7]);
    w.x = *reinterpret_cast<uint32_t*>(&b0);
    w.y = *reinterpret_cast<uint32_t*>(&b1);
    w.z = *reinterpret_cast<uint32_t*>(&b2);
    w.w = *reinterpret_cast<uint32_t*>(&b3);
    dst[q] = w;
  }
  if (a.Xf) {
#pragma unroll
    for (int q = 0; q < 32; q++) a.Xf[(size_t)i * 32 + q] = F[q];
  }
}

// FP64 form: differences of the FP64 state, FP64 pseudo-inverse rows
__global__ void __launch_bounds__(128) k_features(FeatArgs a) {
  constexpr int K = 9, MC = 18;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const size_t N = a.N;
  const double* __restrict__ Pc = reinterpret_cast<const double*>(a.Pc);
  const double g = a.gam;
  double Ui[5];
#pragma unroll
  for (int v = 0; v < 5; v++) Ui[v] = a.U[v * N + i];
  const double r = Ui[0], ir = 1.0 / r;
  const double m2 = Ui[1] * Ui[1] + Ui[2] * Ui[2] + Ui[3] * Ui[3];
  const double p = (g - 1.0) * (Ui[4] - 0.5 * m2 * ir);
  const float c = (float)sqrt(g * p * ir);
  float F[32];
  float ao[5][K];
#pragma unroll
  for (int v = 0; v < 5; v++)
#pragma unroll
    for (int k = 0; k < K; k++) ao[v][k] = 0.f;
#pragma unroll 2
  for (int m = 0; m < MC; m++) {
    const int j = __ldg(&a.sc[(size_t)m * N + i]);
    double Uj[5];
    float d[5];
#pragma unroll
    for (int v = 0; v < 5; v++) {
      Uj[v] = a.U[v * N + j];
      d[v] = (float)(Uj[v] - Ui[v]);
    }
    F[m] = (float)((Uj[0] - r) * ir);
    if (m < 6) {
      const double pj = (g - 1.0) * (Uj[4] - 0.5 * (Uj[1] * Uj[1] + Uj[2] * Uj[2] + Uj[3] * Uj[3]) / Uj[0]);
      F[18 + m] = (float)((pj - p) / p);
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      const float P = (float)Pc[((size_t)k * MC + m) * N + i];
#pragma unroll
      for (int v = 0; v < 5; v++) ao[v][k] = fmaf(P, d[v], ao[v][k]);
    }
  }
  float S[6];
#pragma unroll
  for (int q = 0; q < 6; q++) S[q] = (float)a.mom[q * N + i];
  const float u[3] = {(float)(Ui[1] * ir), (float)(Ui[2] * ir), (float)(Ui[3] * ir)};
  features_finish(F, ao, S, (float)r, c, u, (float)a.inv_h[i], a, i);
}

// mixed form: stencil differences from the float pair of the state (exact
// leading-part subtraction, as in the reconstruction), FP32 arithmetic,
// blocked FP32 pseudo-inverse rows
__global__ void __launch_bounds__(128, 4) k_features_mx(FeatArgs a) {
  constexpr int K = 9, MC = 18;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const float* __restrict__ Pc = reinterpret_cast<const float*>(a.Pc);
  const float2* __restrict__ hl2 = reinterpret_cast<const float2*>(a.Uhl);  // a row: (hi, lo) of 5 variables
  const float g = a.gam;
  float hi[5], lo[5];
  {
    float t[10];
#pragma unroll
    for (int q = 0; q < 5; q++) {
      const float2 w = __ldg(&hl2[(size_t)i * 5 + q]);
      t[2 * q] = w.x;
      t[2 * q + 1] = w.y;
    }
#pragma unroll
    for (int v = 0; v < 5; v++) {
      hi[v] = t[2 * v];
      lo[v] = t[2 * v + 1];
    }
  }
  const float r = hi[0] + lo[0], ir = 1.f / r;
  const float mx = hi[1] + lo[1], my = hi[2] + lo[2], mz = hi[3] + lo[3];
  const float p = (g - 1.f) * ((hi[4] + lo[4]) - 0.5f * (mx * mx + my * my + mz * mz) * ir);
  const float ip = 1.f / p;
  const float c = sqrtf(g * p * ir);
  float F[32];
  float ao[5][K];
#pragma unroll
  for (int v = 0; v < 5; v++)
#pragma unroll
    for (int k = 0; k < K; k++) ao[v][k] = 0.f;
#pragma unroll
  for (int m = 0; m < MC; m++) {
    const int j = __ldg(&a.sc[blk2(m, MC, i)]);
    float t[10];
#pragma unroll
    for (int q = 0; q < 5; q++) {
      const float2 w = __ldg(&hl2[(size_t)j * 5 + q]);
      t[2 * q] = w.x;
      t[2 * q + 1] = w.y;
    }
    float d[5];
#pragma unroll
    for (int v = 0; v < 5; v++) d[v] = (t[2 * v] - hi[v]) + (t[2 * v + 1] - lo[v]);
    F[m] = d[0] * ir;
    if (m < 6) {
      const float rj = t[0] + t[1], mjx = t[2] + t[3], mjy = t[4] + t[5], mjz = t[6] + t[7];
      const float pj = (g - 1.f) * ((t[8] + t[9]) - 0.5f * (mjx * mjx + mjy * mjy + mjz * mjz) / rj);
      F[18 + m] = (pj - p) * ip;
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      const float P = __ldg(&Pc[blk2(k * MC + m, K * MC, i)]);
#pragma unroll
      for (int v = 0; v < 5; v++) ao[v][k] = fmaf(P, d[v], ao[v][k]);
    }
  }
  float S[6];
#pragma unroll
  for (int q = 0; q < 6; q++) S[q] = __ldg(&a.cell[blk(q, kCellRows, i)]);
  const float u[3] = {mx * ir, my * ir, mz * ir};
  features_finish(F, ao, S, r, c, u, __ldg(&a.cell[blk(6, kCellRows, i)]), a, i);
}

__global__ void k_count_flags(const uint8_t* __restrict__ flag, int N, unsigned long long* __restrict__ count) {
  __shared__ unsigned int sm[256];
  unsigned int c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) c += flag[i];
  sm[threadIdx.x] = c;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(count, (unsigned long long)sm[0]);
}

// per-block sums, for two residuals R1 (gated) and R2 (full) of the state U,
// of the cell kinetic-energy rates r = V (u . R_m - |u|^2 R_rho / 2): [sum r1,
// sum r2, sum V, sum |r1 - r2|, sum |r2|] at part[8 b + q] (the fourth is the
// local difference, which cannot cancel between cells)
constexpr int kKeRateSums = 5, kRedStride = 8;
__global__ void __launch_bounds__(256) k_ke_rate_partial(const double* __restrict__ U, const double* __restrict__ R1,
                                                         const double* __restrict__ R2, const double* __restrict__ vol,
                                                         int N, double* __restrict__ part) {
  __shared__ double sm[kKeRateSums][256];
  double acc[kKeRateSums] = {0, 0, 0, 0, 0};
  const size_t n = N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double ir = 1.0 / U[i];
    const double u0 = U[n + i] * ir, u1 = U[2 * n + i] * ir, u2 = U[3 * n + i] * ir;
    const double q = 0.5 * (u0 * u0 + u1 * u1 + u2 * u2);
    const double V = vol[i];
    const double r1 = V * (u0 * R1[n + i] + u1 * R1[2 * n + i] + u2 * R1[3 * n + i] - q * R1[i]);
    const double r2 = V * (u0 * R2[n + i] + u1 * R2[2 * n + i] + u2 * R2[3 * n + i] - q * R2[i]);
    acc[0] += r1;
    acc[1] += r2;
    acc[2] += V;
    acc[3] += fabs(r1 - r2);
    acc[4] += fabs(r2);
  }
#pragma unroll
  for (int q = 0; q < kKeRateSums; q++) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int q = 0; q < kKeRateSums; q++) sm[q][threadIdx.x] += sm[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < kKeRateSums; q++) part[(size_t)blockIdx.x * kRedStride + q] = sm[q][0];
}

// out[q] = sum over blocks, in block order, of part[stride b + q], q < nq
__global__ void k_sum_partials(const double* __restrict__ part, int nb, int stride, int nq, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q < nq; q++) {
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += part[(size_t)b * stride + q];
    out[q] = s;
  }
}

}  // namespace ucns
