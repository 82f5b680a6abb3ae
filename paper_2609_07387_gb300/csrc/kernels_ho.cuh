// P3 and P4 reconstruction and face kernels (FP64), hexahedra.
//
//   k_recon_ho  thread = (cell, variable): central least-squares contraction
//               (K = 19 or 34 modes over 2K members, Eq. 4); with CWENOZ the
//               six directional candidates (linear at P3, quadratic over 18
//               members at P4, Sec. 2.2), the smoothness indicators as the
//               quadratic forms a^T M a of each cell's precomputed matrix M
//               (Eq. 6 reading), the nonlinear weights and the combination.
//               The directional contractions run twice (once for the
//               indicators, once for the combination) rather than holding all
//               six candidates in registers.
//   k_face_ho   ORDER^2 Gauss points per face on ORDER^2 lanes (9 at P3, 16
//               at P4; 32 / ORDER^2 faces per warp); values and gradients of
//               the monomial-form polynomials, HLLC, penalised viscous flux
//               (Eq. 7), and the face total summed by the group's first lane
//               over its lanes in point order (deterministic).
//   k_recon_ho_mx the same in the mixed form, tile by tile (64 cells): the
//               stencil ids and FP32 pseudo-inverses stream through shared
//               memory in bulk-copied chunks, thread = (cell, variable).
//   (the mixed face kernel of every order is k_face_mx, kernels_mixed.cuh)
#pragma once

#include "basis.hpp"
#include "kernels.cuh"
#include "kernels_mixed.cuh"

namespace ucns {

template <int ORDER>
struct HO {
  static constexpr int K = basis_count(ORDER);
  static constexpr int MC = 2 * K;
  static constexpr int KD = ORDER == 4 ? 9 : 3;  // modes of a directional candidate
  static constexpr int MD = 2 * KD;
  static constexpr int NQ = ORDER * ORDER;
};

struct ReconArgsHO {
  const double* __restrict__ U;     // [5][N]
  const int32_t* __restrict__ sc;   // [MC][N]
  const double* __restrict__ Pc;    // [K][MC][N]
  const int32_t* __restrict__ sd;   // [6][MD][N]
  const double* __restrict__ Pd;    // [6][KD][MD][N]
  const double* __restrict__ Msi;   // [K(K+1)/2][N]: smoothness-indicator matrix, upper triangle by rows
  const double* __restrict__ psib;  // [K-3][N]: cell means of the basis monomials of degree >= 2
  const double* __restrict__ inv_h; // [N]
  double* __restrict__ coef;        // [K+1][N][5] physical-unit monomial coefficients
  int N;
  double lam0, lams, eps;
};

// a^T M a over the first KK modes (M: K x K symmetric, upper triangle stored
// by rows: entry (k, l >= k) at q = k K - k (k - 1) / 2 + l - k)
template <int K, int KK>
__device__ __forceinline__ double si_form(const double* __restrict__ M, size_t N, int i, const double (&a)[KK]) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < KK; k++) {
    double t = 0.0;
#pragma unroll
    for (int l = k + 1; l < KK; l++) t = fma(__ldg(&M[(size_t)(k * K - k * (k - 1) / 2 + l - k) * N + i]), a[l], t);
    const double mkk = __ldg(&M[(size_t)(k * K - k * (k - 1) / 2) * N + i]);
    s = fma(a[k], fma(2.0, t, mkk * a[k]), s);
  }
  return s;
}

// directional candidate s of variable v: b = P_s (U_m - U_i) over its members
template <int ORDER>
__device__ __forceinline__ void dir_coeffs(const ReconArgsHO& a, const double* __restrict__ Uv, double ui, int i, int s,
                                           double (&b)[HO<ORDER>::KD]) {
  using H = HO<ORDER>;
  const size_t N = a.N;
#pragma unroll
  for (int k = 0; k < H::KD; k++) b[k] = 0.0;
#pragma unroll 2
  for (int r = 0; r < H::MD; r++) {
    const int j = __ldg(&a.sd[((size_t)s * H::MD + r) * N + i]);
    const double d = Uv[j] - ui;
#pragma unroll
    for (int k = 0; k < H::KD; k++) b[k] = fma(__ldg(&a.Pd[(((size_t)s * H::KD + k) * H::MD + r) * N + i]), d, b[k]);
  }
}

template <int ORDER, bool WENO>
__global__ void __launch_bounds__(128) k_recon_ho(ReconArgsHO a) {
  using H = HO<ORDER>;
  constexpr int K = H::K, MC = H::MC, KD = H::KD, ND = 6;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = tid / 5, v = tid - 5 * (tid / 5);
  if (i >= a.N) return;
  const size_t N = a.N;
  const double* __restrict__ Uv = a.U + (size_t)v * N;
  const double ui = Uv[i];
  double ao[K];
#pragma unroll
  for (int k = 0; k < K; k++) ao[k] = 0.0;
#pragma unroll 2
  for (int m = 0; m < MC; m++) {
    const int j = __ldg(&a.sc[(size_t)m * N + i]);
    const double d = Uv[j] - ui;
#pragma unroll
    for (int k = 0; k < K; k++) ao[k] = fma(__ldg(&a.Pc[((size_t)k * MC + m) * N + i]), d, ao[k]);
  }
  double c[K];
  if constexpr (!WENO) {
#pragma unroll
    for (int k = 0; k < K; k++) c[k] = ao[k];
  } else {
    const double SI0 = si_form<K, K>(a.Msi, N, i, ao);
    double SI[ND];
    double tau = 0.0;
#pragma unroll 1
    for (int s = 0; s < ND; s++) {
      double b[KD];
      dir_coeffs<ORDER>(a, Uv, ui, i, s, b);
      SI[s] = si_form<K, KD>(a.Msi, N, i, b);
      tau += fabs(SI0 - SI[s]);
    }
    tau *= (1.0 / ND);
    // omega~_s = lambda_s (1 + tau / (eps + SI_s)), normalised
    const double w0 = a.lam0 * (1.0 + tau / (a.eps + SI0));
    double ws[ND];
    double wsum = w0;
#pragma unroll
    for (int s = 0; s < ND; s++) {
      ws[s] = a.lams * (1.0 + tau / (a.eps + SI[s]));
      wsum += ws[s];
    }
    const double iws = 1.0 / wsum;
    // p = omega_0 p_1 + sum_s omega_s p_s with p_1 = (p_opt - sum lambda_s p_s)/lambda_0
    const double r0 = (w0 * iws) / a.lam0;
#pragma unroll
    for (int k = 0; k < K; k++) c[k] = r0 * ao[k];
#pragma unroll 1
    for (int s = 0; s < ND; s++) {
      double b[KD];
      dir_coeffs<ORDER>(a, Uv, ui, i, s, b);
      const double e = ws[s] * iws - r0 * a.lams;
#pragma unroll
      for (int k = 0; k < KD; k++) c[k] = fma(e, b[k], c[k]);
    }
  }
  // monomial form in physical units: p = c0 + sum_k (c_k / h^deg_k) (x - x_i)^e_k,
  // c0 = U_i - sum_{deg >= 2} c_k mean(psi_k)
  double c0 = ui;
#pragma unroll
  for (int k = 3; k < K; k++) c0 = fma(-c[k], __ldg(&a.psib[(size_t)(k - 3) * N + i]), c0);
  const double ih = __ldg(&a.inv_h[i]);
  double ihp[ORDER + 1];
  ihp[0] = 1.0;
#pragma unroll
  for (int e = 1; e <= ORDER; e++) ihp[e] = ihp[e - 1] * ih;
  double* out = a.coef + (size_t)i * 5 + v;
  const size_t st = N * 5;
  out[0] = c0;
#pragma unroll
  for (int k = 0; k < K; k++) out[(k + 1) * st] = c[k] * ihp[basis_degree(k)];
}

// value at the physical offset (x, y, z) from the centroid into U and the
// gradient written (ACC = false) or added (ACC = true) into g
template <int ORDER, bool ACC>
__device__ __forceinline__ void eval_side_ho(const double* __restrict__ coef, int N, int cell, double x, double y,
                                             double z, double U[5], double g[5][3]) {
  constexpr int K = basis_count(ORDER);
  const size_t st = (size_t)N * 5;
  const double* p = coef + (size_t)cell * 5;
  double px[ORDER + 1], py[ORDER + 1], pz[ORDER + 1];
  px[0] = py[0] = pz[0] = 1.0;
#pragma unroll
  for (int e = 1; e <= ORDER; e++) {
    px[e] = px[e - 1] * x;
    py[e] = py[e - 1] * y;
    pz[e] = pz[e - 1] * z;
  }
  double gx[5], gy[5], gz[5];
#pragma unroll
  for (int v = 0; v < 5; v++) {
    U[v] = p[v];
    gx[v] = gy[v] = gz[v] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < K; k++) {
    const int ex = basis_exp(k, 0), ey = basis_exp(k, 1), ez = basis_exp(k, 2);
    const double mv = px[ex] * py[ey] * pz[ez];
    const double mx = ex ? ex * px[ex > 0 ? ex - 1 : 0] * py[ey] * pz[ez] : 0.0;
    const double my = ey ? ey * px[ex] * py[ey > 0 ? ey - 1 : 0] * pz[ez] : 0.0;
    const double mz = ez ? ez * px[ex] * py[ey] * pz[ez > 0 ? ez - 1 : 0] : 0.0;
#pragma unroll
    for (int v = 0; v < 5; v++) {
      const double c = p[(k + 1) * st + v];
      U[v] = fma(c, mv, U[v]);
      if (ex) gx[v] = fma(c, mx, gx[v]);
      if (ey) gy[v] = fma(c, my, gy[v]);
      if (ez) gz[v] = fma(c, mz, gz[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; v++) {
    if (ACC) {
      g[v][0] += gx[v];
      g[v][1] += gy[v];
      g[v][2] += gz[v];
    } else {
      g[v][0] = gx[v];
      g[v][1] = gy[v];
      g[v][2] = gz[v];
    }
  }
}

template <int ORDER, bool VISC>
__global__ void __launch_bounds__(128) k_face_ho(FaceArgs a) {
  constexpr int NQ = ORDER * ORDER, FPW = 32 / NQ;  // faces per warp
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int grp = lane / NQ, q = lane - NQ * (lane / NQ);
  const bool in_group = grp < FPW;
  const int f = gw * FPW + (in_group ? grp : 0);
  const bool live = in_group && f < a.F;
  const int fc = live ? f : a.F - 1, qc = in_group ? q : 0;
  const size_t F = a.F;
  const double* __restrict__ fq = a.fq + (size_t)qc * 10 * F + fc;
  const double xl = fq[0], yl = fq[F], zl = fq[2 * F];
  const double xr = fq[3 * F], yr = fq[4 * F], zr = fq[5 * F];
  const double n[3] = {fq[6 * F], fq[7 * F], fq[8 * F]};
  const double area = fq[9 * F];
  const int o = a.fo[fc], nb = a.fn[fc];
  double UL[5], UR[5], gs[5][3];  // gs = grad U_L + grad U_R
  eval_side_ho<ORDER, false>(a.coef, a.N, o, xl, yl, zl, UL, gs);
  eval_side_ho<ORDER, true>(a.coef, a.N, nb, xr, yr, zr, UR, gs);
  double Fc[5];
  hllc_flux(UL, UR, n, a.c, Fc);
  double flux[5];
  if (VISC) {
    // as in k_face: twice the face state and the penalised face gradient
    const double pen2 = 2.0 * a.fpen[fc];
    double Uf2[5], gf2[5][3];
#pragma unroll
    for (int v = 0; v < 5; v++) {
      const double jump2 = pen2 * (UR[v] - UL[v]);
      Uf2[v] = UL[v] + UR[v];
#pragma unroll
      for (int j = 0; j < 3; j++) gf2[v][j] = fma(jump2, n[j], gs[v][j]);
    }
    double Fv[5];
    viscous_flux(Uf2, gf2, n, a.c, Fv);
#pragma unroll
    for (int v = 0; v < 5; v++) flux[v] = (Fc[v] - Fv[v]) * area;
  } else {
#pragma unroll
    for (int v = 0; v < 5; v++) flux[v] = Fc[v] * area;
  }
  // the group's first lane sums its NQ points in point order (every lane takes
  // part in the shuffles; lanes outside a group read group 0 and store nothing)
  const int base = (in_group ? grp : 0) * NQ;
  double tot[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int t = 0; t < NQ; t++)
#pragma unroll
    for (int v = 0; v < 5; v++) tot[v] += __shfl_sync(0xffffffffu, flux[v], base + t);
  if (live && q == 0) {
#pragma unroll
    for (int v = 0; v < 5; v++) a.G[(size_t)v * F + f] = tot[v];
  }
}



// ------------------------------------------------------- mixed P3 / P4
// The mixed form at P3 / P4 (the arithmetic split of the mixed form at P2):
// stencil differences from the float pairs of the FP64 state, FP32
// pseudo-inverses, contractions, smoothness forms and weights; the constant
// term written relative to the reference state U_ref; coefficients FP32
// [K+1][N][5]; FP32 HLLC and viscous flux on reference-relative states, FP32
// face totals (k_rk<s, nfc, float> sums them as float pairs into FP64).
struct ReconArgsHOMx {
  const float* __restrict__ Uhl;    // [N][5][2] float pairs (hi, lo) of the state
  const float* __restrict__ tiles;  // per 64-cell tile its stencil chunks (HOTile)
  const float* __restrict__ Msi;    // [K(K+1)/2][N]
  const float* __restrict__ psib;   // [K-3][N]
  const float* __restrict__ inv_h;  // [N]
  float* __restrict__ coef;         // [N][cs] rows, entries cidx(v, k, K + 1): k = 0 relative to U_ref,
                                    // then the physical-unit coefficients
  int* err;                         // bit 1: a copy wait gave up
  int N, cs;
  float lam0, lams, eps;
  float eref_hi, eref_lo;  // E_ref = p_ref/(gamma-1) as a float pair
};

// The P3/P4 mixed reconstruction's data, tile by tile (64 cells): the central
// stencil in NCC chunks of MCH members, then each of the six directional
// stencils in NDC chunks of MDH members.  A chunk is [members][64] stencil ids
// (int32) followed by its pseudo-inverse entries as pairs of consecutive
// members, [modes][members / 2][64][2]; every chunk is one bulk copy.  Cells
// past N in the last tile have ids 0 and zero entries.
template <int ORDER>
struct HOTile {
  using H = HO<ORDER>;
  static constexpr int K = H::K, MC = H::MC, KD = H::KD, MD = H::MD;
  static constexpr int TC = 64;
  static constexpr int MCH = ORDER == 4 ? 4 : 2, MDH = 6;
  static constexpr int NCC = MC / MCH, NDC = MD / MDH;
  static constexpr int CCS = MCH * TC + K * MCH * TC;  // floats per central chunk
  static constexpr int DCS = MDH * TC + KD * MDH * TC;  // floats per directional chunk
  static constexpr int CENTRAL = NCC * CCS;
  static constexpr int STAGE = CCS > DCS ? CCS : DCS;
  // with CWENOZ the smoothness matrices follow the central chunks: [K(K+1)/2][64]
  // entries in chunks of MSR rows, then the directional chunks
  static constexpr int NQS = K * (K + 1) / 2, MSR = STAGE / TC, NMC = (NQS + MSR - 1) / MSR;
  static constexpr int SMAT = NQS * TC;
  UCNS_HD static constexpr int tile_floats(bool weno) { return CENTRAL + (weno ? SMAT + 6 * NDC * DCS : 0); }
  static constexpr int S = ORDER == 4 ? 3 : 4;  // stages of the copy ring (6 at P4 measured slower)
  static constexpr int THREADS = 5 * TC + 32;   // (cell, variable) threads and one copying warp
  static constexpr size_t smem() { return (size_t)S * STAGE * 4 + (size_t)2 * S * 8; }
  static_assert(MC % MCH == 0 && MD % MDH == 0 && MCH % 2 == 0 && MDH % 2 == 0, "whole member pairs");
  static_assert(CCS % 4 == 0 && DCS % 4 == 0, "16-byte chunks");
};

// a^T M a over the first KK modes of one variable (M as in si_form), FP32
template <int K, int KK>
__device__ __forceinline__ float si_form_f(const float* __restrict__ M, size_t N, int i, const float (&a)[KK]) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < KK; k++) {
    float t = 0.f;
#pragma unroll
    for (int l = k + 1; l < KK; l++) t = fmaf(__ldg(&M[(size_t)(k * K - k * (k - 1) / 2 + l - k) * N + i]), a[l], t);
    const float mkk = __ldg(&M[(size_t)(k * K - k * (k - 1) / 2) * N + i]);
    s = fmaf(a[k], fmaf(2.f, t, mkk * a[k]), s);
  }
  return s;
}

// U_j - U_i of variable v from the float pairs (the leading parts subtract exactly)
__device__ __forceinline__ float pair_diff_ho(const float* __restrict__ hl, int j, int v, float hi_i, float lo_i) {
  const float2 p = __ldg(reinterpret_cast<const float2*>(hl + (size_t)j * 10 + 2 * v));
  return (p.x - hi_i) + (p.y - lo_i);
}

// one chunk's contraction into acc[0 .. KK): members in pairs, in order
template <int KK, int MM>
__device__ __forceinline__ void chunk_contract(const float* chunk, int c, const float* __restrict__ hl, int v,
                                               float hi_i, float lo_i, float (&acc)[KK]) {
  constexpr int TC = 64;
  const float2* P = reinterpret_cast<const float2*>(chunk + MM * TC);
#pragma unroll
  for (int mp = 0; mp < MM / 2; mp++) {
    const int j0 = reinterpret_cast<const int*>(chunk)[(2 * mp) * TC + c];
    const int j1 = reinterpret_cast<const int*>(chunk)[(2 * mp + 1) * TC + c];
    const float d0 = pair_diff_ho(hl, j0, v, hi_i, lo_i), d1 = pair_diff_ho(hl, j1, v, hi_i, lo_i);
#pragma unroll
    for (int k = 0; k < KK; k++) {
      const float2 p = P[(k * (MM / 2) + mp) * TC + c];
      acc[k] = fmaf(p.y, d1, fmaf(p.x, d0, acc[k]));
    }
  }
}

// One block per 64-cell tile: thread (cell c, variable v) = 5 c + v, plus a
// copying warp that streams the tile's chunks (central; with CWENOZ the
// smoothness matrices, then the directional chunks twice, once for the
// indicators and once for the combination) through a ring of S shared-memory
// stages, every wait bounded.
// Per variable the arithmetic is that of the FP64 form in FP32, members and
// modes in the same order.  Blocks per SM: P3 three, P4 two (linear) or one
// (CWENOZ: 168 registers a thread without spills; two blocks at 80 registers
// spill and measured no faster).
template <int ORDER, bool WENO>
__global__ void __launch_bounds__(HOTile<ORDER>::THREADS, ORDER == 4 ? (WENO ? 1 : 2) : 3) k_recon_ho_mx(ReconArgsHOMx a) {
  using T = HOTile<ORDER>;
  constexpr int K = T::K, KD = T::KD, ND = 6, TC = T::TC, S = T::S;
  constexpr int NQ = T::NCC + (WENO ? T::NMC + 2 * ND * T::NDC : 0);  // chunks streamed per tile
  extern __shared__ __align__(128) unsigned char smem[];
  float* st = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(st + S * T::STAGE);
  uint64_t* empty = full + S;
  const int t = threadIdx.x, lane = t & 31, tile = blockIdx.x;
  if (t < S) {
    bar_init(&full[t]);
    bar_init(&empty[t], 5 * TC / 32);
  }
  __syncthreads();
  if (t >= 5 * TC) {  // the copying warp
    if (lane != 0) return;
    const float* base = a.tiles + (size_t)tile * T::tile_floats(WENO);
    int q = 0;
    bool ok = true;
    for (; q < NQ; q++) {
      if (q >= S && !bar_wait(&empty[q % S], (uint32_t)(q / S + 1) & 1u)) {
        ok = false;
        break;
      }
      // chunk q: central chunks first, then the directional ones in two rounds
      const float* src;
      uint32_t bytes;
      if (q < T::NCC) {
        src = base + (size_t)q * T::CCS;
        bytes = T::CCS * 4u;
      } else if (q < T::NCC + T::NMC) {
        const int r0 = (q - T::NCC) * T::MSR;
        src = base + T::CENTRAL + (size_t)r0 * TC;
        bytes = (uint32_t)(min(T::MSR, T::NQS - r0) * TC) * 4u;
      } else {
        const int qd = (q - T::NCC - T::NMC) % (ND * T::NDC);
        src = base + T::CENTRAL + T::SMAT + (size_t)qd * T::DCS;
        bytes = T::DCS * 4u;
      }
      bar_expect(&full[q % S], bytes);
      bulk_load(st + (q % S) * T::STAGE, src, bytes, &full[q % S]);
    }
    if (!ok) atomicOr(a.err, 2);
    // the last copies into each stage land before the block's shared memory is released
    for (int qq = q - 1; qq >= 0 && qq >= q - S; qq--) bar_wait(&full[qq % S], (uint32_t)(qq / S) & 1u);
    return;
  }
  const int c = t / 5, v = t - 5 * (t / 5);
  const int i0 = tile * TC + c;
  const bool live = i0 < a.N;
  const int i = live ? i0 : a.N - 1;
  const size_t N = a.N;
  const float* __restrict__ hl = a.Uhl;
  const float2 pi = __ldg(reinterpret_cast<const float2*>(hl + (size_t)i * 10 + 2 * v));
  const float hi_i = pi.x, lo_i = pi.y;
  int q = 0;
  bool ok = true;
  auto take = [&]() -> const float* {  // wait for chunk q
    ok = ok && __all_sync(0xffffffffu, bar_wait(&full[q % S], (uint32_t)(q / S) & 1u));
    return st + (q % S) * T::STAGE;
  };
  auto give = [&]() {  // this warp is done with chunk q
    __syncwarp();
    if (lane == 0) bar_arrive(&empty[q % S]);
    q++;
  };
  float ao[K];
#pragma unroll
  for (int k = 0; k < K; k++) ao[k] = 0.f;
#pragma unroll 1
  for (int ch = 0; ch < T::NCC; ch++) {
    const float* chunk = take();
    if (!ok) break;
    chunk_contract<K, T::MCH>(chunk, c, hl, v, hi_i, lo_i, ao);
    give();
  }
  float cf[K];
  if constexpr (!WENO) {
#pragma unroll
    for (int k = 0; k < K; k++) cf[k] = ao[k];
  } else {
    // a^T M a of the central coefficients, M's entries from the streamed
    // chunks in row order (each row's diagonal entry read first; the
    // arithmetic as in si_form)
    float SI0 = 0.f;
    {
      const float* mc = take();
#pragma unroll
      for (int k = 0; k < K; k++) {
        const int q0 = k * K - k * (k - 1) / 2;
        auto M = [&](int qq) -> float {
          if (qq % T::MSR == 0 && qq != 0) {
            give();
            mc = take();
          }
          return mc[(qq % T::MSR) * TC + c];
        };
        const float mkk = M(q0);
        float tk = 0.f;
#pragma unroll
        for (int l = k + 1; l < K; l++) tk = fmaf(M(q0 + l - k), ao[l], tk);
        SI0 = fmaf(ao[k], fmaf(2.f, tk, mkk * ao[k]), SI0);
      }
      give();
    }
    float SI[ND];
    float tau = 0.f;
#pragma unroll 1
    for (int s = 0; s < ND && ok; s++) {
      float b[KD];
#pragma unroll
      for (int k = 0; k < KD; k++) b[k] = 0.f;
#pragma unroll 1
      for (int h = 0; h < T::NDC; h++) {
        const float* chunk = take();
        if (!ok) break;
        chunk_contract<KD, T::MDH>(chunk, c, hl, v, hi_i, lo_i, b);
        give();
      }
      SI[s] = si_form_f<K, KD>(a.Msi, N, i, b);
      tau += fabsf(SI0 - SI[s]);
    }
    tau *= (1.f / ND);
    const float w0 = a.lam0 * (1.f + fdiv(tau, a.eps + SI0));
    float ws[ND];
    float wsum = w0;
#pragma unroll
    for (int s = 0; s < ND; s++) {
      ws[s] = a.lams * (1.f + fdiv(tau, a.eps + SI[s]));
      wsum += ws[s];
    }
    const float iws = fdiv(1.f, wsum);
    const float r0 = fdiv(w0 * iws, a.lam0);
#pragma unroll
    for (int k = 0; k < K; k++) cf[k] = r0 * ao[k];
#pragma unroll 1
    for (int s = 0; s < ND && ok; s++) {
      float b[KD];
#pragma unroll
      for (int k = 0; k < KD; k++) b[k] = 0.f;
#pragma unroll 1
      for (int h = 0; h < T::NDC; h++) {
        const float* chunk = take();
        if (!ok) break;
        chunk_contract<KD, T::MDH>(chunk, c, hl, v, hi_i, lo_i, b);
        give();
      }
      const float e = ws[s] * iws - r0 * a.lams;
#pragma unroll
      for (int k = 0; k < KD; k++) cf[k] = fmaf(e, b[k], cf[k]);
    }
  }
  if (!ok) {
    if (lane == 0) atomicOr(a.err, 2);
    return;
  }
  if (!live) return;
  // the constant term relative to U_ref = (1, 0, 0, 0, E_ref), less the means of
  // the non-linear monomials; coefficients in physical units
  float c0 = v == 0 ? (hi_i - 1.f) + lo_i : (v == 4 ? (hi_i - a.eref_hi) + (lo_i - a.eref_lo) : hi_i + lo_i);
#pragma unroll
  for (int k = 3; k < K; k++) c0 = fmaf(-cf[k], __ldg(&a.psib[(size_t)(k - 3) * N + i]), c0);
  const float ih = __ldg(&a.inv_h[i]);
  float ihp[ORDER + 1];
  ihp[0] = 1.f;
#pragma unroll
  for (int e = 1; e <= ORDER; e++) ihp[e] = ihp[e - 1] * ih;
  float* out = a.coef + (size_t)i * a.cs;
  out[cidx(v, 0, K + 1)] = c0;
#pragma unroll
  for (int k = 0; k < K; k++) out[cidx(v, k + 1, K + 1)] = cf[k] * ihp[basis_degree(k)];
}

}  // namespace ucns
