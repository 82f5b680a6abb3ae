// Mixed-precision variants of the reconstruction and face kernels.
//
// FP32: pseudo-inverses and their contractions, smoothness indicators,
// CWENOZ weights, polynomial evaluation, HLLC and viscous flux arithmetic.
// Stencil differences U_j - U_i (cancellation) are taken from a float pair
// (hi, lo) of the FP64 state, whose leading parts subtract exactly, so each
// difference equals the FP64 difference to within its own FP32 rounding.
// FP64: the state itself, the face-flux totals G_f, the residual sum and the
// Runge-Kutta update (k_rk), the dt and diagnostic reductions.
//
// States inside the FP32 flux are carried relative to the reference state
// U_ref = (1, 0, 0, 0, p_ref/(gamma-1)), p_ref = 1/(gamma M^2), so that a
// float holds O(1) numbers: rho = 1 + rho', E = E_ref + E', and the pressure
// p = p_ref + p' with p' = (gamma-1)(E' - |m|^2/(2 rho)).  The momentum flux
// uses p' in place of p: the dropped p_ref n integrates to zero over every
// closed cell (the oint n dS = 0 of the FP64 geometry), so the residual is
// unchanged.  The HLLC star states are formed in difference form
// (U* - U = r U + ...), which keeps every FP32 term O(1).
#pragma once

#include "basis.hpp"
#include "bulk.cuh"
#include "kernels.cuh"

namespace ucns {

struct FluxConstF {
  float gam, gm1, mu, kap, gm1_over_R;
  float p_ref, H_ref;  // reference pressure and enthalpy E_ref + p_ref
};

// The mixed form keeps its per-cell precompute in a blocked layout: cells in
// tiles of kTC consecutive (Morton-ordered) cells, and for every tile all rows
// of an array [rows][kTC] contiguous, so that one bulk copy brings a tile's
// pseudo-inverse rows (or stencil lists) into shared memory.  Cells past N in
// the last tile are zero rows.
constexpr int kTC = 64;

// FP32 division and square root of the mixed form: the hardware approximate
// reciprocal and reciprocal square root (at most 2 ulp: CUDA's __fdividef and
// rsqrtf), an error of the order of the FP32 rounding that the operands
// already carry.  For a physical state every divisor here is a nonzero
// number of moderate magnitude (densities, sound-speed sums, smoothness sums
// plus epsilon, wave-speed differences) and every radicand is positive.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float fsqrt(float x) { return x * rsqrtf(x); }

// index of (row, cell i) in a blocked array [ceil(N / kTC)][rows][kTC]
__host__ __device__ __forceinline__ size_t blk(int row, int rows, int64_t i) {
  return ((size_t)(i / kTC) * rows + row) * kTC + (size_t)(i % kTC);
}

// index of (row, cell i) in a pair-blocked array [ceil(N / kTC)][rows / 2][kTC][2]
// (rows even): rows 2j and 2j + 1 of a cell are adjacent, so one 8-byte load
// reads both (the pseudo-inverse rows of consecutive stencil members)
__host__ __device__ __forceinline__ size_t blk2(int row, int rows, int64_t i) {
  return (((size_t)(i / kTC) * (rows / 2) + row / 2) * kTC + (size_t)(i % kTC)) * 2 + (row & 1);
}

// index of entry k (0: the constant term) of variable v in a mixed-form
// coefficient row with ncf = K + 1 entries per variable: variables 0-3
// interleaved per entry (k 4 + v, so one 16-byte load brings entry k of all
// four, as two packed FP32x2 pairs), variable 4 after them (4 ncf + k)
__host__ __device__ constexpr int cidx(int v, int k, int ncf) { return v < 4 ? k * 4 + v : 4 * ncf + k; }

// blocked per-cell FP32 rows of the mixed form: the six second moments
// (1/V) int xi_a xi_b (xx yy zz xy xz yz), then 1/h
constexpr int kCellRows = 7;

template <int ORDER, bool WENO, int ND>
struct ReconTile {
  static constexpr int K = ORDER == 1 ? 3 : 9;
  static constexpr int MC = 2 * K, MD = 6;
  static constexpr int RC = K * MC;                 // central pseudo-inverse rows
  static constexpr int RD = WENO ? ND * 3 * MD : 0;  // directional pseudo-inverse rows
  static constexpr int SD = WENO ? ND * MD : 0;      // directional stencil rows
  static constexpr int CS = ORDER == 1 ? 20 : 52;    // floats per output row: 5 (K+1) rounded up to 4
  // shared memory of one tile: central rows and stencil, the cell rows,
  // directional rows and stencils (CWENOZ), the tile's output rows, the mbarrier
  static constexpr size_t smem() {
    return (size_t)(RC + MC + kCellRows + RD + SD) * kTC * 4 + (size_t)kTC * CS * 4 + 16;
  }
};

struct ReconArgsMx {
  const float* __restrict__ Uhl;  // [N][5][2]: (hi, lo) = (fl(U), fl(U - hi)) of each variable
  const int32_t* __restrict__ sc;  // pair-blocked, rows m (MC)
  const float* __restrict__ Pc;    // pair-blocked, rows k MC + m (K MC)
  const int32_t* __restrict__ sd;  // pair-blocked, rows s Md + r (nd Md)
  const float* __restrict__ Pd;    // pair-blocked, rows (s 3 + k) Md + r (nd 3 Md)
  const float* __restrict__ cell;  // blocked [tiles][kCellRows][kTC]
  float* __restrict__ coef;        // [N][cs]: entry k of variable v at cidx(v, k, K + 1),
                                   // k = 0 the constant term relative to U_ref
  // gated reconstruction (P2 CWENOZ on the flagged cells only)
  const uint8_t* __restrict__ gate;  // [N] flags (nonzero: CWENOZ)
  const int32_t* __restrict__ sda;   // [N][nd Md] directional stencils, cell-contiguous
  const float* __restrict__ Pda;     // [N][nd 3 Md] directional pseudo-inverse rows, cell-contiguous
  int* err;                        // bit 1 set when a bounded wait gave up
  int N;
  int cs;  // floats per cell row of coef (5 (K+1) rounded up to a multiple of 4)
  float lam0, lams, eps;
  float eref_hi, eref_lo;  // E_ref = p_ref/(gamma-1) as a float pair (rho_ref = 1 exactly)
};

struct FaceArgsMx {
  const float* __restrict__ coef;     // [N][cs] cell rows, 16-byte aligned
  const float* __restrict__ fq;       // [F'][nq][10]: x - x_L, x - x_R', n, |dS| of each Gauss point
  const float* __restrict__ fpen;     // [F']
  const int32_t* __restrict__ fslot;  // [F']: slots of the owner's (low 16 bits) and neighbour's rows in the batch
  const int32_t* __restrict__ bcell;  // [batches][nu]: the batch's distinct cells, slot order
  const int32_t* __restrict__ bcount; // [batches]: how many
  float* __restrict__ G;              // [5][F] FP32 face totals
  int* err;                           // bit 1: a copy wait gave up
  int N, F;                           // F' = F rounded up to whole batches (zero entries)
  int cs;
  int nu;      // slots per batch (at least the largest count)
  int stages;  // pipeline depth, 2 .. kFaceMaxStages
  FluxConstF c;
};

// The face kernel's pipeline.  A persistent block has kFaceWarps warps that
// evaluate (thread = one Gauss point; a warp takes 32 / nq whole faces, so
// 9-point faces leave 5 lanes idle) and kFaceCopyWarps warps that copy,
// batch by batch in turn.  A copying warp brings each batch's Gauss points,
// penalty factors and row slots (bulk copies) and the coefficient rows of its
// distinct cells (each once, a cell shared by several of the batch's faces
// included; 16-byte asynchronous copies spread over the lanes) into one of
// `stages` shared-memory stages, up to stages - 1 batches ahead of the
// evaluating warps, which hand a stage back through its "empty" barrier.
constexpr int kFaceWarps = 16;
constexpr int kFaceCopyWarps = 3;  // copying warp w takes the block's batches k = w mod 3
constexpr int kFaceThreads = 32 * (kFaceWarps + kFaceCopyWarps);
constexpr int kFacePad = 1536;     // the per-face arrays hold whole batches at every order (512, 128, 48, 32 faces)
constexpr int kFaceMaxStages = 6;

// faces per batch for nq Gauss points per face
__host__ __device__ constexpr int face_batch_faces(int nq) { return kFaceWarps * (32 / nq); }

template <int ORDER>
struct FaceTileMx {
  static constexpr int NQ = ORDER * ORDER;
  static constexpr int FPW = 32 / NQ;                                                // faces per warp
  static constexpr int CS = ORDER == 1 ? 20 : (ORDER == 2 ? 52 : (ORDER == 3 ? 100 : 176));  // floats per row
  static constexpr int FB = face_batch_faces(NQ);                                    // faces per batch
  static constexpr int PTS = FB * NQ * 10;                                           // the batch's Gauss points
  static constexpr int NUR = (2 * FB + 31) / 32;  // slot registers per lane of a copying warp
  // a stage: Gauss points, penalties, slot words, then nu rows
  __host__ __device__ static constexpr int stage_floats(int nu) { return PTS + 2 * FB + nu * CS; }
  __host__ __device__ static constexpr size_t smem(int nu, int stages) {
    return (size_t)stages * stage_floats(nu) * 4 + (size_t)2 * kFaceMaxStages * 8;
  }
  static_assert(kFacePad % FB == 0 && (PTS + 2 * FB) % 4 == 0 && CS % 4 == 0, "whole 16-byte copies");
};

// U_j - U_i of variable v from the float pairs: hi_j - hi_i is exact for
// same-sign values within a factor 2 (Sterbenz), so the difference carries no
// cancellation error beyond the final FP32 rounding, as an FP64 subtraction would
__device__ __forceinline__ float pair_diff(const float* __restrict__ hl, int j, int v, float hi_i, float lo_i) {
  // one 8-byte load of (hi, lo); 32-bit row offset (N < 2^31 / 10, checked on the host)
  const float2 p = *reinterpret_cast<const float2*>(hl + j * 10 + 2 * v);
  return (p.x - hi_i) + (p.y - lo_i);
}

// CWENOZ combination of the central coefficients ao (K = 9, xi units) with the
// nd directional linear coefficients b: smoothness indicators (Eq. 6 reading),
// tau, the nonlinear weights and the combined coefficients cf
template <int ND>
__device__ __forceinline__ void cwenoz_mx(const float (&ao)[9], const float (&b)[ND][3], const float (&S)[6],
                                          const ReconArgsMx& a, float (&cf)[9]) {
  const float qx0 = 2.f * ao[3], qx1 = ao[6], qx2 = ao[7];
  const float qy0 = ao[6], qy1 = 2.f * ao[4], qy2 = ao[8];
  const float qz0 = ao[7], qz1 = ao[8], qz2 = 2.f * ao[5];
  auto quad = [&](float x0, float x1, float x2) {
    return S[0] * x0 * x0 + S[1] * x1 * x1 + S[2] * x2 * x2 + 2.f * (S[3] * x0 * x1 + S[4] * x0 * x2 + S[5] * x1 * x2);
  };
  const float SI0 = ao[0] * ao[0] + ao[1] * ao[1] + ao[2] * ao[2] + quad(qx0, qx1, qx2) + quad(qy0, qy1, qy2) +
                    quad(qz0, qz1, qz2) + 4.f * (ao[3] * ao[3] + ao[4] * ao[4] + ao[5] * ao[5]) + ao[6] * ao[6] +
                    ao[7] * ao[7] + ao[8] * ao[8];
  float SI[ND];
  float tau = 0.f;
#pragma unroll
  for (int s = 0; s < ND; s++) {
    SI[s] = b[s][0] * b[s][0] + b[s][1] * b[s][1] + b[s][2] * b[s][2];
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
  for (int k = 0; k < 9; k++) cf[k] = r0 * ao[k];
#pragma unroll
  for (int s = 0; s < ND; s++) {
    const float e = ws[s] * iws - r0 * a.lams;
#pragma unroll
    for (int k = 0; k < 3; k++) cf[k] = fmaf(e, b[s][k], cf[k]);
  }
}

// the K + 1 row entries of variable v: the constant term relative to the
// reference state U_ref = (1, 0, 0, 0, E_ref) (the cell mean minus the mean
// of the non-constant monomials), then the coefficients in physical units
// (linear / h, quadratic / h^2); row points at the cell's row
template <int K>
__device__ __forceinline__ void write_var(float* row, int v, float hi_i, float lo_i, const float (&cf)[K],
                                          const float (&S)[6], float ih, const ReconArgsMx& a) {
  float c0 = v == 0 ? (hi_i - 1.f) + lo_i : (v == 4 ? (hi_i - a.eref_hi) + (lo_i - a.eref_lo) : hi_i + lo_i);
  if (K == 9) {
#pragma unroll
    for (int q = 0; q < 6; q++) c0 = fmaf(-cf[3 + q], S[q], c0);
  }
  const float ih2 = ih * ih;
  row[cidx(v, 0, K + 1)] = c0;
#pragma unroll
  for (int k = 0; k < K; k++) row[cidx(v, k + 1, K + 1)] = cf[k] * (k < 3 ? ih : ih2);
}

// Second phase of a gated P2 CWENOZ tile (after its linear rows are in
// sOut): the flagged cells of the tile are compacted in shared memory, their
// central coefficients ao (xi units, from the linear phase's registers) are
// parked where the central pseudo-inverse rows were (no longer read), and one
// warp per flagged cell finishes it: lane (v, s), v < 5, s < nd, contracts
// directional stencil s of variable v from cell-contiguous copies of the ids
// and rows; lane (v, 0) gathers the nd results by shuffles and runs the same
// cwenoz_mx / write_var as the ungated kernel (whose arithmetic and order
// this reproduces: a fully flagged gate equals it bit for bit), overwriting
// the cell's linear entries in sOut.  Called by every thread of the block.
template <int ND>
__device__ __forceinline__ void gated_cwenoz(const ReconArgsMx& a, const float (&ao)[9], bool flagged, int c, int v,
                                             int i0, float* sP, const float* sC, float* sOut) {
  using T = ReconTile<2, true, ND>;
  constexpr int K = 9, MD = T::MD, CS = T::CS;
  static_assert(5 * ND <= 32, "one lane per (variable, stencil)");
  __shared__ int s_n;
  __shared__ int s_slot[kTC];  // slot of cell c among the flagged
  __shared__ int s_cell[kTC];  // cell of a slot
  const int t = threadIdx.x;
  if (t == 0) s_n = 0;
  __syncthreads();  // also: every linear-phase read of sP is done
  if (flagged && v == 0) {
    const int sl = atomicAdd(&s_n, 1);
    s_slot[c] = sl;
    s_cell[sl] = c;
  }
  __syncthreads();
  const int nf = s_n;
  if (nf == 0) return;
  float* s_ao = sP;  // [nf][48]
  if (flagged) {
#pragma unroll
    for (int k = 0; k < K; k++) s_ao[s_slot[c] * 48 + v * K + k] = ao[k];
  }
  __syncthreads();
  const float* __restrict__ hl = a.Uhl;
  const int lane = t & 31;
  const int lv = lane / ND, lsn = lane - ND * (lane / ND);
  const bool act = lane < 5 * ND;
  const int vv = act ? lv : 0, ss = act ? lsn : 0;
  for (int sl = t >> 5; sl < nf; sl += blockDim.x >> 5) {
    const int cc = s_cell[sl], ii = i0 + cc;
    const float2 pi = *reinterpret_cast<const float2*>(hl + (size_t)ii * 10 + 2 * vv);
    const float hi_i = pi.x, lo_i = pi.y;
    const int2* js = reinterpret_cast<const int2*>(a.sda + (size_t)ii * T::SD + ss * MD);
    const float2* ps = reinterpret_cast<const float2*>(a.Pda + (size_t)ii * T::RD + ss * 3 * MD);
    int jj[MD];
#pragma unroll
    for (int q = 0; q < MD / 2; q++) {
      const int2 w = __ldg(js + q);
      jj[2 * q] = w.x;
      jj[2 * q + 1] = w.y;
    }
    float bk[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int rp = 0; rp < MD / 2; rp++) {  // members r = 2 rp, 2 rp + 1: rows k MD + r, k < 3
      const float d0 = pair_diff(hl, jj[2 * rp], vv, hi_i, lo_i), d1 = pair_diff(hl, jj[2 * rp + 1], vv, hi_i, lo_i);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const float2 P = __ldg(ps + (k * MD + 2 * rp) / 2);
        bk[k] = fmaf(P.y, d1, fmaf(P.x, d0, bk[k]));
      }
    }
    float b[ND][3];
#pragma unroll
    for (int s = 0; s < ND; s++)
#pragma unroll
      for (int k = 0; k < 3; k++) b[s][k] = __shfl_sync(0xffffffffu, bk[k], vv * ND + s);
    if (act && lsn == 0) {
      float aoc[K];
#pragma unroll
      for (int k = 0; k < K; k++) aoc[k] = s_ao[sl * 48 + lv * K + k];
      float S[6];
#pragma unroll
      for (int q = 0; q < 6; q++) S[q] = sC[q * kTC + cc];
      const float ih = sC[6 * kTC + cc];
      float cf[9];
      cwenoz_mx<ND>(aoc, b, S, a, cf);
      write_var<9>(sOut + cc * CS, lv, hi_i, lo_i, cf, S, ih, a);
    }
  }
}

// One block per tile of kTC cells, thread = (cell c of the tile, variable v).
// A single thread starts bulk copies of the tile's central pseudo-inverse rows
// and stencil, its cell rows and (CWENOZ) its directional rows and stencils
// into shared memory; meanwhile every thread loads its own state.  The
// coefficient rows are assembled in shared memory and written back with one
// bulk copy.  GATED (WENO = false, P2): a gated CWENOZ reconstruction, linear
// weights for every cell first, then gated_cwenoz for the flagged ones.
template <int ORDER, bool WENO, int ND, bool GATED>
__global__ void __launch_bounds__(kTC * 5, WENO ? 2 : 3) k_recon_mx(ReconArgsMx a) {
  using T = ReconTile<ORDER, WENO, ND>;
  constexpr int K = T::K, MC = T::MC, MD = T::MD, CS = T::CS;
  extern __shared__ __align__(128) unsigned char smem[];
  float* sP = reinterpret_cast<float*>(smem);
  int32_t* sS = reinterpret_cast<int32_t*>(sP + T::RC * kTC);
  float* sC = reinterpret_cast<float*>(sS + MC * kTC);
  float* sPd = sC + kCellRows * kTC;
  int32_t* sSd = reinterpret_cast<int32_t*>(sPd + T::RD * kTC);
  float* sOut = reinterpret_cast<float*>(sSd + T::SD * kTC);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sOut + kTC * CS);
  const int tile = blockIdx.x, i0 = tile * kTC;
  const int nc = min(kTC, a.N - i0);
  const int t = threadIdx.x, c = t / 5, v = t - 5 * (t / 5);
  if (t == 0) bar_init(bar);
  __syncthreads();
  if (t == 0) {
    constexpr uint32_t bp = T::RC * kTC * 4, bs = MC * kTC * 4, bc = kCellRows * kTC * 4;
    constexpr uint32_t bpd = T::RD * kTC * 4, bsd = T::SD * kTC * 4;
    bar_expect(bar, bp + bs + bc + bpd + bsd);
    bulk_load(sP, a.Pc + (size_t)tile * T::RC * kTC, bp, bar);
    bulk_load(sS, a.sc + (size_t)tile * MC * kTC, bs, bar);
    bulk_load(sC, a.cell + (size_t)tile * kCellRows * kTC, bc, bar);
    if (WENO) {
      bulk_load(sPd, a.Pd + (size_t)tile * T::RD * kTC, bpd, bar);
      bulk_load(sSd, a.sd + (size_t)tile * T::SD * kTC, bsd, bar);
    }
  }
  const bool live = c < nc;
  const int i = i0 + (live ? c : 0);
  const float* __restrict__ hl = a.Uhl;
  const float2 pi = *reinterpret_cast<const float2*>(hl + (size_t)i * 10 + 2 * v);
  const float hi_i = pi.x, lo_i = pi.y;
  const bool ok = bar_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(a.err, 2);
    bar_wait(bar, 0);  // the copies into this block's shared memory end before it exits
    return;
  }
  float ao[K];
#pragma unroll
  for (int k = 0; k < K; k++) ao[k] = 0.f;
  if (live) {
    const int2* sS2 = reinterpret_cast<const int2*>(sS);
    const float2* sP2 = reinterpret_cast<const float2*>(sP);
#pragma unroll 3
    for (int mp = 0; mp < MC / 2; mp++) {  // stencil members m = 2 mp, 2 mp + 1
      const int2 jj = sS2[mp * kTC + c];
      const float d0 = pair_diff(hl, jj.x, v, hi_i, lo_i), d1 = pair_diff(hl, jj.y, v, hi_i, lo_i);
#pragma unroll
      for (int k = 0; k < K; k++) {
        const float2 P = sP2[(k * (MC / 2) + mp) * kTC + c];
        ao[k] = fmaf(P.y, d1, fmaf(P.x, d0, ao[k]));
      }
    }
    float S[6];
#pragma unroll
    for (int q = 0; q < 6; q++) S[q] = sC[q * kTC + c];
    const float ih = sC[6 * kTC + c];
    float* out = sOut + c * CS;
    if constexpr (WENO) {
      float b[ND][3];
      const int2* sSd2 = reinterpret_cast<const int2*>(sSd);
      const float2* sPd2 = reinterpret_cast<const float2*>(sPd);
#pragma unroll
      for (int s = 0; s < ND; s++) {
        b[s][0] = b[s][1] = b[s][2] = 0.f;
#pragma unroll
        for (int rp = 0; rp < MD / 2; rp++) {  // members r = 2 rp, 2 rp + 1
          const int2 jj = sSd2[(s * (MD / 2) + rp) * kTC + c];
          const float d0 = pair_diff(hl, jj.x, v, hi_i, lo_i), d1 = pair_diff(hl, jj.y, v, hi_i, lo_i);
#pragma unroll
          for (int k = 0; k < 3; k++) {
            const float2 P = sPd2[((s * 3 + k) * (MD / 2) + rp) * kTC + c];
            b[s][k] = fmaf(P.y, d1, fmaf(P.x, d0, b[s][k]));
          }
        }
      }
      float cf[9];
      cwenoz_mx<ND>(ao, b, S, a, cf);
      write_var<9>(out, v, hi_i, lo_i, cf, S, ih, a);
    } else {
      write_var<K>(out, v, hi_i, lo_i, ao, S, ih, a);
    }
    if (v == 0) {
#pragma unroll
      for (int q = 5 * (K + 1); q < CS; q++) sOut[c * CS + q] = 0.f;
    }
  }
  if constexpr (GATED) gated_cwenoz<ND>(a, ao, live && a.gate[i], c, v, i0, sP, sC, sOut);
  fence_smem_to_async();
  __syncthreads();
  if (t == 0) bulk_store(a.coef + (size_t)i0 * CS, sOut, (uint32_t)(nc * CS * 4));
}

// float pairs of an FP64 state, cell-contiguous [N][5][2]: (hi, lo) =
// (fl(U), fl(U - hi)) of each variable; thread = (cell, variable)
__global__ void __launch_bounds__(256) k_split(const double* __restrict__ U, float* __restrict__ hl, int N) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 5 * N) return;
  const int i = k / 5, v = k - 5 * (k / 5);
  split_pair(U[(size_t)v * N + i], hl[(size_t)i * 10 + 2 * v], hl[(size_t)i * 10 + 2 * v + 1]);
}

// float pairs of a flat array (the C ABI's ucns_float_pair)
__global__ void __launch_bounds__(256) k_float_pair(const double* __restrict__ u, float* __restrict__ hi,
                                                    float* __restrict__ lo, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) split_pair(u[k], hi[k], lo[k]);
}

// value at the physical offset (x, y, z) from the centroid into U; gradient
// written (ACC = false) or added (ACC = true) into g; the cell's coefficient
// row is read with 16-byte loads.  Variables 0-3 are evaluated in packed
// FP32x2 pairs (0, 1) and (2, 3), whose lanes round exactly as the scalar
// operations of variable 4 (the same FMA sequence per variable).
template <int ORDER, bool ACC>
__device__ __forceinline__ void eval_side_mx(const float* row_, float x, float y, float z, float U[5],
                                             float g[5][3]) {
  constexpr int CS = ORDER == 1 ? 20 : 52;
  constexpr int NCF = ORDER == 1 ? 4 : 10;  // entries per variable
  float4 q[CS / 4];
  const float4* row = reinterpret_cast<const float4*>(row_);
#pragma unroll
  for (int i = 0; i < CS / 4; i++) q[i] = row[i];
  const float2 X = make_float2(x, x), Y = make_float2(y, y), Z = make_float2(z, z);
#pragma unroll
  for (int p = 0; p < 2; p++) {
    auto c = [&](int k) { return p == 0 ? make_float2(q[k].x, q[k].y) : make_float2(q[k].z, q[k].w); };
    float2 u, gx, gy, gz;
    if (ORDER == 1) {
      u = __ffma2_rn(c(1), X, __ffma2_rn(c(2), Y, __ffma2_rn(c(3), Z, c(0))));
      gx = c(1);
      gy = c(2);
      gz = c(3);
    } else {
      const float2 tx = __ffma2_rn(c(4), X, __ffma2_rn(c(7), Y, __ffma2_rn(c(8), Z, c(1))));
      const float2 ty = __ffma2_rn(c(5), Y, __ffma2_rn(c(9), Z, c(2)));
      const float2 tz = __ffma2_rn(c(6), Z, c(3));
      u = __ffma2_rn(X, tx, __ffma2_rn(Y, ty, __ffma2_rn(Z, tz, c(0))));
      gx = __ffma2_rn(c(4), X, tx);
      gy = __ffma2_rn(c(7), X, __ffma2_rn(c(5), Y, ty));
      gz = __ffma2_rn(c(8), X, __ffma2_rn(c(9), Y, __ffma2_rn(c(6), Z, tz)));
    }
    const int v = 2 * p;
    U[v] = u.x;
    U[v + 1] = u.y;
    if (ACC) {
      gx = __fadd2_rn(make_float2(g[v][0], g[v + 1][0]), gx);
      gy = __fadd2_rn(make_float2(g[v][1], g[v + 1][1]), gy);
      gz = __fadd2_rn(make_float2(g[v][2], g[v + 1][2]), gz);
    }
    g[v][0] = gx.x;
    g[v + 1][0] = gx.y;
    g[v][1] = gy.x;
    g[v + 1][1] = gy.y;
    g[v][2] = gz.x;
    g[v + 1][2] = gz.y;
  }
  // variable 4: entries 4 NCF + k
  const float* f = reinterpret_cast<const float*>(q);
  const float c0 = f[4 * NCF], c1 = f[4 * NCF + 1], c2 = f[4 * NCF + 2], c3 = f[4 * NCF + 3];
  float gx, gy, gz;
  if (ORDER == 1) {
    U[4] = fmaf(c1, x, fmaf(c2, y, fmaf(c3, z, c0)));
    gx = c1;
    gy = c2;
    gz = c3;
  } else {
    const float c4 = f[4 * NCF + 4], c5 = f[4 * NCF + 5], c6 = f[4 * NCF + 6];
    const float c7 = f[4 * NCF + 7], c8 = f[4 * NCF + 8], c9 = f[4 * NCF + 9];
    const float tx = fmaf(c4, x, fmaf(c7, y, fmaf(c8, z, c1)));
    const float ty = fmaf(c5, y, fmaf(c9, z, c2));
    const float tz = fmaf(c6, z, c3);
    U[4] = fmaf(x, tx, fmaf(y, ty, fmaf(z, tz, c0)));
    gx = fmaf(c4, x, tx);
    gy = fmaf(c7, x, fmaf(c5, y, ty));
    gz = fmaf(c8, x, fmaf(c9, y, fmaf(c6, z, tz)));
  }
  if (ACC) {
    g[4][0] += gx;
    g[4][1] += gy;
    g[4][2] += gz;
  } else {
    g[4][0] = gx;
    g[4][1] = gy;
    g[4][2] = gz;
  }
}

// HLLC in reference-relative FP32 variables.  W = (rho', m, E'), rho = 1 + rho'.
__device__ __forceinline__ void hllc_flux_mx(const float WL[5], const float WR[5], const float n[3],
                                             const FluxConstF& c, float F[5]) {
  const float rL = 1.f + WL[0], rR = 1.f + WR[0];
  const float irL = fdiv(1.f, rL), irR = fdiv(1.f, rR);
  const float uL[3] = {WL[1] * irL, WL[2] * irL, WL[3] * irL};
  const float uR[3] = {WR[1] * irR, WR[2] * irR, WR[3] * irR};
  const float ppL = c.gm1 * (WL[4] - 0.5f * (WL[1] * uL[0] + WL[2] * uL[1] + WL[3] * uL[2]));
  const float ppR = c.gm1 * (WR[4] - 0.5f * (WR[1] * uR[0] + WR[2] * uR[1] + WR[3] * uR[2]));
  const float pL = c.p_ref + ppL, pR = c.p_ref + ppR;
  const float unL = uL[0] * n[0] + uL[1] * n[1] + uL[2] * n[2];
  const float unR = uR[0] * n[0] + uR[1] * n[1] + uR[2] * n[2];
  const float aL = fsqrt(c.gam * pL * irL), aR = fsqrt(c.gam * pR * irR);
  const float sL = fsqrt(rL), sR = fsqrt(rR), iw = fdiv(1.f, sL + sR);
  const float ut0 = (sL * uL[0] + sR * uR[0]) * iw, ut1 = (sL * uL[1] + sR * uR[1]) * iw,
              ut2 = (sL * uL[2] + sR * uR[2]) * iw;
  // total enthalpy H = (E + p)/rho = (H_ref + E' + p')/rho
  const float Ht = (sL * (c.H_ref + WL[4] + ppL) * irL + sR * (c.H_ref + WR[4] + ppR) * irR) * iw;
  const float at = fsqrt(c.gm1 * (Ht - 0.5f * (ut0 * ut0 + ut1 * ut1 + ut2 * ut2)));
  const float utn = ut0 * n[0] + ut1 * n[1] + ut2 * n[2];
  const float SL = fminf(unL - aL, utn - at);
  const float SR = fmaxf(unR + aR, utn + at);
  const float mL = rL * (SL - unL), mR = rR * (SR - unR);
  const float Ss = fdiv(ppR - ppL + unL * mL - unR * mR, mL - mR);
  // The flux is that of the upwind side (left when S_L >= 0 or S* >= 0),
  // plus S (U* - U) of that side in the star region (S_L < 0 on the left,
  // S_R >= 0 on the right).  Written without branches: the side's
  // quantities are selected first, so a warp whose faces fall on different
  // sides runs one path.  Physical flux: momentum with p', energy with the
  // full E + p.  U* - U with r* = (S* - u_n)/(S - S*): d_rho = rho r*,
  // d_m = r* m + rho* (S* - u_n) n, d_E = r* E + rho* (S* - u_n)(S* + p/(rho (S - u_n))).
  const bool left = 0.f <= SL || 0.f <= Ss;
  const float W0 = left ? WL[0] : WR[0], W1 = left ? WL[1] : WR[1], W2 = left ? WL[2] : WR[2];
  const float W3 = left ? WL[3] : WR[3], W4 = left ? WL[4] : WR[4];
  (void)W0;
  const float r = left ? rL : rR, un = left ? unL : unR, pp = left ? ppL : ppR, p = left ? pL : pR;
  const float S = left ? SL : SR, m = left ? mL : mR;
  const bool in_star = left ? SL < 0.f : 0.f <= SR;
  F[0] = r * un;
  F[1] = W1 * un + pp * n[0];
  F[2] = W2 * un + pp * n[1];
  F[3] = W3 * un + pp * n[2];
  F[4] = (W4 + pp) * un + c.H_ref * un;
  const float ds = Ss - un;
  const float rs = fdiv(ds, S - Ss);
  const float rho_s = r + r * rs;
  const float E = (c.H_ref - c.p_ref) + W4;
  const float t = rho_s * ds;
  const float d0 = S * (r * rs);
  const float d1 = S * fmaf(t, n[0], rs * W1);
  const float d2 = S * fmaf(t, n[1], rs * W2);
  const float d3 = S * fmaf(t, n[2], rs * W3);
  const float d4 = S * fmaf(t, Ss + fdiv(p, m), rs * E);
  // outside the star region these terms may be inf or NaN (S = S*): selected away
  F[0] += in_star ? d0 : 0.f;
  F[1] += in_star ? d1 : 0.f;
  F[2] += in_star ? d2 : 0.f;
  F[3] += in_star ? d3 : 0.f;
  F[4] += in_star ? d4 : 0.f;
}

// viscous flux in FP32 from the reference-relative face state
__device__ __forceinline__ void viscous_flux_mx(const float W[5], const float g[5][3], const float n[3],
                                                const FluxConstF& c, float Fv[5]) {
  const float r = 1.f + W[0];
  const float ir = fdiv(1.f, r);
  const float u[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
  float gu[3][3];
#pragma unroll
  for (int q = 0; q < 3; q++)
#pragma unroll
    for (int j = 0; j < 3; j++) gu[q][j] = (g[1 + q][j] - u[q] * g[0][j]) * ir;
  const float e = ((c.H_ref - c.p_ref) + W[4]) * ir;
  float qn = 0.f;
#pragma unroll
  for (int j = 0; j < 3; j++) {
    const float de = (g[4][j] - e * g[0][j]) * ir - (u[0] * gu[0][j] + u[1] * gu[1][j] + u[2] * gu[2][j]);
    qn += de * n[j];
  }
  const float div = gu[0][0] + gu[1][1] + gu[2][2];
  const float tdiv = (2.f / 3.f) * c.mu * div;
  float work = 0.f;
  Fv[0] = 0.f;
#pragma unroll
  for (int q = 0; q < 3; q++) {
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < 3; j++) t += c.mu * (gu[q][j] + gu[j][q]) * n[j];
    t -= tdiv * n[q];
    Fv[1 + q] = t;
    work += u[q] * t;
  }
  Fv[4] = work + c.kap * c.gm1_over_R * qn;
}

// value and gradient at (x, y, z) of a P3/P4 cell polynomial from its row
// (entries cidx(v, k, K + 1), in global or shared memory): variables 0-3 in
// packed FP32x2 pairs from one 16-byte load per mode, variable 4 from four
// modes per 16-byte load
template <int ORDER, bool ACC>
__device__ __forceinline__ void eval_side_ho_mx(const float* row, float x, float y, float z, float U[5],
                                                float g[5][3]) {
  constexpr int K = basis_count(ORDER), NCF = K + 1;
  const float4* r4 = reinterpret_cast<const float4*>(row);
  float px[ORDER + 1], py[ORDER + 1], pz[ORDER + 1];
  px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
  for (int e = 1; e <= ORDER; e++) {
    px[e] = px[e - 1] * x;
    py[e] = py[e - 1] * y;
    pz[e] = pz[e - 1] * z;
  }
  float e4[4 * ((NCF + 3) / 4)];  // variable 4's entries
#pragma unroll
  for (int jj = 0; jj < (NCF + 3) / 4; jj++) {
    const float4 t = r4[NCF + jj];
    e4[4 * jj] = t.x;
    e4[4 * jj + 1] = t.y;
    e4[4 * jj + 2] = t.z;
    e4[4 * jj + 3] = t.w;
  }
  const float4 c0 = r4[0];
  float2 u01 = make_float2(c0.x, c0.y), u23 = make_float2(c0.z, c0.w);
  float2 gx01 = make_float2(0.f, 0.f), gx23 = gx01, gy01 = gx01, gy23 = gx01, gz01 = gx01, gz23 = gx01;
  float u4 = e4[0], gx4 = 0.f, gy4 = 0.f, gz4 = 0.f;
#pragma unroll
  for (int k = 0; k < K; k++) {
    const int ex = basis_exp(k, 0), ey = basis_exp(k, 1), ez = basis_exp(k, 2);
    const float mv = px[ex] * py[ey] * pz[ez];
    const float4 cq = r4[k + 1];
    const float2 c01 = make_float2(cq.x, cq.y), c23 = make_float2(cq.z, cq.w);
    const float c4 = e4[k + 1];
    u01 = __ffma2_rn(c01, make_float2(mv, mv), u01);
    u23 = __ffma2_rn(c23, make_float2(mv, mv), u23);
    u4 = fmaf(c4, mv, u4);
    if (ex) {
      const float m = ex * px[ex > 0 ? ex - 1 : 0] * py[ey] * pz[ez];
      gx01 = __ffma2_rn(c01, make_float2(m, m), gx01);
      gx23 = __ffma2_rn(c23, make_float2(m, m), gx23);
      gx4 = fmaf(c4, m, gx4);
    }
    if (ey) {
      const float m = ey * px[ex] * py[ey > 0 ? ey - 1 : 0] * pz[ez];
      gy01 = __ffma2_rn(c01, make_float2(m, m), gy01);
      gy23 = __ffma2_rn(c23, make_float2(m, m), gy23);
      gy4 = fmaf(c4, m, gy4);
    }
    if (ez) {
      const float m = ez * px[ex] * py[ey] * pz[ez > 0 ? ez - 1 : 0];
      gz01 = __ffma2_rn(c01, make_float2(m, m), gz01);
      gz23 = __ffma2_rn(c23, make_float2(m, m), gz23);
      gz4 = fmaf(c4, m, gz4);
    }
  }
  const float u[5] = {u01.x, u01.y, u23.x, u23.y, u4};
  const float gx[5] = {gx01.x, gx01.y, gx23.x, gx23.y, gx4}, gy[5] = {gy01.x, gy01.y, gy23.x, gy23.y, gy4},
              gz[5] = {gz01.x, gz01.y, gz23.x, gz23.y, gz4};
#pragma unroll
  for (int v = 0; v < 5; v++) {
    U[v] = u[v];
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
__global__ void __launch_bounds__(kFaceThreads, 1) k_face_mx(FaceArgsMx a) {
  using T = FaceTileMx<ORDER>;
  constexpr int NQ = T::NQ, CS = T::CS, FB = T::FB;
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = a.stages, SF = T::stage_floats(a.nu);
  float* st = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(st + (size_t)S * SF);
  uint64_t* empty = full + kFaceMaxStages;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nbat = (a.F + FB - 1) / FB;
  const int mine = (int)blockIdx.x < nbat ? (nbat - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (t < S) {
    bar_init(&full[t], 33);  // the bulk copies' announcing arrival and the 32 lanes' row-copy arrivals
    bar_init(&empty[t], kFaceWarps);
  }
  __syncthreads();
  if (warp >= kFaceWarps) {
    // a copying warp: the next batch's distinct cells, loaded one batch ahead
    int cell[T::NUR];
    int cnt = 0;
    auto load_cells = [&](int k) {
      const size_t b = (size_t)blockIdx.x + (size_t)k * gridDim.x;
      cnt = __ldg(&a.bcount[b]);
#pragma unroll
      for (int r = 0; r < T::NUR; r++) {
        const int u = lane + 32 * r;
        cell[r] = u < cnt ? __ldg(&a.bcell[b * a.nu + u]) : 0;
      }
    };
    constexpr int PC = CS / 4;  // 16-byte pieces per row
    int sq[PC], pq[PC];
#pragma unroll
    for (int i = 0; i < PC; i++) {
      sq[i] = (32 * i + lane) / PC;
      pq[i] = (32 * i + lane) % PC;
    }
    const int w0 = warp - kFaceWarps;
    int k = w0;
    bool ok = true;
    if (k < mine) load_cells(k);
    for (; k < mine; k += kFaceCopyWarps) {
      const int s = k % S;
      if (k >= S && !bar_wait(&empty[s], (uint32_t)(k / S + 1) & 1u)) {  // batch k - S handed back
        ok = false;
        break;
      }
      const int f0 = ((int)blockIdx.x + k * (int)gridDim.x) * FB;
      float* sr = st + (size_t)s * SF;
      if (lane == 0) {
        bar_expect(&full[s], (uint32_t)(T::PTS + 2 * FB) * 4u);  // the rows arrive through the lanes' arrivals
        bulk_load(sr, a.fq + (size_t)f0 * NQ * 10, T::PTS * 4, &full[s]);
        bulk_load(sr + T::PTS, a.fpen + f0, FB * 4, &full[s]);
        bulk_load(sr + T::PTS + FB, a.fslot + f0, FB * 4, &full[s]);
      }
      // the rows in 16-byte pieces: slots 32 r .. 32 r + 31 are PC x 32 pieces,
      // piece 32 i + lane being piece pq[i] of slot 32 r + sq[i] (consecutive
      // pieces on consecutive lanes); the slot's cell comes from its lane
      float4* dst = reinterpret_cast<float4*>(sr + T::PTS + 2 * FB);
      const float4* src = reinterpret_cast<const float4*>(a.coef);
#pragma unroll
      for (int r = 0; r < T::NUR; r++) {
        if (32 * r >= cnt) break;
#pragma unroll
        for (int i = 0; i < PC; i++) {
          const int c = __shfl_sync(0xffffffffu, cell[r], sq[i]);
          if (32 * r + sq[i] < cnt) async_copy16(dst + (32 * r + sq[i]) * PC + pq[i], src + (size_t)c * PC + pq[i]);
        }
      }
      async_copies_arrive(&full[s]);
      if (k + kFaceCopyWarps < mine) load_cells(k + kFaceCopyWarps);
    }
    if (!ok && lane == 0) atomicOr(a.err, 2);
    // the copies this warp started into the stages' last batches land before
    // the block's shared memory is released (after a give-up: the batches
    // before the one it gave up on)
    const int hi = ok ? mine : k;
    if (lane == 0)
      for (int kk = max(hi - S, 0); kk < hi; kk++)
        if ((kk - w0) % kFaceCopyWarps == 0) bar_wait(&full[kk % S], (uint32_t)(kk / S) & 1u);
    return;
  }
  // this thread's face j of the batch and point q: warp w takes faces
  // w FPW .. w FPW + FPW - 1 (lanes past them compute a copy of the first and
  // write nothing)
  constexpr int FPW = T::FPW;
  const int grp = lane / NQ, in_grp = grp < FPW;
  const int j = warp * FPW + (in_grp ? grp : 0), q = in_grp ? lane - NQ * grp : 0;
  for (int k = 0; k < mine; k++) {
    const int s = k % S;
    const bool ok = __all_sync(0xffffffffu, bar_wait(&full[s], (uint32_t)(k / S) & 1u));
    if (!ok) {
      if (lane == 0) atomicOr(a.err, 2);
      return;
    }
    const int f = ((int)blockIdx.x + k * (int)gridDim.x) * FB + j;
    const float* sr = st + (size_t)s * SF;
    // the point's 10 floats: five 8-byte loads
    const float2* fq = reinterpret_cast<const float2*>(sr + (j * NQ + q) * 10);
    const float2 q0 = fq[0], q1 = fq[1], q2 = fq[2], q3 = fq[3], q4 = fq[4];
    const float n[3] = {q3.x, q3.y, q4.x};
    const float area = q4.y;
    const int slots = reinterpret_cast<const int*>(sr + T::PTS + FB)[j];
    const float* rows = sr + T::PTS + 2 * FB;
    float WL[5], WR[5], gs[5][3];  // gs = grad U_L + grad U_R
    if constexpr (ORDER <= 2) {
      eval_side_mx<ORDER, false>(rows + (slots & 0xffff) * CS, q0.x, q0.y, q1.x, WL, gs);
      eval_side_mx<ORDER, true>(rows + (slots >> 16) * CS, q1.y, q2.x, q2.y, WR, gs);
    } else {
      eval_side_ho_mx<ORDER, false>(rows + (slots & 0xffff) * CS, q0.x, q0.y, q1.x, WL, gs);
      eval_side_ho_mx<ORDER, true>(rows + (slots >> 16) * CS, q1.y, q2.x, q2.y, WR, gs);
    }
    const float pen2 = 2.f * sr[T::PTS + j];
    __syncwarp();
    if (lane == 0) bar_arrive(&empty[s]);  // this warp is done reading the stage
    float Fc[5];
    hllc_flux_mx(WL, WR, n, a.c, Fc);
    float flux[5];
    if (VISC) {
      // twice the penalised face gradient, 2 alpha/L [U] n + (grad U_L + grad U_R):
      // the viscous flux is linear in the gradient and scaling by 2 is exact, so
      // the flux of this gradient is exactly 2 F_v (and the halving of grad U_L +
      // grad U_R drops out)
      float Wf[5], gf2[5][3];
#pragma unroll
      for (int v = 0; v < 5; v++) {
        const float jump2 = pen2 * (WR[v] - WL[v]);
        Wf[v] = 0.5f * (WL[v] + WR[v]);
#pragma unroll
        for (int d = 0; d < 3; d++) gf2[v][d] = fmaf(jump2, n[d], gs[v][d]);
      }
      float Fv2[5];
      viscous_flux_mx(Wf, gf2, n, a.c, Fv2);
#pragma unroll
      for (int v = 0; v < 5; v++) flux[v] = fmaf(-0.5f, Fv2[v], Fc[v]) * area;
    } else {
#pragma unroll
      for (int v = 0; v < 5; v++) flux[v] = Fc[v] * area;
    }
    if constexpr ((NQ & (NQ - 1)) == 0) {  // groups of 1, 4 or 16 lanes: a butterfly
#pragma unroll
      for (int off = 1; off < NQ; off <<= 1)
#pragma unroll
        for (int v = 0; v < 5; v++) flux[v] += __shfl_xor_sync(0xffffffffu, flux[v], off);
    } else {  // 9 lanes: a fixed tree onto the group's first lane
#pragma unroll
      for (int off = 8; off >= 1; off >>= 1)
#pragma unroll
        for (int v = 0; v < 5; v++) {
          const float o = __shfl_down_sync(0xffffffffu, flux[v], off);
          if (q + off < NQ) flux[v] += o;
        }
    }
    if (in_grp && f < a.F && q == 0) {
#pragma unroll
      for (int v = 0; v < 5; v++) a.G[(size_t)v * a.F + f] = flux[v];
    }
  }
}

// diagnostics partial sums from FP32 coefficients (FP64 accumulation)
__global__ void __launch_bounds__(kRedThreads)
    k_diag_partial_mx(const double* __restrict__ U, const float* __restrict__ coef, int cs,
                      int ncf /* entries per variable, K + 1 */, const double* __restrict__ vol, int N,
                      double* __restrict__ part) {
  __shared__ double sm[4][kRedThreads];
  double acc[4] = {0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double r = U[i], ir = 1.0 / r;
    const double u[3] = {U[(size_t)N + i] * ir, U[2 * (size_t)N + i] * ir, U[3 * (size_t)N + i] * ir};
    double g[4][3];  // physical-unit linear coefficients = gradient at the centroid
#pragma unroll
    for (int v = 0; v < 4; v++)
#pragma unroll
      for (int j = 0; j < 3; j++) g[v][j] = (double)coef[(size_t)i * cs + cidx(v, j + 1, ncf)];
    double gu[3][3];
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
      for (int j = 0; j < 3; j++) gu[q][j] = (g[1 + q][j] - u[q] * g[0][j]) * ir;
    const double wx = gu[2][1] - gu[1][2], wy = gu[0][2] - gu[2][0], wz = gu[1][0] - gu[0][1];
    const double dv = gu[0][0] + gu[1][1] + gu[2][2];
    const double V = vol[i];
    acc[0] += V * 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    acc[1] += V * (wx * wx + wy * wy + wz * wz);
    acc[2] += V * dv * dv;
    acc[3] += V;
  }
#pragma unroll
  for (int q = 0; q < 4; q++) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int q = 0; q < 4; q++) sm[q][threadIdx.x] += sm[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < 4; q++) part[(size_t)blockIdx.x * 4 + q] = sm[q][0];
}

}  // namespace ucns
