// C ABI entry points of libucns (declared in include/ucns.h): argument
// checks, device upload of the precompute, and kernel launches on the
// caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "host_arrays.hpp"
#include "kernels.cuh"
#include "kernels_mixed.cuh"
#include "kernels_gate.cuh"
#include "kernels_ho.cuh"
#include "mlp_internal.hpp"
#include "ucns_internal.hpp"

namespace ucns {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

#define UCNS_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(UCNS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

namespace {

template <typename T>
int upload(T** dst, const std::vector<T>& src) {
  if (src.empty()) return UCNS_OK;
  if (cudaMalloc((void**)dst, src.size() * sizeof(T)) != cudaSuccess)
    return fail(UCNS_ERR_NOMEM, "cudaMalloc failed during precompute upload");
  UCNS_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return UCNS_OK;
}

int upload_f32(float** dst, const std::vector<double>& src, size_t npad = 0) {
  std::vector<float> f(src.begin(), src.end());
  if (f.size() < npad) f.resize(npad, 0.f);
  return upload(dst, f);
}

// [rows][N] -> cell-contiguous [N][rows], converted to T
template <typename T, typename S>
int upload_cellwise(T** dst, const std::vector<S>& src, int rows, int64_t N, int64_t Npad = 0) {
  if (src.empty()) return UCNS_OK;
  std::vector<T> b((size_t)std::max(N, Npad) * rows, T(0));
  for (int r = 0; r < rows; r++)
    for (int64_t i = 0; i < N; i++) b[(size_t)i * rows + r] = (T)src[(size_t)r * N + i];
  return upload(dst, b);
}

// [rows][N] -> blocked [ceil(N/kTC)][rows][kTC] (pair = false) or
// pair-blocked [ceil(N/kTC)][rows/2][kTC][2] (pair = true, rows even), zero
// past N, converted to T
template <typename T, typename S>
int upload_blocked(T** dst, const std::vector<S>& src, int rows, int64_t N, bool pair) {
  if (src.empty()) return UCNS_OK;
  if (pair && rows % 2) return fail(UCNS_ERR_INVALID_ARG, "pair-blocked layout needs an even row count");
  const int64_t tiles = (N + kTC - 1) / kTC;
  std::vector<T> b((size_t)tiles * rows * kTC, T(0));
  for (int r = 0; r < rows; r++)
    for (int64_t i = 0; i < N; i++) b[pair ? blk2(r, rows, i) : blk(r, rows, i)] = (T)src[(size_t)r * N + i];
  return upload(dst, b);
}

template <typename T>
int alloc(T** dst, size_t n) {
  if (cudaMalloc((void**)dst, n * sizeof(T)) != cudaSuccess)
    return fail(UCNS_ERR_NOMEM, "cudaMalloc failed for library scratch");
  return UCNS_OK;
}

inline unsigned nblocks(size_t threads, int bs = 256) { return (unsigned)((threads + bs - 1) / bs); }

enum {
  kKindRecon = 0,
  kKindFace = 1,
  kKindRK = 2,
  kKindDt = 3,
  kKindDiag = 4,
  kKindOther = 5,
  kKindFeatures = 6,
  kKindMlp = 7,
  kKinds = 8
};

cudaEvent_t take_event(ucns_mesh* m) {
  if (!m->prof_pool.empty()) {
    void* e = m->prof_pool.back();
    m->prof_pool.pop_back();
    return (cudaEvent_t)e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Runs `launch` (which enqueues kernels on s) between two recorded events
// when the mesh's timing window is open.
template <class Fn>
int timed(ucns_mesh* m, int kind, cudaStream_t s, Fn&& launch) {
  if (!m->prof) return launch();
  cudaEvent_t a = take_event(m), b = take_event(m);
  cudaEventRecord(a, s);
  int rc = launch();
  cudaEventRecord(b, s);
  m->prof_live.push_back({kind, (void*)a, (void*)b});
  return rc;
}

FluxConst flux_const(const ucns_params& p) {
  FluxConst c;
  c.gam = p.gamma;
  c.gm1 = p.gamma - 1.0;
  const double Rg = 1.0 / (p.gamma * p.mach * p.mach);
  const bool visc = p.reynolds > 0.0;
  c.mu = visc ? 1.0 / p.reynolds : 0.0;
  const double cp = p.gamma * Rg / (p.gamma - 1.0);
  c.kap = visc ? c.mu * cp / p.prandtl : 0.0;
  c.gm1_over_R = (p.gamma - 1.0) / Rg;
  return c;
}

FluxConstF flux_const_f(const ucns_params& p) {
  const FluxConst d = flux_const(p);
  FluxConstF c;
  c.gam = (float)d.gam;
  c.gm1 = (float)d.gm1;
  c.mu = (float)d.mu;
  c.kap = (float)d.kap;
  c.gm1_over_R = (float)d.gm1_over_R;
  const double p_ref = 1.0 / (p.gamma * p.mach * p.mach);
  c.p_ref = (float)p_ref;
  c.H_ref = (float)(p.gamma * p_ref / (p.gamma - 1.0));
  return c;
}

bool mixed(const ucns_mesh* m) { return m->P.precision == UCNS_PREC_MIXED; }

// floats per cell row of the mixed-form coefficients: 5 (K+1) rounded up to 4
int coef_row_floats(const ucns_mesh* m) { return (5 * m->NC + 3) / 4 * 4; }

template <int ORDER, bool WENO, int ND, bool GATED = false>
int launch_recon_tiles(const ReconArgsMx& a, cudaStream_t s) {
  constexpr size_t sm = ReconTile<ORDER, WENO, ND>::smem();
  if (a.cs != ReconTile<ORDER, WENO, ND>::CS) return fail(UCNS_ERR_INVALID_ARG, "coefficient row size mismatch");
  UCNS_CUDA(cudaFuncSetAttribute(k_recon_mx<ORDER, WENO, ND, GATED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm));
  const unsigned tiles = (unsigned)((a.N + kTC - 1) / kTC);
  k_recon_mx<ORDER, WENO, ND, GATED><<<tiles, kTC * 5, sm, s>>>(a);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

// P3 / P4, mixed form
template <int ORDER, bool WENO>
int launch_recon_ho_tiles(const ReconArgsHOMx& a, cudaStream_t s) {
  using T = HOTile<ORDER>;
  constexpr size_t sm = T::smem();
  UCNS_CUDA(cudaFuncSetAttribute(k_recon_ho_mx<ORDER, WENO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const unsigned g = (unsigned)((a.N + T::TC - 1) / T::TC);
  k_recon_ho_mx<ORDER, WENO><<<g, T::THREADS, sm, s>>>(a);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int launch_recon_ho_mx(ucns_mesh* m, cudaStream_t s) {
  ReconArgsHOMx a;
  a.Uhl = m->d.Uhl;
  a.tiles = m->d.hot;
  a.Msi = m->d.Msif;
  a.psib = m->d.psibf;
  a.inv_h = m->d.inv_hf;
  a.coef = m->d.coeff;
  a.cs = coef_row_floats(m);
  a.err = m->d.err;
  a.N = (int)m->N;
  const double lsum = m->P.lambda_central + m->nd;
  a.lam0 = (float)(m->P.lambda_central / lsum);
  a.lams = (float)(1.0 / lsum);
  a.eps = (float)m->P.epsilon;
  const double eref = 1.0 / (m->P.gamma * m->P.mach * m->P.mach) / (m->P.gamma - 1.0);
  a.eref_hi = (float)eref;
  a.eref_lo = (float)(eref - (double)a.eref_hi);
  const bool weno = m->nd > 0;
  if (m->K == 19) return weno ? launch_recon_ho_tiles<3, true>(a, s) : launch_recon_ho_tiles<3, false>(a, s);
  return weno ? launch_recon_ho_tiles<4, true>(a, s) : launch_recon_ho_tiles<4, false>(a, s);
}

// the P3/P4 mixed reconstruction's tiles (HOTile): stencil ids, FP32
// pseudo-inverse entries and (CWENOZ) smoothness matrices, zero past N
template <int ORDER>
int upload_ho_tiles(const ucns_mesh* m, const HostArrays& h, bool weno, float** dst) {
  using T = HOTile<ORDER>;
  constexpr int TC = T::TC, K = T::K, MC = T::MC, KD = T::KD, MD = T::MD;
  const int64_t N = m->N, tiles = (N + TC - 1) / TC;
  const int TF = T::tile_floats(weno);
  std::vector<float> b((size_t)tiles * TF, 0.f);
  auto put_id = [](float* at, int32_t id) { std::memcpy(at, &id, 4); };
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < tiles; t++) {
    float* base = b.data() + (size_t)t * TF;
    for (int c = 0; c < TC; c++) {
      const int64_t i = t * TC + c;
      if (i >= N) break;
      for (int ch = 0; ch < T::NCC; ch++) {
        float* chunk = base + (size_t)ch * T::CCS;
        for (int mm = 0; mm < T::MCH; mm++) {
          const int mg = ch * T::MCH + mm;
          put_id(chunk + mm * TC + c, h.sc[(size_t)mg * N + i]);
          for (int k = 0; k < K; k++)
            chunk[T::MCH * TC + ((k * (T::MCH / 2) + mm / 2) * TC + c) * 2 + (mm & 1)] =
                (float)h.Pc[((size_t)k * MC + mg) * N + i];
        }
      }
      if (!weno) continue;
      for (int q = 0; q < T::NQS; q++) base[T::CENTRAL + (size_t)q * TC + c] = (float)h.Msi[(size_t)q * N + i];
      for (int sd = 0; sd < 6; sd++)
        for (int hh = 0; hh < T::NDC; hh++) {
          float* chunk = base + T::CENTRAL + T::SMAT + (size_t)(sd * T::NDC + hh) * T::DCS;
          for (int rr = 0; rr < T::MDH; rr++) {
            const int r = hh * T::MDH + rr;
            put_id(chunk + rr * TC + c, h.sd[((size_t)sd * MD + r) * N + i]);
            for (int k = 0; k < KD; k++)
              chunk[T::MDH * TC + ((k * (T::MDH / 2) + rr / 2) * TC + c) * 2 + (rr & 1)] =
                  (float)h.Pd[(((size_t)sd * KD + k) * MD + r) * N + i];
          }
        }
    }
  }
  return upload(dst, b);
}

int launch_recon_mx(ucns_mesh* m, const double* U, cudaStream_t s) {
  if (m->K > 9) return launch_recon_ho_mx(m, s);
  ReconArgsMx a;
  (void)U;  // read through its float pair m->d.Uhl, written by k_split or the RK stage
  a.Uhl = m->d.Uhl;
  a.sc = m->d.scb;
  a.Pc = m->d.Pcb;
  a.sd = m->d.sdb;
  a.Pd = m->d.Pdb;
  a.cell = m->d.cellb;
  a.coef = m->d.coeff;
  a.gate = m->gate_flag;
  a.sda = m->d.sda;
  a.Pda = m->d.Pda;
  a.err = m->d.err;
  a.N = (int)m->N;
  a.cs = coef_row_floats(m);
  const double lsum = m->P.lambda_central + m->nd;
  a.lam0 = (float)(m->P.lambda_central / lsum);
  a.lams = (float)(1.0 / lsum);
  a.eps = (float)m->P.epsilon;
  const double eref = 1.0 / (m->P.gamma * m->P.mach * m->P.mach) / (m->P.gamma - 1.0);
  a.eref_hi = (float)eref;
  a.eref_lo = (float)(eref - (double)a.eref_hi);
  const bool gated = m->gate_eval_active;
  if (m->K == 3) return launch_recon_tiles<1, false, 6>(a, s);
  if (m->nd == 0) return launch_recon_tiles<2, false, 6>(a, s);
  if (m->nd == 6) return gated ? launch_recon_tiles<2, false, 6, true>(a, s) : launch_recon_tiles<2, true, 6>(a, s);
  return gated ? launch_recon_tiles<2, false, 4, true>(a, s) : launch_recon_tiles<2, true, 4>(a, s);
}

// persistent blocks (as many as fit at once, at most one per batch), as many
// pipeline stages as the shared memory holds
template <int ORDER, bool VISC>
int launch_face_tiles(FaceArgsMx a, cudaStream_t s) {
  using T = FaceTileMx<ORDER>;
  if (a.cs != T::CS) return fail(UCNS_ERR_INVALID_ARG, "coefficient row size mismatch");
  int dev = 0, sms = 0, optin = 0, per_sm = 0;
  UCNS_CUDA(cudaGetDevice(&dev));
  UCNS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  UCNS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  a.stages = kFaceMaxStages;
  while (a.stages > 2 && T::smem(a.nu, a.stages) > (size_t)optin) a.stages--;
  const size_t sm = T::smem(a.nu, a.stages);
  if (sm > (size_t)optin) return fail(UCNS_ERR_INVALID_ARG, "face batch rows exceed shared memory");
  UCNS_CUDA(cudaFuncSetAttribute(k_face_mx<ORDER, VISC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  UCNS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_face_mx<ORDER, VISC>, kFaceThreads, sm));
  const int64_t batches = ((int64_t)a.F + T::FB - 1) / T::FB;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(batches, (int64_t)sms * std::max(per_sm, 1)));
  k_face_mx<ORDER, VISC><<<g, kFaceThreads, sm, s>>>(a);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int launch_face_mx(ucns_mesh* m, cudaStream_t s) {
  FaceArgsMx a;
  a.coef = m->d.coeff;
  a.fq = m->d.fqf;
  a.fpen = m->d.fpenf;
  a.G = reinterpret_cast<float*>(m->d.G);  // FP32 totals in the first half
  a.fslot = m->d.fslot;
  a.bcell = m->d.bcell;
  a.bcount = m->d.bcount;
  a.err = m->d.err;
  a.N = (int)m->N;
  a.F = (int)m->F;
  a.cs = coef_row_floats(m);
  a.nu = m->d.fnu;
  a.stages = 2;
  a.c = flux_const_f(m->P);
  const bool visc = m->P.reynolds > 0.0;
  switch (m->K) {
    case 3: return visc ? launch_face_tiles<1, true>(a, s) : launch_face_tiles<1, false>(a, s);
    case 9: return visc ? launch_face_tiles<2, true>(a, s) : launch_face_tiles<2, false>(a, s);
    case 19: return visc ? launch_face_tiles<3, true>(a, s) : launch_face_tiles<3, false>(a, s);
    default: return visc ? launch_face_tiles<4, true>(a, s) : launch_face_tiles<4, false>(a, s);
  }
}

// P3 / P4 (FP64, hexahedra)
int launch_recon_ho(ucns_mesh* m, const double* U, cudaStream_t s) {
  ReconArgsHO a;
  a.U = U;
  a.sc = m->d.sc;
  a.Pc = m->d.Pc;
  a.sd = m->d.sd;
  a.Pd = m->d.Pd;
  a.Msi = m->d.Msi;
  a.psib = m->d.psib;
  a.inv_h = m->d.inv_h;
  a.coef = m->d.coef;
  a.N = (int)m->N;
  const double lsum = m->P.lambda_central + m->nd;
  a.lam0 = m->P.lambda_central / lsum;
  a.lams = 1.0 / lsum;
  a.eps = m->P.epsilon;
  const unsigned g = nblocks((size_t)m->N * 5, 128);
  const bool weno = m->nd > 0;
  if (m->K == 19) {
    if (weno) k_recon_ho<3, true><<<g, 128, 0, s>>>(a);
    else k_recon_ho<3, false><<<g, 128, 0, s>>>(a);
  } else {
    if (weno) k_recon_ho<4, true><<<g, 128, 0, s>>>(a);
    else k_recon_ho<4, false><<<g, 128, 0, s>>>(a);
  }
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int launch_face_ho(ucns_mesh* m, cudaStream_t s) {
  FaceArgs a;
  a.coef = m->d.coef;
  a.fq = m->d.fq;
  a.fpen = m->d.fpen;
  a.fo = m->d.fo;
  a.fn = m->d.fn;
  a.inv_h = m->d.inv_h;
  a.G = m->d.G;
  a.N = (int)m->N;
  a.F = (int)m->F;
  a.c = flux_const(m->P);
  const bool visc = m->P.reynolds > 0.0;
  const int fpw = 32 / m->nq;  // faces per warp
  const size_t threads = (size_t)((m->F + fpw - 1) / fpw) * 32;
  const unsigned g = nblocks(threads, 128);
  if (m->K == 19) {
    if (visc) k_face_ho<3, true><<<g, 128, 0, s>>>(a);
    else k_face_ho<3, false><<<g, 128, 0, s>>>(a);
  } else {
    if (visc) k_face_ho<4, true><<<g, 128, 0, s>>>(a);
    else k_face_ho<4, false><<<g, 128, 0, s>>>(a);
  }
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int launch_recon_raw(ucns_mesh* m, const double* U, cudaStream_t s) {
  if (mixed(m)) return launch_recon_mx(m, U, s);
  if (m->K > 9) return launch_recon_ho(m, U, s);
  ReconArgs a;
  a.U = U;
  a.sc = m->d.sc;
  a.Pc = m->d.Pc;
  a.sd = m->d.sd;
  a.Pd = m->d.Pd;
  a.mom = m->d.mom;
  a.inv_h = m->d.inv_h;
  a.coef = m->d.coef;
  a.gate = m->gate_eval_active ? m->gate_flag : nullptr;
  a.dev = m->label_out;
  a.dvalid = m->d.dvalid;
  a.N = (int)m->N;
  const double lsum = m->P.lambda_central + m->nd;
  a.lam0 = m->P.lambda_central / lsum;
  a.lams = 1.0 / lsum;
  a.lamc = m->P.lambda_central;
  a.eps = m->P.epsilon;
  const unsigned g = nblocks((size_t)m->N * 5);
  const bool gated = a.gate != nullptr;
  const bool walls = m->n_boundary > 0;
  if (m->K == 3)
    k_recon<1, false, 6, false><<<g, 256, 0, s>>>(a);
  else if (m->nd == 0)
    k_recon<2, false, 6, false><<<g, 256, 0, s>>>(a);
  else if (walls && m->nd == 6)
    k_recon<2, true, 6, false, true><<<g, 256, 0, s>>>(a);
  else if (walls && m->nd == 5)
    k_recon<2, true, 5, false, true><<<g, 256, 0, s>>>(a);
  else if (walls)
    k_recon<2, true, 4, false, true><<<g, 256, 0, s>>>(a);
  else if (m->nd == 5)
    k_recon<2, true, 5, false><<<g, 256, 0, s>>>(a);
  else if (m->nd == 6 && gated)
    k_recon<2, true, 6, true><<<g, 256, 0, s>>>(a);
  else if (m->nd == 6)
    k_recon<2, true, 6, false><<<g, 256, 0, s>>>(a);
  else if (gated)
    k_recon<2, true, 4, true><<<g, 256, 0, s>>>(a);
  else
    k_recon<2, true, 4, false><<<g, 256, 0, s>>>(a);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int launch_face_raw(ucns_mesh* m, cudaStream_t s) {
  if (mixed(m)) return launch_face_mx(m, s);
  if (m->K > 9) return launch_face_ho(m, s);
  FaceArgs a;
  a.coef = m->d.coef;
  a.fq = m->d.fq;
  a.fpen = m->d.fpen;
  a.fo = m->d.fo;
  a.fn = m->d.fn;
  a.inv_h = m->d.inv_h;
  a.G = m->d.G;
  a.N = (int)m->N;
  a.F = (int)m->F;
  a.c = flux_const(m->P);
  for (int v = 0; v < 5; v++) a.uinf[v] = m->uinf[v];
  const bool visc = m->P.reynolds > 0.0;
  const unsigned g = nblocks((size_t)m->F * m->nq);
  if (m->n_boundary > 0) {  // inviscid (checked at precompute)
    if (m->K == 3) k_face<1, false, true><<<g, 256, 0, s>>>(a);
    else k_face<2, false, true><<<g, 256, 0, s>>>(a);
  } else if (m->K == 3) {
    if (visc) k_face<1, true><<<g, 256, 0, s>>>(a);
    else k_face<1, false><<<g, 256, 0, s>>>(a);
  } else {
    if (visc) k_face<2, true><<<g, 256, 0, s>>>(a);
    else k_face<2, false><<<g, 256, 0, s>>>(a);
  }
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int launch_rk_raw(ucns_mesh* m, int stage, const double* U0, const double* Us, double* out,
                  cudaStream_t s, bool keep_pair = false) {
  RKArgs a;
  a.U0 = U0;
  a.Us = Us;
  a.out = out;
  a.G = m->d.G;
  a.cf = m->d.cf;
  a.inv_vol = m->d.inv_vol;
  a.dt = m->d.dt;
  a.err = m->d.err;
  // the next stage (or, keep_pair, the next step) reconstructs out from its float pair
  a.hl = (mixed(m) && (stage == 1 || stage == 2 || (stage == 3 && keep_pair))) ? m->d.Uhl : nullptr;
  a.acc = nullptr;
  a.N = (int)m->N;
  a.F = (int)m->F;
  a.gm1 = m->P.gamma - 1.0;
  const unsigned g = nblocks((size_t)m->N);
#define UCNS_RK(ST)                                                           \
  do {                                                                        \
    if (mixed(m)) {                                                           \
      if (m->nfc == 6) k_rk<ST, 6, float><<<g, 256, 0, s>>>(a);               \
      else k_rk<ST, 4, float><<<g, 256, 0, s>>>(a);                           \
    } else {                                                                  \
      if (m->nfc == 6) k_rk<ST, 6, double><<<g, 256, 0, s>>>(a);              \
      else if (m->nfc == 5) k_rk<ST, 5, double><<<g, 256, 0, s>>>(a);         \
      else k_rk<ST, 4, double><<<g, 256, 0, s>>>(a);                          \
    }                                                                         \
  } while (0)
  switch (stage) {
    case 0: UCNS_RK(0); break;
    case 1: UCNS_RK(1); break;
    case 2: UCNS_RK(2); break;
    default: UCNS_RK(3); break;
  }
#undef UCNS_RK
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

// stage 1..5 of SSP(5,4) (k_rk54): U0 = U^n, Us = the stage's input, out = its result
int launch_rk54_raw(ucns_mesh* m, int stage, const double* U0, const double* Us, double* out, cudaStream_t s,
                    bool keep_pair = false) {
  RKArgs a;
  a.U0 = U0;
  a.Us = Us;
  a.out = out;
  a.G = m->d.G;
  a.cf = m->d.cf;
  a.inv_vol = m->d.inv_vol;
  a.dt = m->d.dt;
  a.err = m->d.err;
  a.hl = (mixed(m) && (stage < 5 || keep_pair)) ? m->d.Uhl : nullptr;
  a.acc = m->d.Uacc;
  a.N = (int)m->N;
  a.F = (int)m->F;
  a.gm1 = m->P.gamma - 1.0;
  const unsigned g = nblocks((size_t)m->N);
#define UCNS_RK54(ST)                                                         \
  do {                                                                        \
    if (mixed(m)) {                                                           \
      if (m->nfc == 6) k_rk54<ST, 6, float><<<g, 256, 0, s>>>(a);             \
      else k_rk54<ST, 4, float><<<g, 256, 0, s>>>(a);                         \
    } else {                                                                  \
      if (m->nfc == 6) k_rk54<ST, 6, double><<<g, 256, 0, s>>>(a);            \
      else if (m->nfc == 5) k_rk54<ST, 5, double><<<g, 256, 0, s>>>(a);       \
      else k_rk54<ST, 4, double><<<g, 256, 0, s>>>(a);                        \
    }                                                                         \
  } while (0)
  switch (stage) {
    case 1: UCNS_RK54(1); break;
    case 2: UCNS_RK54(2); break;
    case 3: UCNS_RK54(3); break;
    case 4: UCNS_RK54(4); break;
    default: UCNS_RK54(5); break;
  }
#undef UCNS_RK54
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

// the CFL time step of U into out[0] (device), partial minima in m->d.red
int launch_dt_to(ucns_mesh* m, const double* U, double* out, cudaStream_t s) {
  const ucns_params& p = m->P;
  const double vc = p.reynolds > 0.0 ? p.prandtl / (2.0 * p.gamma * (1.0 / p.reynolds)) : 0.0;
  k_dt_partial<<<m->d.red_blocks, kRedThreads, 0, s>>>(U, m->d.dtlen, (int)m->N, p.gamma, vc, m->d.red, m->d.err);
  k_dt_final<<<1, kRedThreads, 0, s>>>(m->d.red, m->d.red_blocks, p.cfl, out);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int launch_dt_raw(ucns_mesh* m, const double* U, cudaStream_t s) {
  const ucns_params& p = m->P;
  const double vc = p.reynolds > 0.0 ? p.prandtl / (2.0 * p.gamma * (1.0 / p.reynolds)) : 0.0;
  k_dt_partial<<<m->d.red_blocks, kRedThreads, 0, s>>>(U, m->d.dtlen, (int)m->N, p.gamma, vc,
                                                        m->d.red, m->d.err);
  k_dt_final<<<1, kRedThreads, 0, s>>>(m->d.red, m->d.red_blocks, p.cfl, m->d.dt);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

// The CFL time step of U into m->d.dt at the start of a Runge-Kutta step, on
// the mesh's side stream: it waits for U on s, and s waits for it (join_dt)
// only before the first use of dt (the first RK stage), so the reduction
// overlaps the float pair, the gate and the first reconstruction.
int launch_dt_async(ucns_mesh* m, const double* U, cudaStream_t s) {
  if (!m->aux) {
    cudaStream_t st;
    cudaEvent_t e1, e2;
    UCNS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    m->aux = (void*)st;
    UCNS_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
    m->ev_u = (void*)e1;
    UCNS_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    m->ev_dt = (void*)e2;
  }
  cudaStream_t aux = (cudaStream_t)m->aux;
  UCNS_CUDA(cudaEventRecord((cudaEvent_t)m->ev_u, s));
  UCNS_CUDA(cudaStreamWaitEvent(aux, (cudaEvent_t)m->ev_u, 0));
  const ucns_params& p = m->P;
  DtArgs a;
  a.U = U;
  a.dtlen = m->d.dtlen;
  a.part = m->d.dt_part;
  a.count = m->d.dt_count;
  a.dt = m->d.dt;
  a.err = m->d.err;
  a.N = (int)m->N;
  a.gam = p.gamma;
  a.visc = p.reynolds > 0.0 ? p.prandtl / (2.0 * p.gamma * (1.0 / p.reynolds)) : 0.0;
  a.cfl = p.cfl;
  int rc = timed(m, kKindDt, aux, [&] {
    k_dt_fused<<<nblocks((size_t)m->N), kRedThreads, 0, aux>>>(a);
    UCNS_CUDA(cudaGetLastError());
    return UCNS_OK;
  });
  if (rc) return rc;
  UCNS_CUDA(cudaEventRecord((cudaEvent_t)m->ev_dt, aux));
  return UCNS_OK;
}
int join_dt(ucns_mesh* m, cudaStream_t s) {
  UCNS_CUDA(cudaStreamWaitEvent(s, (cudaEvent_t)m->ev_dt, 0));
  return UCNS_OK;
}

int launch_recon(ucns_mesh* m, const double* U, cudaStream_t s) {
  return timed(m, kKindRecon, s, [&] { return launch_recon_raw(m, U, s); });
}
// float pair of a caller state before a mixed reconstruction of it
int launch_split_raw(ucns_mesh* m, const double* U, cudaStream_t s) {
  k_split<<<nblocks((size_t)5 * m->N), 256, 0, s>>>(U, m->d.Uhl, (int)m->N);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}
int launch_split(ucns_mesh* m, const double* U, cudaStream_t s) {
  if (!mixed(m)) return UCNS_OK;
  return timed(m, kKindOther, s, [&] { return launch_split_raw(m, U, s); });
}
int launch_face(ucns_mesh* m, cudaStream_t s) {
  return timed(m, kKindFace, s, [&] { return launch_face_raw(m, s); });
}
int launch_rk(ucns_mesh* m, int stage, const double* U0, const double* Us, double* out, cudaStream_t s,
              bool keep_pair = false) {
  return timed(m, kKindRK, s, [&] { return launch_rk_raw(m, stage, U0, Us, out, s, keep_pair); });
}
int launch_dt(ucns_mesh* m, const double* U, cudaStream_t s) {
  return timed(m, kKindDt, s, [&] { return launch_dt_raw(m, U, s); });
}
int launch_rk54(ucns_mesh* m, int stage, const double* U0, const double* Us, double* out, cudaStream_t s,
                bool keep_pair = false) {
  return timed(m, kKindRK, s, [&] { return launch_rk54_raw(m, stage, U0, Us, out, s, keep_pair); });
}

// the indicator features of U into X (BF16) and Xf (FP32, or null); the
// mixed form reads U through its float pair, split here
int launch_features(ucns_mesh* m, const double* U, void* X, float* Xf, cudaStream_t s, bool split = true) {
  FeatArgs a;
  a.U = U;
  a.Uhl = m->d.Uhl;
  a.sc = mixed(m) ? m->d.scb : m->d.sc;
  a.Pc = mixed(m) ? (const void*)m->d.Pcb : (const void*)m->d.Pc;
  a.mom = m->d.mom;
  a.inv_h = m->d.inv_h;
  a.cell = m->d.cellb;
  a.X = reinterpret_cast<__nv_bfloat16*>(X);
  a.Xf = Xf;
  a.N = (int)m->N;
  a.gam = (float)m->P.gamma;
  if (mixed(m)) {
    int rc = split ? launch_split_raw(m, U, s) : UCNS_OK;
    if (rc) return rc;
    k_features_mx<<<nblocks((size_t)m->N, 128), 128, 0, s>>>(a);
  } else {
    k_features<<<nblocks((size_t)m->N, 128), 128, 0, s>>>(a);
  }
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

// features of U and the network's flags, once per call of the solver; for the
// mixed form this leaves the float pair of U in m->d.Uhl
int gate_eval(ucns_mesh* m, const double* U, cudaStream_t s, bool* split_done = nullptr) {
  m->gate_eval_active = false;
  if (m->gate_fixed) {  // the caller's flags stand in for the network's
    m->gate_eval_active = true;
    return UCNS_OK;
  }
  if (!m->gate_on || !m->mlp) return UCNS_OK;
  const bool have_pair = split_done && *split_done;
  int rc = timed(m, kKindFeatures, s, [&] { return launch_features(m, U, m->gate_X, nullptr, s, !have_pair); });
  if (rc) return rc;
  if (split_done) *split_done = mixed(m);
  rc = timed(m, kKindMlp, s, [&] {
    return ucnsnet::forward(m->mlp, m->gate_X, m->N, nullptr, m->gate_flag, m->gate_thr, s);
  });
  if (rc) return rc;
  m->gate_eval_active = true;
  return UCNS_OK;
}

int check_ready(const ucns_mesh* m) {
  if (!m) return fail(UCNS_ERR_INVALID_ARG, "mesh handle is NULL");
  if (!m->precomputed) return fail(UCNS_ERR_STATE, "ucns_precompute has not been called");
  return UCNS_OK;
}

int residual_into(ucns_mesh* m, const double* U, double* R, cudaStream_t s) {
  int rc;
  if ((rc = launch_split(m, U, s)) || (rc = launch_recon(m, U, s)) || (rc = launch_face(m, s)) ||
      (rc = launch_rk(m, 0, U, U, R, s)))
    return rc;
  return UCNS_OK;
}

// Diagnostic sums [V KE, V |curl u|^2, V (div u)^2, V] of the coefficients
// the last reconstruction left, into out[0..3] (device)
int diag_sums_into(ucns_mesh* m, const double* U, double* out, cudaStream_t s) {
  if (mixed(m))
    k_diag_partial_mx<<<m->d.red_blocks, kRedThreads, 0, s>>>(U, m->d.coeff, coef_row_floats(m), m->NC, m->d.vol,
                                                             (int)m->N, m->d.red);
  else
    k_diag_partial<double><<<m->d.red_blocks, kRedThreads, 0, s>>>(U, m->d.coef, m->d.vol, (int)m->N, m->d.red);
  k_diag_final<<<1, 32, 0, s>>>(m->d.red, m->d.red_blocks, out);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

// The plain-scheme check of the gate on the state U: the gated and the full
// reconstruction and residual of U, and four measures of their difference:
//  rel[0]  |sum r_gated - sum r_full| / |sum r_full|, r_i = V_i (u . R_m -
//          |u|^2 R_rho / 2) the cells' kinetic-energy rates (the relative error
//          of dKE/dt; ill-conditioned where dKE/dt is near zero);
//  rel[1]  sum |r_gated - r_full| / sum |r_full| (local, cannot cancel);
//  rel[2]  the running estimate of the KE history's relative error: every
//          check adds |sum r_gated - sum r_full| / sum V, the difference of
//          the volume-averaged dKE/dt, times (steps until the next check) * dt
//          / KE, the drift of KE from the full scheme's over that interval to
//          first order;
//  rel[3]  |eps_s,gated - eps_s,full| / eps_s,full, the solenoidal
//          dissipation of the two reconstructions of U;
//  rel[4]  |eps_d,gated - eps_d,full| / max(eps_d,full, 1e-3 eps_s,full), the
//          dilatational one (measured against a thousandth of the solenoidal
//          one where it is smaller: at low Mach number it is below the
//          arithmetic's resolution of the dissipation).
// The gate goes off when rel[2], rel[3] or rel[4] exceeds the bound, or rel[0]
// exceeds the optional rate bound (> 0).  `steps` is the interval to the next
// check.
int gate_check(ucns_mesh* m, const double* U, double* rel, cudaStream_t s, int steps) {
  int rc;
  const size_t n5 = (size_t)5 * m->N;
  if (!m->gate_R && (rc = alloc(&m->gate_R, 2 * n5 + 16))) return rc;
  double* sums = m->gate_R + 2 * n5;  // [0..3] gated diagnostics, [4..7] full, [8..12] KE rates, [13] dt
  if ((rc = gate_eval(m, U, s)) || (rc = residual_into(m, U, m->gate_R, s))) return rc;
  rc = timed(m, kKindOther, s, [&] { return diag_sums_into(m, U, sums, s); });
  if (rc) return rc;
  m->gate_eval_active = false;
  if ((rc = residual_into(m, U, m->gate_R + n5, s))) return rc;
  rc = timed(m, kKindOther, s, [&] {
    int r = diag_sums_into(m, U, sums + 4, s);
    if (r) return r;
    k_ke_rate_partial<<<m->d.red_blocks, 256, 0, s>>>(U, m->gate_R, m->gate_R + n5, m->d.vol, (int)m->N, m->d.red);
    k_sum_partials<<<1, 32, 0, s>>>(m->d.red, m->d.red_blocks, kRedStride, kKeRateSums, sums + 8);
    UCNS_CUDA(cudaGetLastError());
    return launch_dt_to(m, U, sums + 13, s);  // the CFL time step of U, apart from the solver's own
  });
  if (rc) return rc;
  double h[14];
  UCNS_CUDA(cudaMemcpyAsync(h, sums, sizeof h, cudaMemcpyDeviceToHost, s));
  UCNS_CUDA(cudaStreamSynchronize(s));
  const double a = h[8] / h[10], b = h[9] / h[10];
  rel[0] = std::fabs(a - b) / std::fmax(std::fabs(b), 1e-300);
  rel[1] = h[11] / std::fmax(h[12], 1e-300);
  const double ke = h[4] / h[7];
  m->gate_ke_err += std::fabs(a - b) * (double)std::max(steps, 1) * h[13] / std::fmax(ke, 1e-300);
  rel[2] = m->gate_ke_err;
  // eps_s ~ sum V |curl u|^2, eps_d ~ 4/3 sum V (div u)^2 (1/Re and the volume cancel in the ratios)
  const double sg = h[1], sf = h[5], dg = (4.0 / 3.0) * h[2], df = (4.0 / 3.0) * h[6];
  rel[3] = std::fabs(sg - sf) / std::fmax(std::fabs(sf), 1e-300);
  rel[4] = std::fabs(dg - df) / std::fmax(std::fmax(std::fabs(df), 1e-3 * std::fabs(sf)), 1e-300);
  for (int q = 0; q < kGateMeasures; q++) m->gate_last[q] = rel[q];
  m->gate_checks++;
  const bool bad = !(rel[2] <= m->gate_bound) || !(rel[3] <= m->gate_bound) || !(rel[4] <= m->gate_bound) ||
                   (m->gate_bound_rate > 0.0 && !(rel[0] <= m->gate_bound_rate));
  if (bad) {
    m->gate_on = false;
    m->gate_off_step = m->gate_steps;
  }
  return UCNS_OK;
}

// dt_pending: m->d.dt is being computed on the side stream (join before use).
// pair_fresh: m->d.Uhl already holds the float pair of U (mixed form; the
// previous step of the same call wrote it).  keep_pair: the last stage also
// writes the float pair of the new state, for the next step of the same call.
int rk_step_device(ucns_mesh* m, double* U, cudaStream_t s, bool dt_pending = false, bool pair_fresh = false,
                   bool keep_pair = false) {
  int rc;
  double* W = m->d.Ustage;
  const int64_t step = m->gate_steps;
  bool split_done = pair_fresh, checked = false;
  if (!m->gate_fixed && m->gate_on && m->mlp && m->gate_check_every > 0 && step % m->gate_check_every == 0) {
    double rel[kGateMeasures];
    if ((rc = gate_check(m, U, rel, s, m->gate_check_every))) return rc;
    // the check evaluated the flags on this very state (and left its float pair in place)
    checked = m->gate_on;
    m->gate_flags_valid = checked;
    split_done = split_done || mixed(m);
  }
  if (m->gate_on && m->mlp) m->gate_steps++;
  if (!m->gate_fixed && m->gate_on && m->mlp && m->gate_flags_valid && (checked || step % m->gate_eval_every != 0)) {
    m->gate_eval_active = true;  // the flags of the check, or of the last evaluation
  } else {
    if ((rc = gate_eval(m, U, s, &split_done))) return rc;  // flags of U^n serve all three stages
    m->gate_flags_valid = m->gate_eval_active;
  }
  if ((!split_done && (rc = launch_split(m, U, s))) || (rc = launch_recon(m, U, s)) || (rc = launch_face(m, s)) ||
      (dt_pending && (rc = join_dt(m, s))))
    return rc;
  if (m->P.integrator == UCNS_RK_SSP54) {
    // u_1..u_4 in W (in place), the last stage into U
    if ((rc = launch_rk54(m, 1, U, U, W, s))) return rc;
    for (int st = 2; st <= 5; st++)
      if ((rc = launch_recon(m, W, s)) || (rc = launch_face(m, s)) ||
          (rc = launch_rk54(m, st, U, W, st == 5 ? U : W, s, keep_pair)))
        return rc;
    return UCNS_OK;
  }
  if ((rc = launch_rk(m, 1, U, U, W, s))) return rc;
  if ((rc = launch_recon(m, W, s)) || (rc = launch_face(m, s)) || (rc = launch_rk(m, 2, U, W, W, s)))
    return rc;
  if ((rc = launch_recon(m, W, s)) || (rc = launch_face(m, s)) || (rc = launch_rk(m, 3, U, W, U, s, keep_pair)))
    return rc;
  return UCNS_OK;
}

int read_error_word(ucns_mesh* m, cudaStream_t s) {
  int h = 0;
  UCNS_CUDA(cudaMemcpyAsync(&h, m->d.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  UCNS_CUDA(cudaStreamSynchronize(s));
  if (h) {
    UCNS_CUDA(cudaMemsetAsync(m->d.err, 0, sizeof(int), s));
    if (h & 2) return fail(UCNS_ERR_TIMEOUT, "a bounded wait for a bulk copy in the reconstruction gave up");
    return fail(UCNS_ERR_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or non-finite)");
  }
  return UCNS_OK;
}

}  // namespace

// The time-step reduction into caller-chosen scratch and output (used by the
// allocation-free entry point in noalloc.cu): one partial per block of
// kRedThreads cells, nblocks of them, then the CFL minimum into dt_out[0].
static_assert(kRedThreads == kDtBlockCells, "noalloc.cu sizes its partials by the reduction's block size");
int launch_dt_into(const ucns_mesh* m, const double* U, double* partials, int nblocks, double* dt_out,
                   cudaStream_t s) {
  const ucns_params& p = m->P;
  const double vc = p.reynolds > 0.0 ? p.prandtl / (2.0 * p.gamma * (1.0 / p.reynolds)) : 0.0;
  k_dt_partial<<<nblocks, kRedThreads, 0, s>>>(U, m->d.dtlen, (int)m->N, p.gamma, vc, partials, m->d.err);
  k_dt_final<<<1, kRedThreads, 0, s>>>(partials, nblocks, p.cfl, dt_out);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

void device_free(ucns_mesh* m) {
  for (auto& r : m->prof_live) {
    m->prof_pool.push_back(r.a);
    m->prof_pool.push_back(r.b);
  }
  m->prof_live.clear();
  for (void* e : m->prof_pool) cudaEventDestroy((cudaEvent_t)e);
  m->prof_pool.clear();
  if (m->gate_R) cudaFree(m->gate_R);
  m->gate_R = nullptr;
  if (m->gate_X) cudaFree(m->gate_X);
  if (m->gate_flag) cudaFree(m->gate_flag);
  if (m->gate_count) cudaFree(m->gate_count);

  m->gate_X = nullptr;
  m->gate_flag = nullptr;
  m->gate_count = nullptr;
  m->gate_eval_active = false;
  m->gate_fixed = false;
  DeviceMesh& d = m->d;
  void* ptrs[] = {d.fslot, d.bcell, d.bcount, d.inv_vol, d.vol, d.inv_h, d.dtlen, d.mom, d.sc, d.Pc, d.sd, d.Pd, d.Msi, d.psib, d.hot, d.Msif, d.psibf, d.Pcb, d.Pdb, d.scb, d.sdb, d.cellb, d.sda, d.Pda,
                  d.inv_hf, d.fpenf, d.cf, d.fo, d.fn, d.dvalid, d.fq, d.fqf, d.fpen, d.coef, d.coeff, d.Uhl, d.G,
                  d.Ustage, d.Uacc, d.Uhost, d.red, d.dt, d.err, d.dt_part, d.dt_count};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d = DeviceMesh{};
}

}  // namespace ucns

using namespace ucns;

extern "C" {

const char* ucns_last_error(void) { return g_err.c_str(); }

int ucns_mesh_create(const double* nodes, int64_t n_nodes, const int64_t* cell_nodes,
                     int64_t n_cells, int32_t nodes_per_cell, const double* periodic_box,
                     ucns_mesh** out) {
  if (!out) return fail(UCNS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!nodes || !cell_nodes || n_nodes <= 0 || n_cells <= 0)
    return fail(UCNS_ERR_INVALID_ARG, "nodes/cells must be non-NULL and non-empty");
  if (nodes_per_cell != 8 && nodes_per_cell != 6 && nodes_per_cell != 5 && nodes_per_cell != 4)
    return fail(UCNS_ERR_INVALID_ARG, "nodes_per_cell must be 8 (hexahedron), 6 (prism), 5 (pyramid) or 4 (tetrahedron)");
  if (n_cells >= (int64_t(1) << 31) / 10)
    return fail(UCNS_ERR_INVALID_ARG, "too many cells for 32-bit device indexing");
  for (int d = 0; periodic_box && d < 3; d++)
    if (!(periodic_box[d] >= 0.0) || !std::isfinite(periodic_box[d]))
      return fail(UCNS_ERR_INVALID_ARG, "box lengths must be finite and >= 0 (0: the axis is not periodic)");
  ucns_mesh* m = new (std::nothrow) ucns_mesh();
  if (!m) return fail(UCNS_ERR_NOMEM, "out of host memory");
  try {
    m->N = n_cells;
    m->nn = n_nodes;
    m->npc = nodes_per_cell;
    m->nfc = nodes_per_cell == 8 ? 6 : (nodes_per_cell == 4 ? 4 : 5);
    for (int d = 0; d < 3; d++) {
      m->L[d] = periodic_box ? periodic_box[d] : 0.0;
      m->per[d] = m->L[d] > 0.0;
    }
    m->X.assign(nodes, nodes + 3 * n_nodes);
    m->C.assign(cell_nodes, cell_nodes + nodes_per_cell * n_cells);
    int rc = build_topology(m);
    if (rc) {
      delete m;
      return rc;
    }
  } catch (const std::bad_alloc&) {
    delete m;
    return fail(UCNS_ERR_NOMEM, "out of host memory");
  }
  *out = m;
  return UCNS_OK;
}

int ucns_mesh_set_boundary(ucns_mesh* m, const int32_t* kinds, const double* inflow) {
  if (!m || !kinds) return fail(UCNS_ERR_INVALID_ARG, "mesh or kinds is NULL");
  for (int k = 0; k < 6; k++)
    if (kinds[k] < UCNS_BC_SLIP_WALL || kinds[k] > UCNS_BC_SUPERSONIC_INFLOW)
      return fail(UCNS_ERR_INVALID_ARG, "unknown boundary kind");
  bool need_inflow = false;
  for (int k = 0; k < 6; k++) need_inflow = need_inflow || kinds[k] == UCNS_BC_SUPERSONIC_INFLOW;
  if (need_inflow && !inflow) return fail(UCNS_ERR_INVALID_ARG, "an inflow side needs the inflow state");
  if (need_inflow)
    for (int v = 0; v < 5; v++)
      if (!std::isfinite(inflow[v])) return fail(UCNS_ERR_INVALID_ARG, "inflow state must be finite");
  for (int k = 0; k < 6; k++) m->bc[k] = kinds[k];
  for (int v = 0; v < 5; v++) m->uinf[v] = need_inflow ? inflow[v] : 0.0;
  m->precomputed = false;  // the boundary kinds enter the precompute
  return UCNS_OK;
}

static int check_params(const ucns_mesh* m, const ucns_params* p) {
  if (!m || !p) return fail(UCNS_ERR_INVALID_ARG, "mesh or params is NULL");
  if (p->order < 1 || p->order > 4) return fail(UCNS_ERR_INVALID_ARG, "order must be 1, 2, 3 or 4");
  if (p->scheme != UCNS_SCHEME_LINEAR && p->scheme != UCNS_SCHEME_CWENOZ)
    return fail(UCNS_ERR_INVALID_ARG, "unknown scheme");
  if (p->scheme == UCNS_SCHEME_CWENOZ && p->order < 2)
    return fail(UCNS_ERR_INVALID_ARG, "CWENOZ needs order 2 or more");
  if (p->precision != UCNS_PREC_FP64 && p->precision != UCNS_PREC_MIXED)
    return fail(UCNS_ERR_INVALID_ARG, "unknown precision mode");
  if (p->order > 2 && m->npc != 8) return fail(UCNS_ERR_INVALID_ARG, "orders 3 and 4 are built for hexahedra only");
  if (m->n_boundary > 0 && p->reynolds > 0.0)
    return fail(UCNS_ERR_INVALID_ARG, "boundary faces are built for inviscid flows (Re <= 0) only");
  if ((m->n_boundary > 0 || m->npc == 6 || m->npc == 5) && (p->precision != UCNS_PREC_FP64 || p->order > 2))
    return fail(UCNS_ERR_INVALID_ARG, "boundary faces, prisms and pyramids are built in the FP64 form at P1 and P2");
  if (p->integrator != UCNS_RK_SSP3 && p->integrator != UCNS_RK_SSP54)
    return fail(UCNS_ERR_INVALID_ARG, "unknown integrator");
  if (!(p->gamma > 1.0) || !(p->mach > 0.0) || !(p->cfl > 0.0) || !(p->lambda_central > 0.0) ||
      !(p->epsilon > 0.0) || (p->reynolds > 0.0 && !(p->prandtl > 0.0)))
    return fail(UCNS_ERR_INVALID_ARG, "invalid physical parameter");
  return UCNS_OK;
}

int ucns_precompute_host(ucns_mesh* m, const ucns_params* p) {
  int rc = check_params(m, p);
  if (rc) return rc;
  try {
    auto h = std::make_shared<HostArrays>();
    rc = host_precompute(m, p, h.get());
    if (rc) return rc;
    m->host = h;
  } catch (const std::bad_alloc&) {
    return fail(UCNS_ERR_NOMEM, "out of host memory");
  }
  return UCNS_OK;
}

int ucns_stencil(const ucns_mesh* m, int64_t cell, int32_t which, int64_t* members, double* P) {
  if (!m || !members || !P) return fail(UCNS_ERR_INVALID_ARG, "NULL argument");
  if (!m->host) return fail(UCNS_ERR_STATE, "ucns_precompute_host has not been called");
  if (cell < 0 || cell >= m->N) return fail(UCNS_ERR_INVALID_ARG, "cell id out of range");
  if (which < -1 || which >= m->nd) return fail(UCNS_ERR_INVALID_ARG, "no such stencil");
  const HostArrays& h = *m->host;
  const int64_t N = m->N, i = m->iperm[cell];
  if (which < 0) {
    for (int r = 0; r < m->Mc; r++) {
      members[r] = m->perm[h.sc[(size_t)r * N + i]];
      for (int k = 0; k < m->K; k++) P[k * m->Mc + r] = h.Pc[((size_t)k * m->Mc + r) * N + i];
    }
  } else {
    for (int r = 0; r < m->Md; r++) {
      members[r] = m->perm[h.sd[((size_t)which * m->Md + r) * N + i]];
      for (int k = 0; k < m->Kd; k++) P[k * m->Md + r] = h.Pd[(((size_t)which * m->Kd + k) * m->Md + r) * N + i];
    }
  }
  return UCNS_OK;
}

// Batches of the P1/P2 mixed face kernel (fb faces each): per batch the
// distinct cells of its faces' owners and neighbours in order of first use,
// per face the slots of its two rows (owner | neighbour << 16); arrays padded
// to fpad faces.  nu = the largest count, rounded up to a multiple of 4.
static void face_batches(const std::vector<int32_t>& fo, const std::vector<int32_t>& fn, int64_t N, int fb, int64_t fpad,
                  std::vector<int32_t>& fslot, std::vector<int32_t>& bcell, std::vector<int32_t>& bcount, int& nu) {
  const int64_t F = (int64_t)fo.size(), nbat = (F + fb - 1) / fb;
  std::vector<int64_t> stamp((size_t)N, -1);
  std::vector<int32_t> slot((size_t)N, 0);
  fslot.assign((size_t)fpad, 0);
  bcount.assign((size_t)nbat, 0);
  std::vector<int32_t> order;
  order.reserve((size_t)F * 2);
  for (int64_t b = 0; b < nbat; b++) {
    int32_t c = 0;
    for (int64_t f = b * fb; f < std::min(F, (b + 1) * fb); f++) {
      int32_t sl[2];
      const int32_t cells[2] = {fo[f], fn[f]};
      for (int e = 0; e < 2; e++) {
        const int32_t i = cells[e];
        if (stamp[i] != b) {
          stamp[i] = b;
          slot[i] = c++;
          order.push_back(i);
        }
        sl[e] = slot[i];
      }
      fslot[f] = sl[0] | (sl[1] << 16);
    }
    bcount[b] = c;
  }
  int mx = 1;
  for (int32_t c : bcount) mx = std::max(mx, (int)c);
  nu = (mx + 3) / 4 * 4;
  bcell.assign((size_t)nbat * nu, 0);
  size_t o = 0;
  for (int64_t b = 0; b < nbat; b++)
    for (int32_t u = 0; u < bcount[b]; u++) bcell[(size_t)b * nu + u] = order[o++];
}

// the device arrays of a precomputed mesh (host vectors built here may
// throw std::bad_alloc; the caller turns that into an error code)
static int device_upload(ucns_mesh* m, const ucns_params* p, const HostArrays& h) {
  int rc = UCNS_OK;
  device_free(m);
  m->precomputed = false;
  m->P = *p;
  DeviceMesh& d = m->d;
  d.N = (int32_t)m->N;
  d.F = (int32_t)m->F;
  std::vector<int32_t> fo(m->fo), fn(m->fn), cf((size_t)m->nfc * m->N);
  for (int64_t i = 0; i < m->N; i++)
    for (int j = 0; j < m->nfc; j++) cf[(size_t)j * m->N + i] = m->cf[(size_t)i * m->nfc + j];
  for (int64_t f = 0; f < m->F; f++)
    if (fn[f] < 0) fn[f] = -1 - (int32_t)h.fkind[f];  // a boundary face carries its kind
  if ((rc = upload(&d.vol, h.vol)) || (rc = upload(&d.inv_vol, h.inv_vol)) ||
      (rc = upload(&d.inv_h, h.inv_h)) || (rc = upload(&d.dtlen, h.dtlen)) ||
      (rc = upload(&d.mom, h.mom)) || (rc = upload(&d.sc, h.sc)) || (rc = upload(&d.sd, h.sd)) ||
      (rc = upload(&d.cf, cf)) || (rc = upload(&d.fo, fo)) || (rc = upload(&d.fn, fn)) ||
      (m->n_boundary > 0 && (rc = upload(&d.dvalid, h.dvalid)))) {
    device_free(m);
    return rc;
  }
  if (p->precision == UCNS_PREC_MIXED && m->K > 9) {
    const bool weno = m->nd > 0;
    const int64_t fpad = (m->F + kFacePad - 1) / kFacePad * kFacePad;  // whole batches for the face kernel's copies
    std::vector<int32_t> fslot, bcell, bcount;
    int nu = 0;
    face_batches(fo, fn, m->N, face_batch_faces(m->nq), fpad, fslot, bcell, bcount, nu);
    d.fnu = nu;
    rc = m->K == 19 ? upload_ho_tiles<3>(m, h, weno, &d.hot) : upload_ho_tiles<4>(m, h, weno, &d.hot);
    if (rc || (rc = upload_f32(&d.Msif, h.Msi)) ||
        (rc = upload_f32(&d.psibf, h.psib)) || (rc = upload_f32(&d.inv_hf, h.inv_h)) ||
        (rc = upload_cellwise(&d.fqf, h.fq, m->nq * 10, m->F, fpad)) || (rc = upload_f32(&d.fpenf, h.fpen, fpad)) ||
        (rc = upload(&d.fslot, fslot)) || (rc = upload(&d.bcell, bcell)) || (rc = upload(&d.bcount, bcount)) ||
        (rc = alloc(&d.coeff, (size_t)coef_row_floats(m) * m->N)) || (rc = alloc(&d.Uhl, (size_t)10 * m->N))) {
      device_free(m);
      return rc;
    }
  } else if (p->precision == UCNS_PREC_MIXED) {
    const int rc_rows = m->K * m->Mc, rd_rows = m->nd * 3 * m->Md;
    const int64_t fpad = (m->F + kFacePad - 1) / kFacePad * kFacePad;  // whole batches for the face kernel's copies
    std::vector<int32_t> fslot, bcell, bcount;
    int nu = 0;
    face_batches(fo, fn, m->N, face_batch_faces(m->nq), fpad, fslot, bcell, bcount, nu);
    d.fnu = nu;
    std::vector<double> cellrows((size_t)kCellRows * m->N);
    std::copy(h.mom.begin(), h.mom.begin() + (size_t)6 * m->N, cellrows.begin());
    std::copy(h.inv_h.begin(), h.inv_h.end(), cellrows.begin() + (size_t)6 * m->N);
    if ((rc = upload_blocked(&d.Pcb, h.Pc, rc_rows, m->N, true)) ||
        (rc = upload_blocked(&d.Pdb, h.Pd, rd_rows, m->N, true)) ||
        (rc = upload_blocked(&d.scb, h.sc, m->Mc, m->N, true)) ||
        (rc = upload_blocked(&d.sdb, h.sd, m->nd * m->Md, m->N, true)) ||
        (rc = upload_blocked(&d.cellb, cellrows, kCellRows, m->N, false)) ||
        (rc = upload_cellwise(&d.sda, h.sd, m->nd * m->Md, m->N)) ||
        (rc = upload_cellwise(&d.Pda, h.Pd, rd_rows, m->N)) ||
        (rc = upload_cellwise(&d.fqf, h.fq, m->nq * 10, m->F, fpad)) || (rc = upload_f32(&d.fpenf, h.fpen, fpad)) ||
        (rc = upload(&d.fslot, fslot)) || (rc = upload(&d.bcell, bcell)) || (rc = upload(&d.bcount, bcount)) ||
        (rc = upload_f32(&d.inv_hf, h.inv_h)) ||
        (rc = alloc(&d.coeff, (size_t)coef_row_floats(m) * m->N)) || (rc = alloc(&d.Uhl, (size_t)10 * m->N))) {
      device_free(m);
      return rc;
    }
  } else if ((rc = upload(&d.Pc, h.Pc)) || (rc = upload(&d.Pd, h.Pd)) || (rc = upload(&d.fq, h.fq)) ||
             (rc = upload(&d.fpen, h.fpen)) || (rc = upload(&d.Msi, h.Msi)) || (rc = upload(&d.psib, h.psib)) ||
             (rc = alloc(&d.coef, (size_t)m->NC * m->N * 5))) {
    device_free(m);
    return rc;
  }
  d.red_blocks = 4 * 152;
  if ((rc = alloc(&d.G, (size_t)5 * m->F)) ||
      (rc = alloc(&d.Ustage, (size_t)5 * m->N)) || (rc = alloc(&d.red, (size_t)kRedStride * d.red_blocks)) ||
      (p->integrator == UCNS_RK_SSP54 && (rc = alloc(&d.Uacc, (size_t)5 * m->N))) ||
      (rc = alloc(&d.dt, 2)) || (rc = alloc(&d.err, 1)) || (rc = alloc(&d.dt_part, (size_t)nblocks(m->N))) ||
      (rc = alloc(&d.dt_count, 1))) {
    device_free(m);
    return rc;
  }
  UCNS_CUDA(cudaMemset(d.err, 0, sizeof(int)));
  UCNS_CUDA(cudaMemset(d.dt_count, 0, sizeof(unsigned)));
  UCNS_CUDA(cudaDeviceSynchronize());
  m->precomputed = true;
  return UCNS_OK;
}

int ucns_precompute(ucns_mesh* m, const ucns_params* p) {
  int rc = check_params(m, p);
  if (rc) return rc;
  HostArrays h;
  try {
    rc = host_precompute(m, p, &h);
    m->host.reset();
  } catch (const std::bad_alloc&) {
    rc = fail(UCNS_ERR_NOMEM, "out of host memory");
  }
  if (rc) return rc;
  try {
    return device_upload(m, p, h);
  } catch (const std::bad_alloc&) {
    device_free(m);
    return fail(UCNS_ERR_NOMEM, "out of host memory while uploading the precompute");
  }
}

int ucns_residual(ucns_mesh* m, const double* U, double* R, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U || !R || U == R) return fail(UCNS_ERR_INVALID_ARG, "U and R must be distinct device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = gate_eval(m, U, s))) return rc;
  if ((rc = launch_split(m, U, s)) || (rc = launch_recon(m, U, s)) || (rc = launch_face(m, s)) ||
      (rc = launch_rk(m, 0, U, U, R, s)))
    return rc;
  return UCNS_OK;
}

int ucns_rk_step(ucns_mesh* m, double* U, double* dt_inout, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U) return fail(UCNS_ERR_INVALID_ARG, "U is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const bool given = dt_inout && *dt_inout > 0.0;
  if (given) {
    k_set_scalar<<<1, 1, 0, s>>>(m->d.dt, *dt_inout);  // by value: no host buffer outlives the call
    UCNS_CUDA(cudaGetLastError());
  } else if ((rc = launch_dt_async(m, U, s))) {
    return rc;
  }
  if ((rc = rk_step_device(m, U, s, !given))) return rc;
  if (dt_inout && !given) {
    UCNS_CUDA(cudaMemcpyAsync(dt_inout, m->d.dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    return read_error_word(m, s);
  }
  return UCNS_OK;
}

// n_steps CFL steps of a device state within one call: the float pair of the
// state carries from one step to the next (the caller cannot touch U in
// between); the simulated time accumulates on the device
int rk_steps_device(ucns_mesh* m, double* U, int32_t n_steps, cudaStream_t s) {
  int rc;
  double* tacc = m->d.dt + 1;  // device accumulator of the simulated time
  k_set_scalar<<<1, 1, 0, s>>>(tacc, 0.0);
  for (int k = 0; k < n_steps; k++) {
    if ((rc = launch_dt_async(m, U, s)) || (rc = rk_step_device(m, U, s, true, k > 0, k + 1 < n_steps))) return rc;
    k_add_scalar<<<1, 1, 0, s>>>(tacc, m->d.dt);  // after the step, which joined the time step
  }
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int ucns_rk_steps(ucns_mesh* m, double* U, int32_t n_steps, double* t_inout, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U || n_steps < 0) return fail(UCNS_ERR_INVALID_ARG, "U is NULL or n_steps < 0");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = rk_steps_device(m, U, n_steps, s))) return rc;
  double t = 0.0;
  UCNS_CUDA(cudaMemcpyAsync(&t, m->d.dt + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  if ((rc = read_error_word(m, s))) return rc;
  if (t_inout) *t_inout += t;
  return UCNS_OK;
}

int ucns_rk_steps_host(ucns_mesh* m, double* U_host, int32_t n_steps, double* t_inout, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U_host || n_steps < 0) return fail(UCNS_ERR_INVALID_ARG, "U_host is NULL or n_steps < 0");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)5 * m->N * sizeof(double);
  if (!m->d.Uhost && (rc = alloc(&m->d.Uhost, (size_t)5 * m->N))) return rc;
  UCNS_CUDA(cudaMemcpyAsync(m->d.Uhost, U_host, bytes, cudaMemcpyHostToDevice, s));
  if ((rc = rk_steps_device(m, m->d.Uhost, n_steps, s))) return rc;
  double t = 0.0;
  UCNS_CUDA(cudaMemcpyAsync(U_host, m->d.Uhost, bytes, cudaMemcpyDeviceToHost, s));
  UCNS_CUDA(cudaMemcpyAsync(&t, m->d.dt + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  if ((rc = read_error_word(m, s))) return rc;
  if (t_inout) *t_inout += t;
  return UCNS_OK;
}

int ucns_float_pair(const double* u, float* hi, float* lo, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!u || !hi || !lo))) return fail(UCNS_ERR_INVALID_ARG, "u, hi, lo must be non-NULL, n >= 0");
  if (n == 0) return UCNS_OK;
  const int64_t blocks = (n + 255) / 256;
  if (blocks > INT32_MAX) return fail(UCNS_ERR_INVALID_ARG, "n too large");
  k_float_pair<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(u, hi, lo, n);
  UCNS_CUDA(cudaGetLastError());
  return UCNS_OK;
}

int ucns_check_state(ucns_mesh* m, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  return read_error_word(m, (cudaStream_t)stream);
}

int ucns_alu_peak(int32_t which, double* flops_per_s, int32_t* n_sm, void* stream) {
  if (which < 0 || which > 2 || !flops_per_s) return fail(UCNS_ERR_INVALID_ARG, "which in 0..2, flops_per_s non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  UCNS_CUDA(cudaGetDevice(&dev));
  UCNS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (n_sm) *n_sm = sms;
  const int blocks = sms * 8, threads = 256;
  const int iters = which == 1 ? 1 << 12 : 1 << 15;
  cudaEvent_t e0, e1;
  UCNS_CUDA(cudaEventCreate(&e0));
  UCNS_CUDA(cudaEventCreate(&e1));
  double best = 0.0;
  for (int rep = 0; rep < 4; rep++) {  // the first launch warms up
    cudaEventRecord(e0, s);
    if (which == 0) k_peak_ffma<<<blocks, threads, 0, s>>>(iters, 1.000001f);
    else if (which == 1) k_peak_dfma<<<blocks, threads, 0, s>>>(iters, 1.000001);
    else k_peak_ffma2<<<blocks, threads, 0, s>>>(iters, 1.000001f);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(UCNS_ERR_CUDA, std::string("peak kernel: ") + cudaGetErrorString(e));
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double fl = 2.0 * kPeakChains * (which == 2 ? 2.0 : 1.0) * (double)iters * blocks * threads;
    if (rep > 0) best = std::fmax(best, fl / (ms * 1e-3));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  UCNS_CUDA(cudaGetLastError());
  *flops_per_s = best;
  return UCNS_OK;
}

int ucns_probe_bounded_wait(ucns_mesh* m, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  k_bulk_wait_probe<<<1, 32, 0, s>>>(m->d.err, 1ll << 21);  // ~1 ms at 2 GHz
  UCNS_CUDA(cudaGetLastError());
  return read_error_word(m, s);
}

int ucns_time_step(ucns_mesh* m, const double* U, double* dt, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U || !dt) return fail(UCNS_ERR_INVALID_ARG, "U or dt is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = launch_dt(m, U, s))) return rc;
  UCNS_CUDA(cudaMemcpyAsync(dt, m->d.dt, sizeof(double), cudaMemcpyDeviceToHost, s));
  return read_error_word(m, s);
}

int ucns_diagnostics(ucns_mesh* m, const double* U, ucns_diag* out, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U || !out) return fail(UCNS_ERR_INVALID_ARG, "U or out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  m->gate_eval_active = false;  // diagnostics always use the full scheme
  if ((rc = launch_split(m, U, s)) || (rc = launch_recon(m, U, s))) return rc;
  rc = timed(m, kKindDiag, s, [&] {
    if (mixed(m))
      k_diag_partial_mx<<<m->d.red_blocks, kRedThreads, 0, s>>>(U, m->d.coeff, coef_row_floats(m), m->NC,
                                                                 m->d.vol, (int)m->N, m->d.red);
    else
      k_diag_partial<double><<<m->d.red_blocks, kRedThreads, 0, s>>>(U, m->d.coef, m->d.vol, (int)m->N, m->d.red);
    // the final sums land in the first 4 doubles of G (free between residuals)
    k_diag_final<<<1, 32, 0, s>>>(m->d.red, m->d.red_blocks, m->d.G);
    UCNS_CUDA(cudaGetLastError());
    return UCNS_OK;
  });
  if (rc) return rc;
  double h[4];
  UCNS_CUDA(cudaMemcpyAsync(h, m->d.G, sizeof h, cudaMemcpyDeviceToHost, s));
  UCNS_CUDA(cudaStreamSynchronize(s));
  const double mu = m->P.reynolds > 0.0 ? 1.0 / m->P.reynolds : 1.0;
  out->kinetic_energy = h[0] / h[3];
  out->eps_solenoidal = mu * h[1] / h[3];
  out->eps_dilatational = 4.0 / 3.0 * mu * h[2] / h[3];
  out->volume = h[3];
  return UCNS_OK;
}

int ucns_profile(ucns_mesh* m, int32_t enable) {
  if (!m) return fail(UCNS_ERR_INVALID_ARG, "mesh handle is NULL");
  if (enable) {
    for (auto& r : m->prof_live) {
      m->prof_pool.push_back(r.a);
      m->prof_pool.push_back(r.b);
    }
    m->prof_live.clear();
    for (int k = 0; k < kKinds; k++) {
      m->prof_ms[k] = 0.0;
      m->prof_n[k] = 0;
    }
  }
  m->prof = enable != 0;
  return UCNS_OK;
}

int ucns_profile_read(ucns_mesh* m, double* ms, int64_t* launches) {
  if (!m || !ms || !launches) return fail(UCNS_ERR_INVALID_ARG, "NULL argument");
  for (auto& r : m->prof_live) {
    UCNS_CUDA(cudaEventSynchronize((cudaEvent_t)r.b));
    float t = 0.f;
    UCNS_CUDA(cudaEventElapsedTime(&t, (cudaEvent_t)r.a, (cudaEvent_t)r.b));
    m->prof_ms[r.kind] += t;
    m->prof_n[r.kind] += 1;
    m->prof_pool.push_back(r.a);
    m->prof_pool.push_back(r.b);
  }
  m->prof_live.clear();
  for (int k = 0; k < kKinds; k++) {
    ms[k] = m->prof_ms[k];
    launches[k] = m->prof_n[k];
  }
  return UCNS_OK;
}

int ucns_gate_features(ucns_mesh* m, const double* U, void* X, float* Xf, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U || !X) return fail(UCNS_ERR_INVALID_ARG, "U or X is NULL");
  if (((uintptr_t)X & 15) != 0) return fail(UCNS_ERR_INVALID_ARG, "X must be 16-byte aligned");
  if (m->K != 9 || m->nfc == 5 || m->n_boundary > 0)
    return fail(UCNS_ERR_INVALID_ARG, "features need a periodic P2 mesh of hexahedra or tetrahedra");
  return launch_features(m, U, X, Xf, (cudaStream_t)stream);
}

int ucns_gate_labels(ucns_mesh* m, const double* U, float* dev, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U || !dev) return fail(UCNS_ERR_INVALID_ARG, "U or dev is NULL");
  if (mixed(m) || m->nd == 0 || m->K != 9 || m->n_boundary > 0 || m->nfc == 5)
    return fail(UCNS_ERR_INVALID_ARG, "labels need a periodic FP64 P2 CWENOZ mesh of hexahedra or tetrahedra");
  cudaStream_t s = (cudaStream_t)stream;
  UCNS_CUDA(cudaMemsetAsync(dev, 0, sizeof(float) * m->N, s));
  m->gate_eval_active = false;
  m->label_out = dev;
  rc = launch_recon(m, U, s);
  m->label_out = nullptr;
  return rc;
}

// the gate's device buffers (features, flags, counter), once per mesh
static int gate_buffers(ucns_mesh* m) {
  int rc;
  if (!m->gate_X) {
    if ((rc = alloc((uint8_t**)&m->gate_X, (size_t)m->N * 64)) || (rc = alloc(&m->gate_flag, (size_t)m->N)) ||
        (rc = alloc(&m->gate_count, 1)))
      return rc;
  }
  return UCNS_OK;
}

int ucns_gate_attach(ucns_mesh* m, ucns_mlp* mlp, float threshold) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (mlp && (m->K != 9 || m->nd == 0 || m->n_boundary > 0 || m->nfc == 5))
    return fail(UCNS_ERR_INVALID_ARG, "the gate needs a periodic P2 CWENOZ mesh of hexahedra or tetrahedra");
  if (mlp && (rc = gate_buffers(m))) return rc;
  m->mlp = mlp;
  m->gate_thr = threshold;
  m->gate_flags_valid = false;
  if (!mlp) m->gate_on = false;
  return UCNS_OK;
}

int ucns_gate_enable(ucns_mesh* m, int32_t enable) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (enable && !m->mlp) return fail(UCNS_ERR_STATE, "no network attached");
  m->gate_on = enable != 0;
  m->gate_flags_valid = false;
  if (m->gate_on) m->gate_off_step = -1;
  return UCNS_OK;
}

int ucns_gate_configure(ucns_mesh* m, int32_t eval_every, int32_t check_every, double bound, double bound_rate) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (eval_every < 1 || check_every < 0 || !(bound > 0.0) || !(bound_rate >= 0.0))
    return fail(UCNS_ERR_INVALID_ARG, "eval_every >= 1, check_every >= 0, bound > 0 and bound_rate >= 0");
  m->gate_eval_every = eval_every;
  m->gate_flags_valid = false;
  m->gate_check_every = check_every;
  m->gate_bound = bound;
  m->gate_bound_rate = bound_rate;
  m->gate_steps = 0;
  m->gate_checks = 0;
  m->gate_off_step = -1;
  m->gate_ke_err = 0.0;
  for (int q = 0; q < kGateMeasures; q++) m->gate_last[q] = -1.0;
  return UCNS_OK;
}

int ucns_gate_check(ucns_mesh* m, const double* U, double* rel_diff, int32_t* disabled, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!U || !rel_diff) return fail(UCNS_ERR_INVALID_ARG, "U or rel_diff is NULL");
  if (!m->mlp || !m->gate_on) return fail(UCNS_ERR_STATE, "the gate is not enabled");
  rc = gate_check(m, U, rel_diff, (cudaStream_t)stream, m->gate_check_every);
  if (rc) return rc;
  if (disabled) *disabled = m->gate_on ? 0 : 1;
  return UCNS_OK;
}

int ucns_gate_status(const ucns_mesh* m, int32_t* enabled, int64_t* counts, double* last) {
  if (!m) return fail(UCNS_ERR_INVALID_ARG, "mesh handle is NULL");
  if (enabled) *enabled = (m->gate_on && m->mlp) ? 1 : 0;
  if (counts) {
    counts[0] = m->gate_steps;
    counts[1] = m->gate_checks;
    counts[2] = m->gate_off_step;
  }
  if (last)
    for (int q = 0; q < kGateMeasures; q++) last[q] = m->gate_last[q];
  return UCNS_OK;
}

int ucns_gate_set_flags(ucns_mesh* m, const uint8_t* flags, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!flags) {
    m->gate_fixed = false;
    m->gate_flags_valid = false;
    return UCNS_OK;
  }
  if (m->K != 9 || m->nd == 0 || m->n_boundary > 0 || m->nfc == 5)
    return fail(UCNS_ERR_INVALID_ARG, "the gate needs a periodic P2 CWENOZ mesh of hexahedra or tetrahedra");
  if ((rc = gate_buffers(m))) return rc;
  UCNS_CUDA(cudaMemcpyAsync(m->gate_flag, flags, (size_t)m->N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  m->gate_fixed = true;
  m->gate_flags_valid = false;
  return UCNS_OK;
}

int ucns_gate_flags(ucns_mesh* m, uint8_t* flags, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!flags) return fail(UCNS_ERR_INVALID_ARG, "flags is NULL");
  if (!m->gate_flag) return fail(UCNS_ERR_STATE, "no flags: neither a network nor caller flags were set");
  UCNS_CUDA(cudaMemcpyAsync(flags, m->gate_flag, (size_t)m->N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return UCNS_OK;
}

int ucns_gate_flagged(ucns_mesh* m, int64_t* n_flagged, void* stream) {
  int rc = check_ready(m);
  if (rc) return rc;
  if (!n_flagged) return fail(UCNS_ERR_INVALID_ARG, "n_flagged is NULL");
  if (!m->gate_flag) return fail(UCNS_ERR_STATE, "no network attached");
  cudaStream_t s = (cudaStream_t)stream;
  UCNS_CUDA(cudaMemsetAsync(m->gate_count, 0, sizeof(unsigned long long), s));
  k_count_flags<<<4 * 152, 256, 0, s>>>(m->gate_flag, (int)m->N, m->gate_count);
  unsigned long long h = 0;
  UCNS_CUDA(cudaMemcpyAsync(&h, m->gate_count, sizeof h, cudaMemcpyDeviceToHost, s));
  UCNS_CUDA(cudaStreamSynchronize(s));
  *n_flagged = (int64_t)h;
  return UCNS_OK;
}

int ucns_cell_order(const ucns_mesh* m, int64_t* perm) {
  if (!m || !perm) return fail(UCNS_ERR_INVALID_ARG, "mesh or perm is NULL");
  std::memcpy(perm, m->perm.data(), sizeof(int64_t) * m->N);
  return UCNS_OK;
}

int ucns_mesh_info(const ucns_mesh* m, int64_t* info) {
  if (!m || !info) return fail(UCNS_ERR_INVALID_ARG, "mesh or info is NULL");
  info[0] = m->N;
  info[1] = m->F;
  info[2] = m->K;
  info[3] = m->Mc;
  info[4] = m->nd;
  info[5] = m->Md;
  info[6] = m->nq;
  info[7] = m->nfc;
  return UCNS_OK;
}

void ucns_mesh_destroy(ucns_mesh* m) {
  if (!m) return;
  device_free(m);
  if (m->aux) cudaStreamDestroy((cudaStream_t)m->aux);
  if (m->ev_u) cudaEventDestroy((cudaEvent_t)m->ev_u);
  if (m->ev_dt) cudaEventDestroy((cudaEvent_t)m->ev_dt);
  delete m;
}

}  // extern "C"
