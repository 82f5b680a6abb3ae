// Internal data model of libucns: host topology/geometry built once by
// ucns_mesh_create / ucns_precompute, and the device-resident structure-of-
// arrays copy the kernels read (Sec. 3.2: flat arrays with explicit offsets,
// persistent device residency; cells in a Morton order).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "ucns.h"

namespace ucns {

struct HostArrays;
constexpr int kMaxK = 34;   // non-constant modes of a quartic in 3-D (P4)
constexpr int kMaxMc = 68;  // central stencil size 2K
constexpr int kMaxDir = 6;  // directional stencils = faces of the element
constexpr int kGateMeasures = 5;  // measures of the gate's plain-scheme check
constexpr int kDtBlockCells = 256;  // cells per partial minimum of the time-step reduction

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

// Device pointers of one precomputed mesh (all in internal cell order).
struct DeviceMesh {
  int32_t N = 0, F = 0;
  // cells
  double* inv_vol = nullptr;  // [N]
  double* vol = nullptr;      // [N]
  double* inv_h = nullptr;    // [N] 1/h_i, h_i = V_i^(1/3)
  double* dtlen = nullptr;    // [N] CFL length 2 V_i / sum_f |S_f|
  double* mom = nullptr;      // [6][N] (1/V) int xi_a xi_b: xx yy zz xy xz yz
  int32_t* sc = nullptr;      // [Mc][N] central stencil
  double* Pc = nullptr;       // [K][Mc][N] central pseudo-inverse
  int32_t* sd = nullptr;      // [nd][Md][N] directional stencils
  double* Pd = nullptr;       // [nd][Kd][Md][N]
  double* Msi = nullptr;      // P3/P4: [K(K+1)/2][N] smoothness-indicator matrix (upper triangle, row-major)
  float* hot = nullptr;       // P3/P4 mixed form: stencil ids and FP32 pseudo-inverses in 64-cell tiles; FP32 Msi, psib
  float* Msif = nullptr;
  float* psibf = nullptr;
  double* psib = nullptr;     // P3/P4: [K-3][N] cell means of the non-linear basis monomials (xi units)
  // mixed precision: FP32 pseudo-inverses and the stencils in the pair-blocked
  // layout [ceil(N/64)][rows/2][64][2] (tiles of 64 consecutive cells, row
  // pairs of a cell adjacent), the cell rows blocked [ceil(N/64)][rows][64]
  float* Pcb = nullptr;       // rows k Mc + m
  float* Pdb = nullptr;       // rows (s 3 + k) Md + r
  int32_t* scb = nullptr;     // rows m
  int32_t* sdb = nullptr;     // rows s Md + r
  float* cellb = nullptr;     // rows: the six second moments, then 1/h
  int32_t* sda = nullptr;     // [N][nd Md] directional stencils, cell-contiguous (gated CWENOZ)
  float* Pda = nullptr;       // [N][nd 3 Md] directional rows, cell-contiguous
  float* inv_hf = nullptr;    // [N]
  float* fpenf = nullptr;     // [F] ([F'] padded to whole face batches in the P1/P2 mixed form)
  int32_t* fslot = nullptr;   // [F'] mixed face batches: owner | neighbour << 16 row slots
  int32_t* bcell = nullptr;   // [batches][fnu] the batch's distinct cells
  int32_t* bcount = nullptr;  // [batches]
  int32_t fnu = 0;            // slots per batch
  int32_t* cf = nullptr;      // [nfc][N] face id << 1 | (cell is the neighbour)
  // faces
  int32_t* fo = nullptr;      // [F] owner
  int32_t* fn = nullptr;      // [F] neighbour; on a boundary face -1 - its boundary kind
  uint8_t* dvalid = nullptr;  // [N] bit s: directional candidate s exists (meshes with boundary faces)
  double* fq = nullptr;       // [nq][10][F] x-x_L(3) x-x_R'(3) n(3) |dS|(1), physical offsets
  float* fqf = nullptr;       // FP32 copy, point-contiguous [F][nq][10]
  double* fpen = nullptr;     // [F] alpha / L_int
  // scratch owned by the handle
  double* coef = nullptr;     // [NC][N][5] reconstructed monomial coefficients
  float* coeff = nullptr;     // FP32 coefficients (mixed)
  float* Uhl = nullptr;       // [N][5][2] float pairs (hi, lo) of the state being reconstructed (mixed)
  double* G = nullptr;        // [5][F] face flux integrals (mixed form: [5][F] floats in the first half)
  double* Ustage = nullptr;   // [5][N] Runge-Kutta stage state
  double* Uacc = nullptr;     // [5][N] SSP(5,4) accumulator of the last stage's combination
  double* Uhost = nullptr;    // [5][N] device copy for the host-buffer entry point
  double* red = nullptr;      // reduction partials
  double* dt = nullptr;       // [1] device time step
  int* err = nullptr;         // [1] device error word
  double* dt_part = nullptr;  // [ceil(N/256)] block minima of the fused time-step kernel
  unsigned* dt_count = nullptr;  // [1] its finished-block counter (zero between launches)
  int red_blocks = 0;
};

}  // namespace ucns

struct ucns_mesh {
  // ---- topology (host) ----
  int64_t N = 0, nn = 0;
  int npc = 0, nfc = 0;  // nodes and faces per cell: 8/6 hexahedron, 6/5 prism, 5/5 pyramid, 4/4 tetrahedron
  double L[3] = {0, 0, 0};
  int per[3] = {0, 0, 0};  // periodic axes (box length > 0)
  int64_t n_boundary = 0;  // faces on non-periodic sides of the box
  // boundary kind of each box side x-, x+, y-, y+, z-, z+ (UCNS_BC_*) and the inflow state
  int bc[6] = {0, 0, 0, 0, 0, 0};
  double uinf[5] = {0, 0, 0, 0, 0};
  std::vector<double> X;        // [nn][3]
  std::vector<int64_t> C;       // [N][npc] (user order)
  std::vector<int64_t> canon;   // node -> canonical node
  std::vector<int64_t> perm;    // internal -> user
  std::vector<int64_t> iperm;   // user -> internal
  // faces, internal numbering; owner = the cell with the lower user id
  int64_t F = 0;
  std::vector<int32_t> fo, fn;  // internal cell ids
  std::vector<int8_t> flf;      // owner-local face index
  std::vector<int32_t> cf;      // [N][nfc] internal, face << 1 | is_neighbour
  // ---- precompute ----
  bool precomputed = false;
  ucns_params P{};
  int K = 0, Mc = 0, nd = 0, Md = 0, Kd = 0, nq = 0, NC = 0;  // Kd: modes of a directional candidate
  ucns::DeviceMesh d;
  std::shared_ptr<ucns::HostArrays> host;  // kept only by ucns_precompute_host
  // learned troubled-cell gate
  struct ::ucns_mlp* mlp = nullptr;  // not owned
  float gate_thr = 0.f;
  bool gate_on = false;
  void* gate_X = nullptr;              // [N][32] BF16 features
  uint8_t* gate_flag = nullptr;        // [N]
  unsigned long long* gate_count = nullptr;
  bool gate_eval_active = false;       // flags valid for the reconstructions of this call
  bool gate_fixed = false;             // flags given by the caller (ucns_gate_set_flags), no network
  int gate_check_every = 0;
  int gate_eval_every = 1;
  bool gate_flags_valid = false;       // flags of an earlier step may be reused
  double gate_bound = 1e-4;            // on the estimated KE history error and the dissipation difference
  double gate_bound_rate = 0.0;        // on the relative difference of the total KE rates (0: not used)
  int64_t gate_steps = 0;              // gated steps since ucns_gate_configure
  int64_t gate_checks = 0;             // plain-scheme checks run
  int64_t gate_off_step = -1;          // gated step at which a check switched the gate off
  double gate_ke_err = 0.0;            // running estimate of the KE history's relative error
  double gate_last[5] = {-1.0, -1.0, -1.0, -1.0, -1.0};  // the last check's measures (kGateMeasures)
  // gate_R below: [2][5][N] residuals of the check, then 16 doubles of its sums
  double* gate_R = nullptr;            // [2][5][N] residuals of the check
  float* label_out = nullptr;          // set only inside ucns_gate_labels
  // side stream of the time-step reduction (it overlaps the first stage's
  // reconstruction) and its two events (cudaStream_t / cudaEvent_t), created
  // on first use, released by ucns_mesh_destroy
  void* aux = nullptr;
  void* ev_u = nullptr;
  void* ev_dt = nullptr;
  // opt-in kernel timing
  bool prof = false;
  struct ProfRec {
    int kind;
    void* a;
    void* b;
  };
  std::vector<ProfRec> prof_live;
  std::vector<void*> prof_pool;
  double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t prof_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace ucns {
int build_topology(ucns_mesh* m);
struct HostArrays;
int host_precompute(ucns_mesh* m, const ucns_params* p, HostArrays* h);
void device_free(ucns_mesh* m);
}  // namespace ucns
