/*
 * ucns.h -- C ABI of the GB300 residual / SSP-RK library (libucns.so).
 *
 * Computes the explicit residual of the high-order cell-centred finite-volume
 * discretisation of the compressible Navier-Stokes equations (Sec. 2.2,
 * Eqs. 1-2): k-exact least-squares reconstruction (Eqs. 3-4) with CWENOZ
 * nonlinear weights over central and directional stencils (Eqs. 5-6),
 * gradients at face Gauss points, HLLC inviscid flux and viscous flux with
 * the interface jump penalty (Eq. 7), periodic boundaries, an owner-side
 * residual sum, and the explicit SSP Runge-Kutta update (Eq. 8; the
 * three-stage third-order Shu-Osher form by default, or the paper's
 * five-stage fourth-order scheme, ucns_params.integrator).
 *
 * Conventions shared by every call
 *  - Every function returns an int status: UCNS_OK (0) or a negative
 *    UCNS_ERR_* code; ucns_last_error() then returns a thread-local message.
 *    No C++ exception crosses this boundary.
 *  - Flow states are conserved variables (rho, rho u, rho v, rho w, rho E) in
 *    structure-of-arrays layout [5][n_cells] of float64, stored in the
 *    library's INTERNAL cell order (a locality-preserving Morton order).
 *    ucns_cell_order() returns the permutation to and from the caller's
 *    order.  Unless a name ends in _host, state pointers are CUDA device
 *    pointers owned by the caller; the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it; calls that return host values
 *    synchronise that stream before returning.
 *  - The mesh handle owns all topology, geometry, stencil, pseudo-inverse and
 *    scratch storage (host and device).  One handle must not be used from two
 *    host threads at once.
 *  - Non-dimensionalisation: rho0 = 1, U0 = 1, L = 1, T0 = 1, gas constant
 *    R = 1/(gamma M^2), constant viscosity mu = 1/Re, conductivity
 *    kappa = mu c_p / Pr.
 */
#ifndef UCNS_H
#define UCNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define UCNS_OK 0
#define UCNS_ERR_INVALID_ARG (-1)  /* NULL/ill-sized argument, unsupported option */
#define UCNS_ERR_MESH (-2)         /* inverted cell, unpaired/non-manifold face, bad node id */
#define UCNS_ERR_STENCIL (-3)      /* too few stencil cells or rank-deficient least squares */
#define UCNS_ERR_CUDA (-4)         /* CUDA runtime failure (message names the call) */
#define UCNS_ERR_NONPHYSICAL (-5)  /* a state with rho <= 0, p <= 0 or non-finite */
#define UCNS_ERR_TIMEOUT (-6)      /* a bounded device wait ran out */
#define UCNS_ERR_STATE (-7)        /* call order: e.g. residual before precompute */
#define UCNS_ERR_NOMEM (-8)        /* host or device allocation failed */

#define UCNS_SCHEME_LINEAR 0  /* optimal central polynomial only (linear weights) */
#define UCNS_SCHEME_CWENOZ 1  /* CWENOZ over central + directional stencils */

#define UCNS_PREC_FP64 0   /* every step in FP64 */
#define UCNS_PREC_MIXED 1  /* FP32 pseudo-inverses, contractions and flux arithmetic;
                              stencil differences from a float pair of the FP64 state
                              (exact leading-part subtraction); FP64 state, face
                              totals, RK accumulation and reductions */

/* Explicit SSP Runge-Kutta integrator of the semi-discrete system (Eq. 8). */
#define UCNS_RK_SSP3 0   /* three-stage third-order SSP-RK (Shu-Osher form), the default */
#define UCNS_RK_SSP54 1  /* five-stage fourth-order SSP-RK of Spiteri and Ruuth, the
                            paper's integrator (SSP coefficient 1.508) */

/* Scheme parameters (Sec. 2.2). */
typedef struct ucns_params {
  int32_t order;      /* reconstruction degree r: 1 (P1) to 4 (P4); orders 3 and 4
                         on hexahedra, in the FP64 form */
  int32_t scheme;     /* UCNS_SCHEME_*; CWENOZ needs order 2 or more (linear
                         directional candidates at P2 and P3, quadratic at P4) */
  int32_t precision;  /* UCNS_PREC_* */
  int32_t integrator; /* UCNS_RK_* (0: SSP-RK3) */
  double gamma;       /* ratio of specific heats (1.4) */
  double prandtl;     /* Pr (0.71) */
  double reynolds;    /* Re; <= 0 selects the inviscid (Euler) flux only */
  double mach;        /* reference Mach number M (sets R = 1/(gamma M^2)) */
  double cfl;         /* CFL number of the time-step control */
  double lambda_central; /* un-normalised linear weight of the central stencil
                            (directional stencils: 1); e.g. 1000 */
  double epsilon;     /* epsilon of Eq. 6 (e.g. 1e-6) */
  double alpha;       /* viscous jump penalty alpha of Eq. 7 (4/3) */
} ucns_params;

/* Volume-averaged diagnostics (Taylor-Green): KE = sum V rho|u|^2/2 / sum V;
 * eps_s = sum V |curl u|^2 / (Re sum V); eps_d = 4/3 sum V (div u)^2/(Re sum V),
 * with u and grad u at each centroid from the cell average and the
 * reconstructed polynomial (Re <= 0: the sums without 1/Re). */
typedef struct ucns_diag {
  double kinetic_energy;
  double eps_solenoidal;
  double eps_dilatational;
  double volume;
} ucns_diag;

typedef struct ucns_mesh ucns_mesh; /* opaque, library-owned */

/* Build the mesh topology (Sec. 3.2 flat arrays; one GPU, periodic wrap in
 * place of the halo exchange).
 *  nodes       host [n_nodes][3] float64, copied.
 *  cell_nodes  host [n_cells][nodes_per_cell] int64 node ids, copied.
 *              nodes_per_cell = 8 (hexahedron, VTK node order), 6 (triangular
 *              prism: base 0 1 2 counter-clockwise seen from the top 3 4 5,
 *              node k + 3 above node k), 5 (pyramid: base 0 1 2 3
 *              counter-clockwise seen from the apex 4) or 4 (tetrahedron,
 *              positive orientation); one element type per mesh (Sec. 2.2's
 *              element types).
 *  periodic_box host [3] box lengths (NULL: none); an axis of length > 0 is
 *              periodic (nodes equal modulo the length are one node), an axis
 *              of length 0 is not: the element faces on its two planes are
 *              boundary faces, of the kinds ucns_mesh_set_boundary sets.  Every
 *              other element face must pair with exactly one other.
 *  out         receives the handle; free it with ucns_mesh_destroy.
 * Errors: INVALID_ARG (also n_cells >= 2^31 / 10 = 214,748,364: device
 * indexing is 32-bit), MESH (bad node id, non-positive volume, unpaired or
 * non-manifold face), NOMEM. */
int ucns_mesh_create(const double* nodes, int64_t n_nodes, const int64_t* cell_nodes,
                     int64_t n_cells, int32_t nodes_per_cell, const double* periodic_box,
                     ucns_mesh** out);

/* Boundary kinds of the box sides of non-periodic axes (the paper's
 * boundary-condition kernel, Sec. 3.6: ghost states at the boundary Gauss
 * points), for inviscid flows: the ghost state of a boundary Gauss point is
 * the mirror image of the owner's reconstructed state (UCNS_BC_SLIP_WALL, and
 * UCNS_BC_SYMMETRY, the same for a symmetry plane: density and energy kept,
 * normal momentum reversed), that state itself (UCNS_BC_SUPERSONIC_OUTFLOW:
 * extrapolation), or the given state (UCNS_BC_SUPERSONIC_INFLOW); the face
 * flux is HLLC between the two.  A boundary face's side is the axis of the
 * largest component of its outward area vector and that component's sign.
 * Stencils stop at boundary faces (one-sided), and a cell has no directional
 * candidate across a boundary face, its linear weights being normalised over
 * the candidates it has.
 *  kinds   host int32 [6]: the kinds of the sides x-, x+, y-, y+, z-, z+
 *          (sides of periodic axes are ignored); default all UCNS_BC_SLIP_WALL.
 *  inflow  host [5] conserved inflow state, needed when a side is an inflow.
 * Takes effect at the next ucns_precompute (the mesh needs one again).
 * Errors: INVALID_ARG. */
#define UCNS_BC_SLIP_WALL 0
#define UCNS_BC_SYMMETRY 1
#define UCNS_BC_SUPERSONIC_OUTFLOW 2
#define UCNS_BC_SUPERSONIC_INFLOW 3
int ucns_mesh_set_boundary(ucns_mesh* mesh, const int32_t* kinds, const double* inflow);

/* Geometry, quadrature, stencils and least-squares pseudo-inverses
 * (Eq. 4: P' = A^+ diag(|V_m|), A_mk = int_{V_m} phi_k, by Householder QR in
 * FP64 on the host), uploaded to the current CUDA device once.  May be called
 * again with other parameters (re-uploads).  Meshes with boundary faces need
 * an inviscid flow (reynolds <= 0); boundary faces, prisms and pyramids are
 * built in the FP64 form at P1 and P2.  Device memory is dominated by the
 * pseudo-inverses: per cell about 2.7 KB (P2 FP64 CWENOZ), 9 / 33 KB (P3 / P4
 * FP64) and 4.4 / 16.2 KB (P3 / P4 mixed, held in 64-cell tile records); the
 * host needs the FP64 arrays and, briefly, the device layout's copy.  Errors:
 * INVALID_ARG, STENCIL, CUDA, NOMEM (also when the host runs out of memory
 * while building the device arrays; nothing stays allocated). */
int ucns_precompute(ucns_mesh* mesh, const ucns_params* params);

/* Host half of ucns_precompute only (no CUDA call): geometry, stencils and
 * pseudo-inverses are computed in FP64 and kept in host memory so that
 * ucns_stencil can inspect them; the device is not touched.  Errors as
 * ucns_precompute (except CUDA). */
int ucns_precompute_host(ucns_mesh* mesh, const ucns_params* params);

/* Members and pseudo-inverse of one stencil of cell `cell` (caller's id),
 * from the host data of ucns_precompute_host.
 *  which    -1: central stencil (M = central size, K modes);
 *           s in [0, directional stencils): the directional stencil of the
 *           cell's local face s (M = directional size, M/2 modes: linear, or
 *           quadratic at P4).
 *  members  host int64 [M]: caller's cell ids, in the library's order.
 *  P        host float64 [modes][M] row-major: P' = A^+ diag(|V_m|) of Eq. 4.
 *           Row k belongs to the basis monomial psi_k = xi^e_k, xi =
 *           (x - x_i)/|V_i|^(1/3): x y z xx yy zz xy xz yz (P2), then the
 *           cubics xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz (P3), then the
 *           quartics xxxx xxxy xxxz xxyy xxyz xxzz xyyy xyyz xyzz xzzz yyyy
 *           yyyz yyzz yzzz zzzz (P4).
 * Errors: STATE (no host precompute), INVALID_ARG. */
int ucns_stencil(const ucns_mesh* mesh, int64_t cell, int32_t which, int64_t* members, double* P);

/* R = dU/dt (Eq. 2) for the state U.  U, R: device [5][n_cells] float64,
 * internal order, must not overlap.  Errors: STATE, INVALID_ARG, CUDA. */
int ucns_residual(ucns_mesh* mesh, const double* U, double* R, void* stream);

/* One step of the mesh's SSP Runge-Kutta integrator (three residual
 * evaluations for UCNS_RK_SSP3, five for UCNS_RK_SSP54) of U in place.
 *  dt_inout  NULL: dt = CFL condition evaluated on the device from U, kept on
 *            the device (no host synchronisation);
 *            *dt_inout > 0: use that dt;
 *            *dt_inout <= 0: compute dt as above and return it in *dt_inout
 *            (synchronises the stream).
 * Returns UCNS_ERR_NONPHYSICAL if the device found a non-physical new state;
 * that check is read back only when the call synchronises (dt returned) or in
 * ucns_check_state().  Errors: STATE, INVALID_ARG, CUDA, NONPHYSICAL. */
int ucns_rk_step(ucns_mesh* mesh, double* U, double* dt_inout, void* stream);

/* n_steps SSP-RK steps of U (device [5][n_cells], internal order, updated in
 * place), each with the CFL time step computed on the device, in one call:
 * the same arithmetic as n_steps calls of ucns_rk_step(dt_inout = NULL), bit
 * for bit, with less per-step work around the kernels (the mixed form carries
 * its float pair of the state from one step to the next, since nothing can
 * modify U in between).  *t_inout (host, may be NULL) is advanced by the total
 * simulated time.  Synchronises (reads the time and the error word).
 * Errors: STATE, INVALID_ARG, CUDA, NONPHYSICAL. */
int ucns_rk_steps(ucns_mesh* mesh, double* U, int32_t n_steps, double* t_inout, void* stream);

/* Host-buffer variant: copies U_host (pinned or pageable [5][n_cells], internal
 * order) to a library-owned device buffer, runs n_steps SSP-RK steps with the
 * CFL time step, copies the result back and synchronises.  *t_inout (may be
 * NULL) is advanced by the total simulated time. */
int ucns_rk_steps_host(ucns_mesh* mesh, double* U_host, int32_t n_steps, double* t_inout,
                       void* stream);

/* Read and clear the device error word written by the RK and dt kernels
 * (synchronises the stream).  UCNS_OK or UCNS_ERR_NONPHYSICAL. */
int ucns_check_state(ucns_mesh* mesh, void* stream);

/* Measured arithmetic throughput of this GPU (no counterpart in the paper;
 * the denominators of the kernels' ALU rooflines): which = 0 FP32 FMA
 * (scalar), 1 FP64 FMA, 2 FP32 FMA in packed pairs; *flops_per_s (host)
 * receives the best of three timed launches of 8 blocks per SM x 256 threads,
 * each thread running 8 independent FMA chains (an FMA = 2 flops); *n_sm
 * (may be NULL) the SM count.  Synchronises.  Errors: INVALID_ARG, CUDA. */
int ucns_alu_peak(int32_t which, double* flops_per_s, int32_t* n_sm, void* stream);

/* Exercises the give-up path of the reconstruction's bounded waits (no
 * counterpart in the paper): one thread waits about a millisecond for a phase
 * of a fresh mbarrier that nothing completes -- no copy or MMA is in flight --
 * then sets the timeout bit of the mesh's device error word, which this call
 * reads and clears.  Returns UCNS_ERR_TIMEOUT, the status a real stalled bulk
 * copy gives at the next synchronising call; a following ucns_check_state
 * returns UCNS_OK.  Errors: STATE, INVALID_ARG, CUDA. */
int ucns_probe_bounded_wait(ucns_mesh* mesh, void* stream);

/* The CFL time step of U written to device memory, allocating nothing.
 * No counterpart in the paper: this serves callers that must not allocate
 * device memory on their call path -- code running under a fixed device-memory
 * budget or a pool-only allocator, or that cannot afford cudaMalloc's implicit
 * device synchronisation -- and still need the time-step reduction.
 *  U    device [5][n_cells] float64, internal order (input).
 *  dt   device pointer to one float64 (output): CFL * min over cells, the same
 *       value as ucns_time_step.  Nothing is synchronised or copied to the host.
 * The per-block partial minima live in a file-scope device array of 32768
 * doubles (256 KiB) that every GPU which loads the library holds until the
 * process exits; meshes above 8,388,608 cells are rejected with
 * UCNS_ERR_INVALID_ARG.  The first call on a device (with that device
 * current) resolves the array's device address, so make that first call
 * before any stream capture; the address is kept for the life of the process,
 * so do not use this call after a context reset (cudaDeviceReset).  Every
 * call shares the array; each call writes the partials it reads, so nothing
 * needs clearing, but calls that overlap on
 * the GPU (e.g. on two streams) race on it.  A non-physical state sets the
 * mesh's error word as in ucns_time_step (read it with ucns_check_state).
 * Errors: INVALID_ARG, STATE, CUDA. */
int ucns_time_step_static(const ucns_mesh* mesh, const double* U, double* dt, void* stream);

/* The float pair of FP64 values as the mixed form stores its states (no
 * counterpart in the paper, which computes in FP64 only; its Sec. 7 names
 * mixed precision as future work): hi[k] = fl32(u[k]) and lo[k] =
 * fl32(u[k] - hi[k]), both rounded to nearest even, so that hi + lo carries
 * u to about 2^-48 relative and the difference of two pairs taken leading
 * part first is exact up to its final rounding.  Formed from the bit patterns
 * with one FP64 -> FP32 rounding (the routine the solver's kernels use);
 * lo = 0 where |u| < 2^-74 or hi is not a normal FP32 number.
 *  u      device [n] float64 (input);  hi, lo  device [n] float32 (output).
 *  n      >= 0.   Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
int ucns_float_pair(const double* u, float* hi, float* lo, int64_t n, void* stream);

/* Diagnostics of U (device [5][n_cells]) into *out (host).  Synchronises. */
int ucns_diagnostics(ucns_mesh* mesh, const double* U, ucns_diag* out, void* stream);

/* The CFL time step of U (device), returned in *dt (host).  Synchronises. */
int ucns_time_step(ucns_mesh* mesh, const double* U, double* dt, void* stream);

/* ---- learned troubled-cell indicator --------------------------------- */
/* A small network (32 -> 64 -> 64 -> 1, ReLU, logistic output) predicts from
 * 32 per-cell features whether a cell's CWENOZ weights depart from the linear
 * ones; gated cells keep CWENOZ, the others take the linear-weight (optimal
 * central) polynomial, which skips the directional stencils.  Weights are
 * BF16 copies of FP32 master weights; products run on the tensor cores
 * (tcgen05) with FP32 accumulation.  Parameters (FP32, flat, in order):
 * W1 [64][32], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1] = 6337 values.
 * Feature rows are BF16 [n][32], 16-byte aligned device memory. */
typedef struct ucns_mlp ucns_mlp; /* opaque, library-owned, on the current device */

#define UCNS_MLP_PARAMS 6337
#define UCNS_GATE_FEATURES 32

/* He-normal initial weights from `seed`, zero biases, Adam state zero. */
int ucns_mlp_create(uint64_t seed, ucns_mlp** out);
void ucns_mlp_destroy(ucns_mlp* mlp);
/* Copy the FP32 master weights to / from host float[UCNS_MLP_PARAMS]
 * (setting them also resets the Adam state).  Synchronous. */
int ucns_mlp_get_params(const ucns_mlp* mlp, float* theta);
int ucns_mlp_set_params(ucns_mlp* mlp, const float* theta);
/* Logits z (device float[n]) of n feature rows X (device BF16 [n][32]). */
int ucns_mlp_forward(ucns_mlp* mlp, const void* X, int64_t n, float* z, void* stream);
/* The same forward pass, also writing the first hidden layer as the second
 * layer's product reads it: h1 = bf16(relu(W1 x + b1)) (device BF16
 * [n][64], 16-byte aligned), with the logits z (device float[n]).  For
 * inspecting the network, e.g. counting where its FP32 accumulation rounds
 * h1 to the other BF16 neighbour than an exact evaluation would. */
int ucns_mlp_hidden(ucns_mlp* mlp, const void* X, int64_t n, void* h1, float* z, void* stream);
/* Gradient (device float[UCNS_MLP_PARAMS]) of the class-weighted binary
 * cross-entropy L = (1/n) sum_i c(y_i) [softplus(z_i) - y_i z_i], c(1) = w_pos,
 * c(0) = w_neg, over n rows X with labels y (device float[n], 0 or 1).
 * Deterministic (fixed reduction order).  Weights unchanged. */
int ucns_mlp_grad(ucns_mlp* mlp, const void* X, const float* y, int64_t n, float w_pos, float w_neg,
                  float* grad, void* stream);
/* Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) over consecutive
 * batches of `batch` rows (a multiple of 8) of (X, y): one step per batch.
 * Asynchronous on `stream`. */
int ucns_mlp_train(ucns_mlp* mlp, const void* X, const float* y, int64_t n, int64_t batch, float lr,
                   float w_pos, float w_neg, void* stream);
/* Read and clear the network's device error word (synchronises): UCNS_OK or
 * UCNS_ERR_TIMEOUT if a bounded tensor-core wait gave up. */
int ucns_mlp_check(ucns_mlp* mlp, void* stream);
/* Exercises the give-up path of the network's bounded mbarrier waits: one
 * thread waits about a millisecond for a phase of a fresh mbarrier that no
 * MMA commit completes (nothing is issued), sets the network's error word,
 * and ucns_mlp_check reads and clears it.  Returns UCNS_ERR_TIMEOUT; a
 * following ucns_mlp_check returns UCNS_OK.  Errors: INVALID_ARG, CUDA. */
int ucns_mlp_probe_bounded_wait(ucns_mlp* mlp, void* stream);

/* The 32 features of every cell of U (device [5][n_cells]), as BF16 rows into
 * X (device [n_cells][32], internal order) and, if Xf is not NULL, as FP32
 * into Xf (device float [n_cells][32]).  Needs order 2.  Features, from the
 * cell average and the optimal central polynomial p_opt of Eq. 4:
 * 0-17 (rho_m - rho_i)/rho_i over the central stencil; 18-23 (p_m - p_i)/p_i
 * over its first 6 members; 24-28 SI_v/(SI_v + q_v^2) for each variable, SI of
 * p_opt as in Eq. 6, q = 0.1 (rho, rho a, rho a, rho a, rho a^2); 29 |u|/a;
 * 30 h|div u|/a; 31 h|curl u|/a with h = |V|^(1/3). */
int ucns_gate_features(ucns_mesh* mesh, const double* U, void* X, float* Xf, void* stream);
/* Training labels of the plain scheme: dev[i] = max over variables and
 * stencils of |omega_s - lambda_s| for the CWENOZ weights of U (device float
 * [n_cells]); the label is dev > threshold.  Needs an FP64 CWENOZ mesh. */
int ucns_gate_labels(ucns_mesh* mesh, const double* U, float* dev, void* stream);
/* Attach a trained network (not owned; keep it alive while attached): when
 * enabled, each ucns_rk_step / ucns_residual first evaluates the features of
 * its input state and the network once, and cells with logit > threshold use
 * CWENOZ while the others use the linear weights.  mlp = NULL detaches. */
int ucns_gate_attach(ucns_mesh* mesh, ucns_mlp* mlp, float logit_threshold);
int ucns_gate_enable(ucns_mesh* mesh, int32_t enable);
/* Cadence of the gate and the plain-scheme check (the plain scheme judges
 * the gate's error).  The features and the network are evaluated at the first
 * gated step and then every eval_every-th ucns_rk_step (>= 1); the flags in
 * between are reused.  With check_every > 0, every check_every-th gated
 * ucns_rk_step first reconstructs its input state both gated and with the
 * full scheme, evaluates both residuals, and forms four measures of their
 * difference, with r_i = V_i (u_i . R_m,i - |u_i|^2 R_rho,i / 2) the cells'
 * kinetic-energy rates under each:
 *   [0] |sum r_gated - sum r_full| / |sum r_full|, the relative error of
 *       dKE/dt (ill-conditioned where dKE/dt is near zero);
 *   [1] sum |r_gated - r_full| / sum |r_full|, the local difference, which
 *       differences of opposite sign cannot hide;
 *   [2] a running estimate of the relative error the gate puts into the
 *       kinetic-energy history: each check adds |sum r_gated - sum r_full| /
 *       sum V (the difference of the volume-averaged dKE/dt) times
 *       check_every times the CFL time step of the state, divided by the
 *       volume-averaged kinetic energy (KE's drift from the full scheme's
 *       until the next check, to first order);
 *   [3] |eps_s,gated - eps_s,full| / eps_s,full, the solenoidal dissipation
 *       (ucns_diag) of the two reconstructions of the state;
 *   [4] |eps_d,gated - eps_d,full| / max(eps_d,full, 1e-3 eps_s,full), the
 *       dilatational one (against a thousandth of the solenoidal one where
 *       it is smaller: at low Mach numbers it lies below the arithmetic's
 *       resolution of the dissipation);
 *   [3] and [4] are the gate's error in the dissipation histories at that
 *   state.  The gate is switched off for the rest of the run when [2], [3] or
 * [4] exceeds `bound` (the target error of the kinetic-energy and
 * dissipation histories), or [0] exceeds bound_rate (bound_rate = 0: not
 * used).  A check
 * synchronises the stream.  check_every = 0 disables the checks.  Resets the
 * step and check counters and the running estimate.  Defaults: eval_every 1,
 * check_every 0, bound 1e-4, bound_rate 0. */
int ucns_gate_configure(ucns_mesh* mesh, int32_t eval_every, int32_t check_every, double bound,
                        double bound_rate);
/* Run one check now on U (counted as check_every steps, at least 1): the five
 * measures above into host double[5] `measures`, and *disabled (may be NULL)
 * whether the gate is now off. */
int ucns_gate_check(ucns_mesh* mesh, const double* U, double* measures, int32_t* disabled, void* stream);
/* State of the gate (host outputs, each may be NULL): *enabled whether it is
 * on (a network attached and not switched off); counts[0..2] = gated steps
 * and checks since ucns_gate_configure, and the gated step at which a check
 * switched it off (-1: none); last[0..4] = the five measures of the last
 * check (-1 before the first).  No device work. */
int ucns_gate_status(const ucns_mesh* mesh, int32_t* enabled, int64_t* counts, double* last);

/* Caller-given flags in place of the network (Sec. 2.2, Eqs. 5-6 with a
 * per-cell choice of the polynomial): flags is device uint8 [n_cells] in the
 * internal order, nonzero = the cell keeps CWENOZ, 0 = the cell takes the
 * optimal central polynomial p_opt (linear weights).  Copied on `stream`
 * (asynchronous; the caller's buffer may be reused once the stream has passed
 * this point).  While set, every ucns_residual / ucns_rk_step(s) of the mesh
 * uses these flags and neither the features, the network nor the plain-scheme
 * check run (an attached network is kept but idle); ucns_diagnostics and
 * ucns_gate_labels still use the full scheme.  flags = NULL returns to the
 * network (or to CWENOZ everywhere without one).  Lets a caller supply its
 * own troubled-cell indicator, and a test drive the gated kernels with any
 * mask.  Needs a P2 CWENOZ mesh; allocates the gate's buffers on first use.
 * Errors: STATE, INVALID_ARG, NOMEM, CUDA. */
int ucns_gate_set_flags(ucns_mesh* mesh, const uint8_t* flags, void* stream);
/* Copy the flags of the last gate evaluation (or the caller's flags) to
 * device uint8 [n_cells] `flags` (internal order), asynchronously on
 * `stream`.  Errors: STATE (no flags yet), INVALID_ARG, CUDA. */
int ucns_gate_flags(ucns_mesh* mesh, uint8_t* flags, void* stream);

/* Number of cells the last gate evaluation routed to CWENOZ (synchronises). */
int ucns_gate_flagged(ucns_mesh* mesh, int64_t* n_flagged, void* stream);

/* Opt-in per-kernel timing with CUDA events recorded on the launch stream
 * around every kernel the library enqueues (enable != 0 starts a new
 * measurement window; 0 stops recording).  ucns_profile_read synchronises on
 * the recorded events and returns, per kernel kind (0 reconstruction,
 * 1 face flux, 2 residual/RK update, 3 time step, 4 diagnostics, 5 other,
 * 6 indicator features, 7 indicator network), the summed milliseconds and
 * launch counts since the window started (host double[8], int64[8]). */
int ucns_profile(ucns_mesh* mesh, int32_t enable);
int ucns_profile_read(ucns_mesh* mesh, double* ms, int64_t* launches);

/* perm[k] = caller's cell id of internal cell k (host int64 [n_cells]). */
int ucns_cell_order(const ucns_mesh* mesh, int64_t* perm);

/* info[0..7] = n_cells, n_faces, K (modes), central stencil size,
 * directional stencils per cell, directional stencil size, face quadrature
 * points, faces per cell (host int64 [8]). */
int ucns_mesh_info(const ucns_mesh* mesh, int64_t* info);

/* Thread-local message of the last failing call on this thread. */
const char* ucns_last_error(void);

/* Free a handle and everything it owns (NULL-safe, idempotent per handle). */
void ucns_mesh_destroy(ucns_mesh* mesh);

#ifdef __cplusplus
}
#endif
#endif /* UCNS_H */
