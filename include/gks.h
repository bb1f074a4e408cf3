/* gks.h -- C ABI of the GB300 gas-kinetic solver for 3D hybrid unstructured meshes.
 *
 * The library advances the semi-discrete finite-volume system dQ_i/dt = L(Q_i)
 * (Yang, Pan & Xu, arXiv 2203.09047, Section 3.1, Eqs. semi and finite) on meshes of
 * tetrahedra, pyramids, prisms and hexahedra, with the third-order WENO reconstruction of
 * Section 2 (Eqs. weno and indicator), the time-dependent gas-kinetic flux of Section 3.2
 * (Eqs. flux-1 and flux-2) integrated over each face by the 2x2 Gauss rule of Eq. flux-qud, and
 * the two-stage fourth-order time discretisation of Section 3.3.
 *
 * Conventions shared by every call:
 *  - Every call returns a gks_status; GKS_OK is 0. gks_last_error gives a text for the last
 *    failure of a solver. Nothing is thrown across the ABI.
 *  - Host arrays passed in are copied; the caller keeps ownership.
 *  - State arrays are float64, structure of arrays [5][n_cells] (rho, rho U, rho V, rho W, rho E),
 *    in the caller's cell order. Unless a call says otherwise they may be host or device
 *    pointers (unified addressing decides); device pointers must be on the solver's device.
 *    The library never frees or keeps caller pointers beyond a call.
 *  - All device work is enqueued on the stream given to gks_init; calls that return values to
 *    the host (gks_max_dt, status checks) synchronise that stream.
 *  - A solver is not thread-safe. Results are bit-reproducible for a fixed mesh, parameters
 *    and device: cell sums run in a fixed face order and no floating-point atomics are used.
 */
#ifndef GKS_H
#define GKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GKS_OK = 0,
  GKS_E_INVAL = 1,       /* bad argument */
  GKS_E_NOMEM = 2,       /* device or host allocation failed */
  GKS_E_CUDA = 3,        /* a CUDA runtime call failed */
  GKS_E_MESH = 4,        /* non-conforming, inverted or unmatched cell/face */
  GKS_E_SINGULAR = 5,    /* a stencil least-squares system is rank deficient */
  GKS_E_NONPHYSICAL = 6, /* rho <= 0, p <= 0 or NaN in a state or a reconstructed value */
  GKS_E_TIMEOUT = 7      /* a bounded device wait gave up (reported by the status checks) */
} gks_status;

typedef struct gks_mesh gks_mesh;     /* opaque: topology, stencils, cell order */
typedef struct gks_solver gks_solver; /* opaque: device geometry, buffers, state */

/* Cell kinds: the value is the number of distinct vertices. */
enum { GKS_TET = 4, GKS_PYR = 5, GKS_PRI = 6, GKS_HEX = 8 };
/* Boundary condition per axis of the bounding box: periodic; slip (reflecting) walls; no-slip
 * walls (Section 5: adiabatic or isothermal, possibly moving; their velocity and temperature are
 * solver parameters, wall_u and wall_T below); far field by Riemann invariants (Section 5.4;
 * the far-field state is the solver parameter farfield). */
enum { GKS_BC_PERIODIC = 0, GKS_BC_REFLECT = 1, GKS_BC_NOSLIP = 2, GKS_BC_FARFIELD = 3 };
/* Flux variants (Section 3.2): the smooth flux of Eq. flux-2 read as
 * g0 [1 - tau (a.u + A) + t A], or the full flux of Eq. flux-1. */
enum { GKS_FLUX_SMOOTH = 0, GKS_FLUX_FULL = 1 };
/* Collision time (Section 5): zero; inviscid tau = eps dt + C |pl-pr|/(pl+pr) dt;
 * viscous tau = mu/p + C |pl-pr|/(pl+pr) dt with p the interface pressure; viscous with the
 * power law of Section 5.4, mu(T) = mu (T/T_ref)^mu_pow with T = p/rho of the interface
 * equilibrium. */
enum { GKS_TAU_ZERO = 0, GKS_TAU_INVISCID = 1, GKS_TAU_VISCOUS = 2, GKS_TAU_POWER_LAW = 3 };
/* Arithmetic: GKS_PREC_FP64, FP64 everywhere. GKS_PREC_MIXED: FP32 reconstruction and flux
 * with the state, the stencil differences, the face sums and the two-stage update in float-float
 * arithmetic (each value an unevaluated sum of two FP32 numbers, about 48 significant bits;
 * error-free TwoSum and FMA TwoProduct), which conserves mass, momentum and energy to about
 * 2^-46 relative per update and executes no FP64 instruction on the hot path.
 * GKS_PREC_MIXED_FP64UPD: the same FP32 reconstruction and flux, with FP64 face sums and the
 * FP64 two-stage update of an FP64 state (the reconstruction reads its float-pair copy);
 * gks_step keeps that state in FP64 throughout (gks_step_implicit updates the float-pair copy,
 * as in GKS_PREC_MIXED). */
enum { GKS_PREC_FP64 = 0, GKS_PREC_MIXED = 1, GKS_PREC_MIXED_FP64UPD = 2 };

typedef struct {
  double gamma;      /* specific heat ratio; K = (5 - 3 gamma)/(gamma - 1) internal dofs */
  double mu;         /* dynamic viscosity (0: Euler) */
  double Pr;         /* Prandtl number; 1 is the BGK value. Other values apply the heat-flux
                        correction of the BGK-NS scheme (energy flux + (1/Pr - 1) q, q the heat
                        flux of the interface distribution), smooth flux only; the VJP
                        supports Pr = 1 only */
  int flux_mode;     /* GKS_FLUX_* */
  int tau_model;     /* GKS_TAU_* */
  double tau_eps;    /* eps of the inviscid collision time (Section 5: 0.01) */
  double tau_C;      /* C of the pressure-jump term (Section 5: 1) */
  double weno_gamma; /* linear weight of each sub-stencil (Section 2: 0.0125) */
  double weno_eps;   /* epsilon of the nonlinear weights (not printed; default 1e-8) */
  int weno_pow;      /* exponent of tau/(beta+eps) in the nonlinear weights (printed: 1) */
  int precision;     /* GKS_PREC_* */
  double T_ref;      /* GKS_TAU_POWER_LAW: reference temperature p/rho (> 0) */
  double mu_pow;     /* GKS_TAU_POWER_LAW: exponent (Section 5.4: 0.7) */
  /* No-slip walls, per plane axis + 3 side (side 1 the upper plane of the axis): velocity and
   * temperature p/rho (<= 0: adiabatic). The ghost at a wall's Gauss points has the owner's
   * density, U_g = 2 U_w - U and p_g = p (adiabatic) or T_g = 2 T_w - T (isothermal); ghost cells
   * in the stencils take U_g = 2 U_w - U at the same density and pressure. The wall flux has no
   * mass component; at an adiabatic wall its energy component is U_w . (momentum flux). Ignored
   * on periodic and slip planes. */
  double wall_u[6][3];
  double wall_T[6];
  /* Far-field planes: the state (rho, U, V, W, p) outside. The ghost at a far-field plane, in
   * the stencils and at the Gauss points, is the characteristic boundary state: the outgoing
   * invariant u_n + 2c/(gamma-1) from inside, the incoming u_n - 2c/(gamma-1) from this state,
   * entropy and tangential velocity from the upwind side (supersonic inflow: this state,
   * supersonic outflow: the inside state); it carries no gradient at the Gauss points. One state
   * per plane (axis + 3 side), default (1, 0, 0, 0, 1/1.4). */
  double farfield[6][5];
  /* Positivity fallback at the Gauss points (not in the paper, which prints no positivity
   * treatment; off by default): with gp_fallback != 0, a side whose reconstructed state at a face
   * Gauss point has rho <= 0 or p <= 0 (or NaN) takes its cell average with a zero gradient,
   * the first-order state, before any wall ghost is formed from it. The face flux stays one
   * value per face, so conservation is kept. Off: such a state stops the step with
   * GKS_E_NONPHYSICAL (the paper's method as printed). gks_residual_vjp differentiates the
   * fallback: the cotangent of a side that fell back goes to its cell average. */
  int gp_fallback;
} gks_params;

/* Fill *p with the defaults above (gamma 1.4, Euler, smooth flux, zero collision time,
 * weno_gamma 0.0125, weno_eps 1e-8, weno_pow 1, FP64, T_ref 1, mu_pow 0.7, stationary
 * adiabatic walls, far field at rest with rho 1 and p 1/1.4, no Gauss-point fallback). */
void gks_params_default(gks_params* p);

/* Build the mesh topology on the host.
 *   xyz        [n_nodes][3] node coordinates.
 *   cell_type  [n_cells] GKS_TET/PYR/PRI/HEX.
 *   cell_nodes [n_cells][8] node indices in the degenerate-hexahedron slots of Section 2:
 *              tet {p1 p2 p3 p3 p4 p4 p4 p4}, pyramid {p1 p2 p3 p4 p5 p5 p5 p5},
 *              prism {p1 p2 p3 p3 p4 p5 p6 p6}, hex {p1..p8}; the face labels F_p of Section 2
 *              (prism F3 read as {p1 p2 p5 p4}) fix the sub-stencils.
 *   bc, lo, hi the bounding box [lo, hi] and a condition per axis. Faces on a periodic axis
 *              match their translated image; unmatched faces must lie on a wall plane (slip or
 *              no-slip axis).
 * Builds faces, the big stencils S_i (face neighbours, then neighbours of neighbours, as a set
 * of (cell, periodic/mirror transform) pairs) and the sub-stencils of Section 2, and a
 * Morton reorder of cells used internally. Errors: GKS_E_INVAL (bad type/index),
 * GKS_E_MESH (face shared by more than two cells, unmatched face off a reflecting plane,
 * periodic vertices not related by one translation), GKS_E_NOMEM. *out is NULL on error. */
gks_status gks_mesh_create(int64_t n_nodes, const double* xyz, int64_t n_cells,
                           const int8_t* cell_type, const int64_t* cell_nodes, const int bc[3],
                           const double lo[3], const double hi[3], gks_mesh** out);

/* Cell order inside the library (the caller's order is kept at the ABI): cells are grouped by
 * kind, then ordered by the caller's index, the Morton code of the vertex mean (default), or the
 * reverse Cuthill-McKee order of the face graph. */
enum { GKS_REORDER_NONE = 0, GKS_REORDER_MORTON = 1, GKS_REORDER_RCM = 2 };
typedef struct {
  int reorder;     /* GKS_REORDER_* */
  int min_stencil; /* 0: the big stencil of Section 2 as printed (face neighbours and their face
                      neighbours). n > 0 (a reading, not in the paper; at most 64): a big stencil
                      with fewer than n members takes the face neighbours of its members, member
                      by member in stencil order and face by face in face-label order, until it
                      has n members (images across more than two wall planes are skipped). On the
                      layered hybrid generator, whose transition layers hold six pyramids sharing
                      the cube centre and the split-pyramid tetrahedra, the printed stencils give
                      a linearly unstable reconstruction; 18 (twice the nine unknowns of the
                      quadratic) removes the instability. */
} gks_mesh_options;

/* gks_mesh_create with options (opt = NULL: GKS_REORDER_MORTON, min_stencil 0). Errors as
 * gks_mesh_create, and GKS_E_INVAL for an unknown reorder or min_stencil outside [0, 64]. */
gks_status gks_mesh_create_ex(int64_t n_nodes, const double* xyz, int64_t n_cells,
                              const int8_t* cell_type, const int64_t* cell_nodes, const int bc[3],
                              const double lo[3], const double hi[3],
                              const gks_mesh_options* opt, gks_mesh** out);

/* Counts of a built mesh: cells, faces, total stencil entries. */
gks_status gks_mesh_counts(const gks_mesh* m, int64_t* n_cells, int64_t* n_faces,
                           int64_t* n_stencil);

/* Last mesh-construction error text (valid until the next gks_mesh_create on this thread). */
const char* gks_mesh_last_error(void);

/* Create a solver on the current CUDA device: copies the mesh to the device, computes in FP64
 * the cell and face quadrature (27-point trilinear, Section 2; 2x2 bilinear, Eq. flux-qud), the
 * least-squares pseudo-inverses of every big stencil and sub-stencil, and stores them in the
 * precision of p->precision. `stream` is a cudaStream_t (NULL: the legacy default stream) on
 * which every later call enqueues its work. The mesh may be destroyed afterwards.
 * With moving no-slip walls or far-field planes it also sets up the ghost cells of the stencil
 * images whose flow variables are not a sign change of their source cell (refreshed before
 * every reconstruction).
 * Errors: GKS_E_INVAL (params: gamma, mu, Pr, the modes, the WENO constants, T_ref > 0 for the
 * power law, finite wall data, far-field states with rho > 0 and p > 0), GKS_E_MESH (inverted
 * cell; too many ghost cells for the stencil entry format), GKS_E_SINGULAR (rank-deficient
 * stencil), GKS_E_NOMEM, GKS_E_CUDA. */
gks_status gks_init(const gks_mesh* m, const gks_params* p, void* stream, gks_solver** out);

/* Copy a state [5][n_cells] (caller order, host or device) into the solver. */
gks_status gks_set_state(gks_solver* s, const double* Q);
/* Copy the solver's state out to [5][n_cells] (caller order, host or device).
 * State, time and step count are the whole checkpoint: with GKS_PREC_FP64 and
 * GKS_PREC_MIXED_FP64UPD (FP64 state) a run resumed from it by gks_set_state continues bit for
 * bit. GKS_PREC_MIXED keeps the state as float-float pairs; their FP64 form rounds a pair whose
 * parts lie more than 53 bits apart, so a resumed run agrees with the uninterrupted one to the
 * mixed path's precision, not bit for bit. */
gks_status gks_get_state(gks_solver* s, double* Q);

/* Largest stable step for the current state: cfl * min_i h_i / (|U_i| + c_i + 2 mu/(rho_i h_i)),
 * h_i = |Omega_i| / (largest face area of cell i). Synchronises the stream.
 * Errors: GKS_E_NONPHYSICAL. */
gks_status gks_max_dt(gks_solver* s, double cfl, double* dt);

/* The 27-point quadrature of every cell (3 Gauss-Legendre points per direction mapped by the
 * trilinear map of Eq. trilinear, Section 2), for cell averages of given fields (initial data,
 * exact solutions) and volume-weighted norms: xq [n_cells][27][3] points, wq [n_cells][27]
 * weights times |J| (they sum to the cell volume), caller order, host or device pointers.
 * Uses temporary device memory and synchronises the stream. */
gks_status gks_cell_quadrature(gks_solver* s, double* xq, double* wq);

/* Advance the solver's state by nsteps two-stage fourth-order steps of size dt (Section 3.3):
 *   Q*      = Q^n + dt/2 L(Q^n) + dt^2/8 Lt(Q^n)
 *   Q^{n+1} = Q^n + dt L(Q^n) + dt^2/6 (Lt(Q^n) + 2 Lt(Q*))
 * where L and Lt = dL/dt come from the time-dependent face flux fitted on [0, dt/2] and [0, dt].
 * Asynchronous on the solver's stream; a non-physical state is reported by gks_check. */
gks_status gks_step(gks_solver* s, double dt, int nsteps);

/* Synchronise the stream and report GKS_E_NONPHYSICAL if any earlier step or residual met
 * rho <= 0, p <= 0 or NaN (the device flag is then cleared). */
gks_status gks_check(gks_solver* s);

/* Test hook for the bounded wait of the reconstruction (the paper has no counterpart): every
 * later reconstruction of this solver waits for its mbarrier (completed by the bulk copy of the
 * sub-stencil entries into shared memory, where a range stages them) at most wait_tries tries
 * per wait (0: the library default of 2^22), and with withhold_copies != 0 issues no copy and
 * expects 16 bytes more than the copies bring, so the barrier never completes, every block
 * gives up after its tries with nothing in flight, and the next status check (gks_check,
 * gks_residual) returns GKS_E_TIMEOUT, in every precision. The reconstruction's output is then
 * undefined; gks_debug_recon_wait(s, 0, 0) restores normal operation.
 * Errors: GKS_E_INVAL (s NULL, wait_tries < 0). */
gks_status gks_debug_recon_wait(gks_solver* s, int wait_tries, int withhold_copies);

/* The two stage combinations of gks_step (Section 3.3) on caller arrays, for a rollout built
 * from gks_residual calls (a differentiable rollout, or a caller's own stepping):
 *   stage 1: out = Q + dt/2 L + dt^2/8 Lt              (Lts is not read; may be NULL)
 *   stage 2: out = Q + dt L + dt^2/6 (Lt + 2 Lts)
 * Q, L, Lt, Lts, out: device pointers to n float64 values each (any layout, the same for all;
 * out may alias Q); enqueued on `stream` (a cudaStream_t, NULL the legacy stream), not
 * synchronised. Errors: GKS_E_INVAL (stage not 1 or 2, dt <= 0, n < 0, a missing array), with a
 * message in gks_last_error(NULL); GKS_E_CUDA. */
gks_status gks_s2o4_stage(int64_t n, int stage, double dt, const double* Q, const double* L,
                          const double* Lt, const double* Lts, double* out, void* stream);
/* The transpose of gks_s2o4_stage: for a cotangent g of out, gQ = g, gL = c1 g, gLt = c2 g and
 * (stage 2) gLts = 2 c2 g, with c1, c2 = dt/2, dt^2/8 (stage 1) or dt, dt^2/6 (stage 2). Device
 * pointers to n float64 values; gLts is not written in stage 1 (may be NULL). Same errors. */
gks_status gks_s2o4_stage_vjp(int64_t n, int stage, double dt, const double* g, double* gQ,
                              double* gL, double* gLt, double* gLts, void* stream);

/* nsteps implicit steps for steady problems (Section 4, Jacobi iteration): per step the
 * residual averaged over [0, dt], |Omega_i| Res_i = -sum_f s_f int_0^dt F_f dt / dt (the
 * reconstruction and flux of gks_step), then the backward-Euler system with the residual's
 * change linearised by the flux splitting (T(Q_i) + T(Q_p) - r_f (Q_p - Q_i))/2 . n S:
 *   (|Omega_i|/dt + 1/2 sum_f r_f S_f) dQ_i + 1/2 sum_f [T_n(Q_p + dQ_p) - T_n(Q_p) - r_f dQ_p] S_f
 *     = |Omega_i| Res_i,
 * solved by kmax >= 1 Jacobi iterations from dQ^(0) = |Omega_i| Res_i / D_i, and
 * Q^{n+1} = Q^n + dQ^(kmax). T_n is the Euler flux through the face (n out of cell i, S the
 * face area), r_f = max over both sides of |U . n| + c at Q^n; a wall face couples a cell to
 * its mirror image. The first call allocates the step's buffers (face normals, residual,
 * diagonal, two iterates). Errors: GKS_E_INVAL (dt <= 0, nsteps < 0, kmax < 1), GKS_E_NOMEM,
 * GKS_E_CUDA; non-physical states are reported by gks_check. */
gks_status gks_step_implicit(gks_solver* s, double dt, int nsteps, int kmax);

/* Evaluate L(Q) and its time derivative Lt for a given state Q (Eq. finite):
 *   L_i  = -(1/|Omega_i|) sum_f s_if F_f^n,   Lt_i = -(1/|Omega_i|) sum_f s_if dF_f/dt,
 * F^n = (4 F(dt/2) - F(dt))/dt and dF/dt = 4 (F(dt) - 2 F(dt/2))/dt^2 from the time integrals
 * F(delta) of the face flux. Q, L, Lt are [5][n_cells] in caller order, host or device.
 * Does not change the solver's state. Synchronises the stream and returns GKS_E_NONPHYSICAL
 * for a non-physical state or reconstructed value. */
gks_status gks_residual(gks_solver* s, const double* Q, double dt, double* L, double* Lt);

/* Vector-Jacobian product of gks_residual at Q for a fixed dt:
 *   gQ = (dL/dQ)^T gL + (dLt/dQ)^T gLt,
 * all [5][n_cells] float64 in caller order, host or device. Hand-written reverse of the face
 * sums, the gas-kinetic flux (Eqs. flux-1/flux-2 with the collision-time models of Section 5),
 * the Gauss-point evaluation and the WENO reconstruction (least squares, smoothness indicators
 * and nonlinear weights of Section 2, the derivative of |x| taken as sign(x) with +1 at 0), in
 * FP64 regardless of the solver's precision; deterministic (per-face and per-cell writes,
 * reverse-stencil gathers, no atomics). The first call allocates the adjoint buffers (and, for
 * a mixed-precision solver, an FP64 copy of the geometry). The flux adjoint keeps up to 1.7 KB
 * of stack per thread: when the context's per-thread stack limit (cudaLimitStackSize) is
 * smaller, the call raises it, which reserves local memory for every resident thread of the
 * context for as long as the context lives and may synchronise the device. Synchronises the
 * stream; returns GKS_E_NONPHYSICAL for a non-physical state. */
gks_status gks_residual_vjp(gks_solver* s, const double* Q, double dt, const double* gL,
                            const double* gLt, double* gQ);

/* Per-kernel timing for benchmarks and traces (a utility of this library; the paper has no
 * counterpart). With enable != 0 every later hot-path launch is
 * bracketed by CUDA events on the solver's stream. gks_timing_read synchronises the stream and
 * returns, for the kinds 0 reconstruction, 1 face flux, 2 face sum + update, the summed device
 * milliseconds and the number of launches since the last read, then resets them. */
gks_status gks_timing_enable(gks_solver* s, int enable);
gks_status gks_timing_read(gks_solver* s, double ms[3], int64_t counts[3]);

/* Algorithmic bytes (a utility of this library; the paper has no counterpart) of one pass of
 * each hot kernel over the mesh (0 reconstruction, 1 face flux,
 * 2 face sum + update as in a two-stage step) for this solver's mesh and precision: every array
 * the kernel must read or write counted once (re-reads through the caches are not counted). */
gks_status gks_kernel_bytes(const gks_solver* s, double bytes[3]);

/* Kernel launches (a utility of this library; the paper has no counterpart) in one pass of
 * each hot kernel (0 reconstruction: one launch per range of
 * tiles of one cell kind, plus the ghost refresh when moving no-slip walls need ghost cells;
 * 1 face flux; 2 face sum + update), for counting the launches of a timed region from the pass
 * counts of gks_timing_read. */
gks_status gks_launches_per_pass(const gks_solver* s, int64_t launches[3]);

/* Algorithmic operation count (a utility of this library; the paper has no counterpart) of one
 * face Gauss point of the flux kernel for a flux mode and
 * collision-time model: *flops counts +, -, *, / (an FMA as two), *special counts exp, erfc and
 * sqrt. Computed on the host by running the kernel's own templated arithmetic with a counting
 * scalar type. Returns 0 on success. Not thread-safe. */
int gks_flux_opcount(int flux_mode, int tau_model, double* flops, double* special);

/* Measured FP32 and FP64 FMA throughput of the current device in TFLOP/s (an FMA counts as two
 * flops): independent FMA chains in every thread of a grid of several waves, timed with CUDA
 * events on an internal stream; the denominators of the ALU-bound flux rooflines. A utility of
 * this library (the paper has no counterpart). Allocates and frees 8 bytes of device memory
 * and synchronises the device's work on its own stream. Errors: GKS_E_INVAL, GKS_E_CUDA (text in
 * gks_last_error(NULL)). */
gks_status gks_alu_peaks(double* fp32_tflops, double* fp64_tflops);

/* Allocation-free CFL time-step bound, for callers that cannot call cudaMalloc: processes
 * whose device memory is owned by another allocator (a framework pool that has reserved the
 * device) or latency-critical loops that must not pay for cudaMalloc's implicit device
 * synchronisation. The paper has no counterpart; it is the time-step reduction of gks_max_dt
 * written as a stand-alone call whose scratch is a fixed array inside the library. Its viscosity
 * mu is one constant, so it equals gks_max_dt for the collision-time models with constant
 * viscosity and not for GKS_TAU_POWER_LAW, whose bound uses mu(T) of each cell.
 *   n_cells  number of cells, at most 16,777,216 (65,536 blocks of 256 cells: the scratch holds
 *            one 8-byte partial minimum per block, 512 KiB per device); larger n is rejected with
 *            GKS_E_INVAL and a message in gks_last_error(NULL).
 *   Q        device pointer, float64 [5][n_cells] conserved variables (any cell order).
 *   h        device pointer, float64 [n_cells] length of each cell in the same order (the solver
 *            uses |Omega_i| / largest face area).
 *   dt       device pointer to one float64: receives cfl * min_i h_i / (|U_i| + c_i +
 *            2 mu / (rho_i h_i)), or -1 if any cell has rho <= 0, p <= 0 or NaN (each tested on the
 *            primitive itself, before the bound is formed).
 *   stream   cudaStream_t on which both kernels are enqueued; the call does not synchronise.
 * It calls no cudaMalloc, cudaFree or allocating library routine. The first call on a device
 * looks up the device address of the scratch array (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture. Every call on a device shares the
 * one scratch array, so calls whose kernels overlap on the GPU (different streams, no ordering)
 * race on it; order them on one stream. The looked-up address is kept per device ordinal for
 * the life of the process: the call assumes the runtime's primary context of that device and no
 * cudaDeviceReset between calls. Returns GKS_OK once both kernels are enqueued. */
gks_status gks_cfl_dt_noalloc(int64_t n_cells, const double* Q, const double* h, double gamma,
                              double mu, double cfl, double* dt, void* stream);

/* Domain decomposition for several ranks (one process per GPU; a plan, the caller moves the
 * data). The paper runs one GPU. The cells are split into nranks contiguous ranges of the
 * Morton order of their vertex means (the first n_cells % nranks ranks take one cell more). A
 * rank's residual (Eq. finite) reads the reconstruction polynomials of its cells and of their
 * face neighbours, and each polynomial its big stencil (Section 2), so the rank's halo is every
 * other cell in {j} + stencil(j) for j in {i} + face neighbours(i), i owned (up to three face
 * rings). A two-stage step exchanges the halo twice (Q^n and Q*), and the time step is the
 * minimum over the ranks. Cell ids are the caller's. Errors: GKS_E_INVAL (nranks < 1, rank out
 * of range, more ranks than cells), GKS_E_NOMEM. The mesh may be destroyed afterwards. */
typedef struct gks_partition gks_partition;
gks_status gks_partition_create(const gks_mesh* m, int nranks, int rank, gks_partition** out);
/* Number of owned and halo cells of this rank. */
gks_status gks_partition_counts(const gks_partition* p, int64_t* n_owned, int64_t* n_halo);
/* Owned cells (Morton order), halo cells sorted by (owning rank, id) and their owning ranks;
 * arrays of the counts' sizes, any may be NULL. */
gks_status gks_partition_cells(const gks_partition* p, int64_t* owned, int64_t* halo,
                               int32_t* halo_owner);
/* The owned cells that rank `peer` holds in its halo, in that rank's halo order (cells = NULL:
 * only *n); the peer receives them into its halo entries owned by this rank, in order. */
gks_status gks_partition_send(const gks_partition* p, int peer, int64_t* n, int64_t* cells);
void gks_partition_destroy(gks_partition* p);

/* Text of the solver's last error (s = NULL: the last mesh-construction or stand-alone-call
 * error on this thread). */
const char* gks_last_error(const gks_solver* s);

void gks_destroy(gks_solver* s);
void gks_mesh_destroy(gks_mesh* m);

#ifdef __cplusplus
}
#endif

#endif /* GKS_H */
