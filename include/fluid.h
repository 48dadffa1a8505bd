/*
 * fluid.h -- C ABI of the GB300 finite-volume compressible Navier-Stokes solver.
 *
 * The library computes the semi-discrete right-hand side R = dU/dt of the compressible
 * Navier-Stokes equations (paper Section 2.1, Eq. NSE and Eq. ODE) for a cell-averaged state on a
 * structured Cartesian grid, uniform or tanh-stretched per axis, and advances it with an explicit
 * TVD Runge-Kutta scheme (Section 2.1).  Convective face fluxes come from WENO5 reconstruction of
 * the primitive variables and the HLLC Riemann solver (Section 2.1, Section 3.1); dissipative
 * fluxes (Newtonian stress with the Stokes hypothesis, Fourier heat flux; Section 2.1) from
 * fourth-order central differences.  Boundary conditions assign halo cells (Section 3.2):
 * periodic, zero-gradient, isothermal or adiabatic no-slip wall, the disturbance ("porous") wall
 * with one wall-normal transpiration parameter per wall cell, and a Dirichlet inflow profile.
 *
 * Conventions common to every entry point
 *   - State arrays are device pointers to FP64 structure-of-arrays data U[5][pz][py][px] with
 *     x fastest, variables (rho, rho u, rho v, rho w, E).  Every active axis a (a < ndim) carries
 *     FLUID_HALO = 3 halo cells per side: p_a = n_a + 6; inactive axes have n_a = 1, p_a = 1.
 *     The caller owns these buffers; they must be 8-byte aligned and must not alias unless stated.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  All work is
 *     enqueued asynchronously on it; nothing synchronises unless the function says so.
 *   - Every function returns a fluid_status.  Nothing throws across the ABI.  On failure the
 *     message of fluid_last_error() says why.  A CUDA launch error is returned as FLUID_ECUDA by the
 *     call that detects it (errors of asynchronous work surface at the next synchronising call).
 *   - The solver object is not thread-safe: one host thread at a time per solver.
 *   - The library allocates device memory only in fluid_create (scratch owned by the solver,
 *     released by fluid_destroy).
 */
#ifndef FLUID_H
#define FLUID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLUID_ABI_VERSION 1
#define FLUID_HALO 3

typedef enum fluid_status {
  FLUID_OK = 0,
  FLUID_EINVAL = 1,      /* invalid argument or configuration */
  FLUID_ENOMEM = 2,      /* device allocation failed */
  FLUID_ECUDA = 3,       /* a CUDA runtime call failed */
  FLUID_ENONFINITE = 4,  /* a state value became NaN/Inf, or a wall ghost temperature <= 0 */
  FLUID_ETIMEOUT = 5,    /* a bounded wait ran out */
  FLUID_EBUSY = 6,       /* resource temporarily unavailable */
  FLUID_EBUDGET = 7,     /* request exceeds the memory budget */
  FLUID_ENOTSUP = 8      /* configuration recognised but not supported by this build */
} fluid_status;

/* boundary kinds (per axis and side) -- halo assignment of Section 3.2 */
enum {
  FLUID_BC_PERIODIC = 0,
  FLUID_BC_ZERO_GRADIENT = 1, /* transmissive: halo = first interior cell */
  FLUID_BC_WALL = 2,          /* isothermal no-slip: mirrored velocity, T_ghost = 2 T_w - T, same p */
  FLUID_BC_ADIABATIC = 3,     /* adiabatic no-slip: mirrored velocity, same rho and p */
  FLUID_BC_POROUS = 4,        /* isothermal no-slip with wall-normal transpiration v_w,i (below) */
  FLUID_BC_INFLOW = 5,        /* Dirichlet: fixed primitive profile (fluid_set_inflow) */
  FLUID_BC_EXCHANGE = 6       /* sub-domain face of a block decomposition (Section 2.2): the three
                                 halo layers of U hold the neighbouring sub-domain's cells, written
                                 by fluid_unpack_halo, and are read as they are */
};
/* grid mapping per axis: face coordinate x(eta), eta = index / n */
enum {
  FLUID_STRETCH_UNIFORM = 0,
  FLUID_STRETCH_TANH2 = 1,    /* x = lo + (hi-lo)/2 (1 + tanh(beta (2 eta - 1)) / tanh beta) */
  FLUID_STRETCH_TANH1 = 2     /* x = lo + (hi-lo) (1 - tanh(beta (1 - eta)) / tanh beta) */
};
enum { FLUID_VISC_NONE = 0, FLUID_VISC_CONSTANT = 1, FLUID_VISC_POWER = 2, FLUID_VISC_SUTHERLAND = 3 };
/* Reconstruction of the face states (config field `weno`): WENO5-JS, WENO5-Z, or the paper's
 * channel scheme TENO6-A with its interpolation limiter (Sec. 3.1; FP64 path only). */
enum { FLUID_WENO_JS = 0, FLUID_WENO_Z = 1, FLUID_TENO6A = 2 };
enum { FLUID_PREC_FP64 = 0, FLUID_PREC_MIXED = 1 };

/*
 * Configuration of one solve.  Versioned by struct_size (set it to sizeof(fluid_config)).
 *   ndim           1, 2 or 3; axes a >= ndim are inactive (n[a] == 1)
 *   n[a]           interior cells per axis (active axes: 3 .. 2^20); the product of the padded
 *                  sizes must stay below 2^31 / 9 (FP64), 2^31 / 12 (mixed) and 2^31 / 36 (adjoint)
 *                  so that the kernels' 32-bit row * cells + cell indices cannot overflow
 *   lo, hi         domain extent per axis (face coordinates of the boundaries), hi > lo
 *   stretch, beta  grid mapping per axis (beta > 0 for the tanh mappings)
 *   bc[a][side]    boundary kind for side 0 (low) and 1 (high); periodic must pair with periodic
 *   t_wall[a][s]   wall temperature for FLUID_BC_WALL / FLUID_BC_POROUS faces
 *   gamma, gas_R   ideal gas: p = (gamma - 1)(E - rho |u|^2 / 2), T = p / (rho R)
 *   prandtl        lambda = mu c_p / Pr, c_p = gamma R / (gamma - 1)
 *   visc_law       mu(T): constant mu_ref; power mu_ref (T/T_ref)^visc_exp;
 *                  Sutherland mu_ref (T/T_ref)^1.5 (T_ref + suth_S) / (T + suth_S); NONE = Euler
 *   weno, weno_eps WENO5-JS (eps default 1e-6) or WENO5-Z (q = 2, eps default 1e-40); eps <= 0
 *                  selects the default
 *   body_force     constant force per unit volume f; source S = (0, f, f . u)
 *   cfl, dt_fixed  dt = cfl * min(dx/(|u|+c), dx^2/(2 max(4/3, gamma/Pr) mu/rho)) over cells and
 *                  active axes, or dt_fixed when > 0
 *   precision      FLUID_PREC_FP64: all arithmetic in FP64.  FLUID_PREC_MIXED: WENO5 weights and
 *                  reconstruction, HLLC wave speeds and star correction, and the dissipative
 *                  stencils in FP32, in a delta form (FP64 cell differences rounded once, face
 *                  flux = FP64 cell-centre Euler flux + FP32 increment); the state, primitive
 *                  conversion, face-flux assembly, flux differences and RK3 combination stay FP64
 *   porous_*       porous strip on face (porous_axis, porous_side), which must have kind
 *                  FLUID_BC_POROUS: wall cells porous_begin .. porous_begin + porous_count - 1 along
 *                  the first other active axis carry v_w,i = (A / phi0) phi_i sin(2 pi kappa x_i)
 *                  (Section 3.2's disturbance v = A sin(2 pi kappa x) when phi_i = phi0); where
 *                  that axis has an exchange face the strip may extend into its 3 halo cells (the
 *                  neighbouring block's wall cells, which the block's corner ghost cells need)
 *   adjoint        nonzero: allocate the adjoint scratch (about 92 doubles per padded cell) so
 *                  that the fluid_adjoint_* entry points and fluid_wall_heat_loss can be used
 */
typedef struct fluid_config {
  uint32_t struct_size;
  int32_t ndim;
  int32_t n[3];
  int32_t stretch[3];
  int32_t bc[3][2];
  int32_t visc_law;
  int32_t weno;
  int32_t precision;
  int32_t porous_axis, porous_side, porous_begin, porous_count;
  double lo[3], hi[3], beta[3];
  double t_wall[3][2];
  double gamma, gas_R, prandtl;
  double mu_ref, T_ref, visc_exp, suth_S;
  double weno_eps;
  double body_force[3];
  double cfl, dt_fixed;
  double porous_A, porous_kappa, porous_phi0;
  int32_t adjoint;          /* nonzero: also allocate the scratch of the adjoint entry points */
  int32_t visc_order;       /* central differences of the dissipative fluxes: 4 (or 0), or 6 as in
                               the paper's channel computation (FP64 path only, no adjoint) */
  /* Placement of this solve as one block of a decomposed global grid (Section 2.2 splits the
   * domain into blocks, one per device).  global_n[a] == 0: axis a is not split (offset[a] == 0).
   * Otherwise the grid mapping of axis a is that of global_n[a] cells on [lo[a], hi[a]], and this
   * block holds its cells offset[a] .. offset[a] + n[a] - 1, so that its centres, widths and
   * metrics are bitwise those of the global grid at the same cells. */
  int32_t global_n[3];
  int32_t offset[3];
} fluid_config;

typedef struct fluid_solver fluid_solver; /* opaque; owned by the library */

/* Validate cfg and create a solver on the current CUDA device; allocates the solver's scratch
 * (primitive and gradient fields, stage buffer, face-flux accumulator, grid metrics).
 * Errors: FLUID_EINVAL (bad cfg, out == NULL), FLUID_ENOMEM, FLUID_ECUDA. */
int fluid_create(const fluid_config* cfg, fluid_solver** out);

/* Release the solver and its scratch (synchronises the device first).  NULL is a no-op. */
void fluid_destroy(fluid_solver* s);

/* Message of the last failure on s, or of the last failed fluid_create when s == NULL. */
const char* fluid_last_error(const fluid_solver* s);

/* Padded sizes p[0..2] (x, y, z) of the state arrays; cells = p0 p1 p2 per variable. */
int fluid_padded_dims(const fluid_solver* s, int32_t p[3]);

/* Copy the grid of axis a (0..2) to host arrays of length p[a]: cell centres xc and widths dx
 * (face-coordinate differences).  Either pointer may be NULL. */
int fluid_get_grid(const fluid_solver* s, int axis, double* xc, double* dx);

/* Set the porous-wall parameters phi[0..n-1] (device pointer, n == porous_count) and recompute the
 * wall transpiration velocities v_w on `stream`.  Until called, phi_i = phi0. */
int fluid_set_wall_params(fluid_solver* s, const double* phi_dev, int n, void* stream);

/* Set the Dirichlet inflow profile of face (axis, side) from device memory: primitives
 * (rho, u, v, w, p) shaped [5][T2][T1], T1/T2 the padded sizes of the lower/higher other axis,
 * count = 5 * T1 * T2 doubles; copied into solver storage on `stream`. */
int fluid_set_inflow(fluid_solver* s, int axis, int side, const double* W_dev, size_t count,
                     void* stream);

/* Convert primitives W[5][pz][py][px] (rho, u, v, w, p) to conservative U over all padded cells:
 * E = p / (gamma - 1) + rho |u|^2 / 2.  W and U may be the same buffer. */
int fluid_prim_to_cons(fluid_solver* s, const double* W_dev, double* U_dev, void* stream);

/* Right-hand side of Eq. ODE: R = -sum_d (F_{d,+} - F_{d,-}) / dx_d + S for every interior cell,
 * with F = F^c - F^d the convective minus dissipative face flux and S the body-force source.  U
 * is read only (its halos are not read or written: boundary values are built from the interior);
 * R has U's padded shape and only its interior is written.  U and R must not alias. */
int fluid_rhs(fluid_solver* s, const double* U_dev, double* R_dev, void* stream);

/* CFL time step of the state U (see fluid_config.cfl), written to *dt_dev (one double, device). */
int fluid_compute_dt(fluid_solver* s, const double* U_dev, double* dt_dev, void* stream);

/* Advance U in place by nsteps steps of the third-order TVD (Shu-Osher) Runge-Kutta scheme:
 *   U1 = Un + dt R(Un); U2 = 3/4 Un + 1/4 (U1 + dt R(U1)); Un+1 = 1/3 Un + 2/3 (U2 + dt R(U2)),
 * dt from the CFL rule of each step's initial state (or dt_fixed) and clipped so that the solver
 * time never passes t_end (t_end <= 0 means no limit; steps after t_end leave U unchanged).  The
 * solver time and last dt live on the device.  Halos of U are left unspecified. */
int fluid_step(fluid_solver* s, double* U_dev, int nsteps, double t_end, void* stream);

/* One RK3 step like fluid_step (one step, no t_end) that also writes the two intermediate stage
 * states U1 = Un + dt R(Un) and U2 = 3/4 Un + 1/4 (U1 + dt R(U1)) to the caller's buffers (same
 * shape as U, interior written); used to replay a segment before its adjoint. */
int fluid_step_stages(fluid_solver* s, double* U_dev, double* U1_dev, double* U2_dev, void* stream);

/* ---- discrete adjoint (the gradient of Section 3.2's end-to-end optimisation through the
 * differentiable disturbance wall, written by hand instead of automatic differentiation).  Needs
 * cfg.adjoint != 0 and, for the step adjoint, a frozen time step (cfg.dt_fixed > 0).  FP64 only. */

/* Vector-Jacobian product of the right-hand side (the operation of fluid_rhs) at state U: given a
 * cotangent mu of R on the interior cells (padded shape; halos ignored), writes
 * gU = (dR/dU)^T mu on the interior (halos untouched) and, if gphi_dev is not NULL and the
 * configuration has a porous face, adds (dR/dphi)^T mu to gphi_dev[0 .. porous_count-1].  The
 * WENO5 weights and the HLLC branch are differentiated exactly; ties take the forward's choice. */
int fluid_adjoint_rhs(fluid_solver* s, const double* U_dev, const double* mu_dev, double* gU_dev,
                      double* gphi_dev, void* stream);

/* Adjoint of one RK3 step with the frozen dt: on input lam holds dJ/dU^{n+1} (interior), on output
 * dJ/dU^n; (dU^{n+1}/dphi)^T lam is added to gphi_dev (may be NULL).  U1_dev / U2_dev are the stage
 * states of the step from fluid_step_stages, or NULL to recompute them from Un.  lam must not
 * alias the other arrays. */
int fluid_adjoint_step(fluid_solver* s, const double* Un_dev, const double* U1_dev,
                       const double* U2_dev, double* lam_dev, double* gphi_dev, void* stream);

/* Integrated wall heat flux J = sum over the wall cells of q_w * face area, q_w = -lambda(T_w)
 * dT/dn by the fourth-order normal stencil through the mirrored halo (derivative along +axis), on
 * the isothermal or porous face (axis, side).  Writes J to *J_dev (device) and, if dJdU_dev is not
 * NULL, dJ/dU on the whole padded array (zero except the two wall-adjacent cell layers). */
int fluid_wall_heat_loss(fluid_solver* s, const double* U_dev, int axis, int side, double* J_dev,
                         double* dJdU_dev, void* stream);

/* ---- block decomposition (Section 2.2: the padded domain is split into blocks, one per device,
 * and each right-hand side first exchanges N_h = 3 halo layers with the neighbouring blocks).  A
 * sub-domain solver has FLUID_BC_EXCHANGE on the faces it shares with another block (and on both
 * faces of a split periodic axis) and global_n / offset in its configuration.  Before every
 * right-hand side (every RK3 stage) the caller refreshes the exchange halos of the stage's input
 * state, axis by axis in the order x, y, z: fluid_pack_halo on both faces of the axis, hand each
 * buffer to the neighbour across that face, fluid_unpack_halo of the received ones.  A buffer of
 * axis a covers the three layers next to the face over the padded range of the axes below a and
 * the interior range of the axes above a; halos filled by the earlier axes thus travel on, which
 * gives the edge and corner cells of blocks that touch diagonally.  The time step is the minimum
 * over blocks of fluid_compute_dt (one min-reduction), and fluid_rk3_stage advances each block. */

/* Doubles in one packed halo buffer of axis a (either side): 5 * 3 * (product over the other
 * axes b of p[b] for b < a, n[b] for b > a). */
int fluid_halo_count(const fluid_solver* s, int axis, size_t* count);

/* Copy the three interior cell layers of U next to face (axis, side) into buf (device,
 * fluid_halo_count doubles, laid out [5][layer][t2][t1] with t1 < t2 the other axes, layers in
 * increasing index order).  Side 0 packs layers h .. h+2, which become the halo of the neighbour
 * below; side 1 packs n .. n+2, the halo of the neighbour above.  FLUID_EINVAL for a bad axis or
 * pointer. */
int fluid_pack_halo(fluid_solver* s, const double* U_dev, int axis, int side, double* buf_dev,
                    void* stream);

/* Write buf (as packed by the neighbour across face (axis, side): its side-1 buffer for side 0,
 * its side-0 buffer for side 1) into the three halo layers of U at that face.  U's interior is
 * not touched.  FLUID_EINVAL for a bad axis or pointer. */
int fluid_unpack_halo(fluid_solver* s, double* U_dev, int axis, int side, const double* buf_dev,
                      void* stream);

/* One stage of the TVD-RK3 step of fluid_step with a given dt > 0:
 *   stage 1: Ud = Un + dt R(Un) (pass Us = Un);  stage 2: Ud = 3/4 Un + 1/4 (Us + dt R(Us));
 *   stage 3: Ud = 1/3 Un + 2/3 (Us + dt R(Us)).
 * R(Us) reads the halo cells of Us on FLUID_BC_EXCHANGE faces as they are (refresh them first)
 * and builds every other halo from the interior, exactly as fluid_rhs.  Only interior cells of Ud
 * are written; Ud may be the same buffer as Us or Un (the combination is per cell).  The solver
 * time is not advanced.  With the dt of fluid_step, three calls give bitwise fluid_step's
 * result.  This is the way sub-domain solvers advance: fluid_step, fluid_step_stages, the adjoint
 * entry points and fluid_wall_heat_loss return FLUID_EINVAL for a configuration with exchange
 * faces. */
int fluid_rk3_stage(fluid_solver* s, int stage, const double* Un_dev, const double* Us_dev,
                    double* Ud_dev, double dt, void* stream);

/* Wall heat flux and wall shear on the isothermal or porous face (axis, side) of a 2-D or 3-D
 * solve (Section 3.2's quantities of the boundary layer; also the channel walls): per wall cell,
 * laid out [n_t2][n_t1] with t1 < t2 the other axes, q_w = -lambda(T_w) dT/dn and
 * tau_w = mu(T_w) du_t1/dn (t1 the first other axis, derivatives along +axis) by the
 * fourth-order face stencil through the mirrored ghost cells.  Written to qw_dev / tw_dev
 * (device, either may be NULL).  Works for either precision (the primitives are formed in FP64).
 * FLUID_EINVAL for another face kind or bad arguments. */
int fluid_wall_fluxes(fluid_solver* s, const double* U_dev, int axis, int side, double* qw_dev,
                      double* tw_dev, void* stream);

/* Synchronise `stream` and read the solver time and the last step's dt (either may be NULL). */
int fluid_get_time(fluid_solver* s, double* t, double* last_dt, void* stream);

/* Set the solver time (enqueued on `stream`). */
int fluid_set_time(fluid_solver* s, double t, void* stream);

/* Synchronise `stream`; return FLUID_ENONFINITE if any stage produced a non-finite value or a
 * non-positive ghost temperature since the last check (and clear the flag), else FLUID_OK. */
int fluid_check(fluid_solver* s, void* stream);

/* Launch shape of the face kernels: threads per block (a multiple of 32 in [32, 128]; 0 = 128)
 * and cells per thread segment along the face axis (0 = automatic: the longest of 64/32/16/8/4
 * that still fills the GPU), for every axis (fluid_autotune_faces picks one per axis).  For FLUID_PREC_MIXED the y and z face kernels are shared-memory
 * tiles of 2 warps (block 64) or 4 warps (otherwise) by default; seg < 0 selects the register-window
 * marching kernels with |seg| cells per segment and `block` threads instead; seg = 1 selects the
 * 4-warp tiles whose (hi, lo) rows are staged into shared memory by bulk copies (cp.async.bulk on an
 * mbarrier; a copy that does not complete within its bounded wait makes fluid_check return
 * FLUID_ECUDA).  With the tiles,
 * fluid_step folds each RK3 stage (and the primitives of its result) into the last axis's tile
 * kernel, with the same arithmetic as the separate stage kernel.  FP64 results and those of the two
 * mixed tiles are bitwise the same for every shape; the mixed register-window kernels agree with
 * the tiles to FP32 rounding. */
int fluid_tune_faces(fluid_solver* s, int block, int seg);

/* Time the FP64 face kernels (blocks of 128 threads with segments of 8 to 32 cells and the
 * automatic choice, then blocks of 64 and 32 threads with the fastest segment length) on the
 * primitives of U_dev (device, the solver's padded layout; not modified) and keep the fastest shape
 * per axis; the launch shape never changes a result, so this only changes speed.
 * Enqueued on `stream` and synchronised; uses the solver's scratch, so no other call on the solver
 * may run meanwhile.  No-op (FLUID_OK) for FLUID_PREC_MIXED.  FLUID_EINVAL for a NULL solver or a
 * foreign pointer, FLUID_ECUDA on a launch error. */
int fluid_autotune_faces(fluid_solver* s, const double* U_dev, void* stream);

/* Kernel classes reported by the profiler. */
enum {
  FLUID_KERNEL_PRIM_BC = 0,  /* primitives + boundary halos */
  FLUID_KERNEL_GRAD = 1,     /* centre velocity gradients */
  FLUID_KERNEL_FACE_X = 2,   /* WENO5 + HLLC + dissipative flux + divergence along x */
  FLUID_KERNEL_FACE_Y = 3,
  FLUID_KERNEL_FACE_Z = 4,
  FLUID_KERNEL_STAGE = 5,    /* RK3 stage combination (+ source) */
  FLUID_KERNEL_DT = 6,       /* CFL reduction */
  FLUID_KERNEL_SOURCE = 7,   /* body-force source of fluid_rhs */
  FLUID_KERNEL_ADJ_FACE = 8, /* adjoint face kernels and their gathers */
  FLUID_KERNEL_ADJ_CELL = 9, /* adjoint per-cell kernels (source, halos, primitives, phi) */
  FLUID_KERNEL_COUNT = 10
};

/* Kernel timing.  While enabled, every launch step of the solver (one kernel, or a face kernel with
 * its seam kernel, a stage kernel with its halo kernel) is bracketed by a CUDA event pair recorded
 * on the launch stream (the measured time is the kernels' device time plus event overhead of a few
 * microseconds).  fluid_profile_read synchronises on the pending events, adds them to per-class
 * totals and returns the total milliseconds and the number of kernels launched in class `kind`;
 * reset != 0 clears all totals after reading. */
int fluid_profile_enable(fluid_solver* s, int enable);
int fluid_profile_read(fluid_solver* s, int kind, double* total_ms, int64_t* launches, int reset);

/* FMA-throughput probe (synchronises `stream`): kind 0 = FP64, 1 = FP32; writes achieved GFLOP/s
 * (2 flops per FMA) of a kernel of independent FMA chains over every SM. */
int fluid_measure_peak(int kind, double* gflops, void* stream);

/* Accuracy check of the reciprocal the kernels use in place of division (a Newton-Raphson step
 * from the hardware estimate): fast[i] = that reciprocal of y[i], ieee[i] = 1.0 / y[i], for n
 * device values.  For tests. */
int fluid_check_rcp(const double* y_dev, double* fast_dev, double* ieee_dev, int n, void* stream);

/* Accuracy check of the reciprocal square root and square root the kernels use (a third-order
 * step from the hardware estimate): rsqrt[i] and sqrt[i] of y[i] as the kernels compute them,
 * ieee[i] = CUDA's correctly rounded sqrt(y[i]), for n device values.  For tests. */
int fluid_check_sqrt(const double* y_dev, double* rsqrt_dev, double* sqrt_dev, double* ieee_dev,
                     int n, void* stream);

/* Accuracy check of the power-law viscosity ratio (T / T_ref)^e as the kernels compute it: for an
 * exponent that is a ratio p / q of small integers (0.7 = 7 / 10) one Halley step for y^q = x^p
 * from an FP32 estimate, otherwise the library exp(e log x).  fast[i] = that value of x[i],
 * lib[i] = exp(e log x[i]) (CUDA's library), for n device values.  For tests. */
int fluid_check_pow(const double* x_dev, double* fast_dev, double* lib_dev, int n, double e,
                    void* stream);


/* Check of the FP32 -> FP64 widening the mixed face kernels build from the bit fields with integer
 * operations: bits[i] = that widening of x[i], cvt[i] = the conversion instruction's result, for n
 * device values.  For tests. */
int fluid_check_widen(const float* x_dev, double* bits_dev, double* cvt_dev, int n, void* stream);


/* Check of the bulk-copy staging the mixed y / z tiles can use (fluid_tune_faces seg = 1): one warp
 * stages nrows (1..8) rows of 36 floats from src_dev (16-byte aligned, device) into shared memory
 * with cp.async.bulk on an mbarrier expecting the rows' bytes plus extra_bytes, waits with the
 * tiles' bounded wait and writes the rows to dst_dev.  extra_bytes > 0 makes the wait run out
 * (every copy lands, the expected count is never reached): FLAG_STAGING (4) is then ORed into
 * *flags_dev (device) and dst_dev is not written.  Enqueued on `stream`.  For tests. */
int fluid_check_bulk_staging(const float* src_dev, float* dst_dev, int nrows, int extra_bytes,
                             unsigned* flags_dev, void* stream);


/* fluid_rhs without a solver object and without allocating: the same right-hand side as
 * fluid_rhs, for callers that cannot call cudaMalloc -- for example a host whose device memory is
 * owned by its own pool or arena and which forbids allocations behind its back, or a
 * latency-critical caller that cannot afford cudaMalloc's implicit device synchronisation.  The
 * paper has no counterpart; it is an interface convenience of this library.
 *
 * All scratch (primitives, velocity gradients, grid metrics, flags) lives in one fixed file-scope
 * device array of 2^21 doubles (16 MiB), reserved on every GPU the process uses until it exits.
 * A grid fits when its scratch fits: 15 doubles per padded cell with viscosity (6 without) plus
 * its metrics, i.e. cubes up to 45^3 interior cells viscous / 64^3 inviscid in 3-D, squares up to
 * 367^2 / 584^2 in 2-D; larger grids return FLUID_EINVAL with a message giving the need.  The
 * caller passes the input U and the output R exactly as for fluid_rhs (same layout, R interior
 * written, halos untouched).  Porous faces use phi_i = phi0; inflow faces return FLUID_ENOTSUP
 * (they need fluid_set_inflow); it computes in FP64 only (FLUID_PREC_MIXED returns
 * FLUID_ENOTSUP), and blocks of a decomposed grid (exchange faces, global_n) return
 * FLUID_ENOTSUP.  Non-finite / ghost-temperature flags are not reported.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 * caches it; make that first call before any stream capture.  The cached address belongs to the
 * device's primary context: after cudaDeviceReset, do not call this entry point again in the
 * process on that device.  Every call shares the one array and
 * it keeps the last call's contents: calls whose work overlaps on the GPU (different streams or
 * host threads without ordering) race and give wrong results.  Nothing is allocated on the device
 * or the host; errbuf (may be NULL) receives a message of at most errlen - 1 characters. */
int fluid_rhs_noalloc(const fluid_config* cfg, const double* U_dev, double* R_dev, void* stream,
                      char* errbuf, size_t errlen);

/* ---- serving: continuous batching of many independent solves (a design sweep) -------------------
 * A server owns one GPU and a scheduler thread.  Requests are admitted first-fit in arrival order
 * as soon as their device footprint (fluid_serve_footprint) fits the HBM budget next to the solves
 * already running and a slot is free; each running solve keeps its state on the device.  With
 * cfg.batch, compatible solves join a bucket and advance together, chunk by chunk: every kernel of
 * a chunk is one launch over all the bucket's solves (a table in device memory lists them; the
 * launches' blocks walk every solve's own launch grid), the chunk is a CUDA graph captured once
 * per bucket, and between chunks the table is rewritten as solves join (admission) and leave
 * (retirement), so a request that arrives while others run waits at most one chunk.  Solves that
 * cannot be batched run on their own stream in chunks replayed from a graph captured per solve, the
 * first of each grid shape timing the face kernels' launch shapes.  Buckets and single solves
 * overlap on the device; finished solves are copied back and their memory admits waiting
 * requests.  Results do not depend on the mix: every solve computes exactly what fluid_step
 * computes alone. */
typedef struct fluid_server fluid_server;

typedef struct fluid_serve_config {
  uint32_t struct_size;        /* sizeof(fluid_serve_config) */
  int32_t device;              /* CUDA device of the server */
  int32_t max_active;          /* concurrently running solves, >= 1 */
  int32_t chunk_steps;         /* RK3 steps per graph replay, >= 1 */
  int32_t use_graphs;          /* capture CUDA graphs (per bucket, or per solve when not batched) */
  int32_t autotune;            /* time launch shapes once per grid shape (solves that run alone) */
  uint64_t hbm_budget_bytes;   /* admission budget for all running solves */
  int32_t batch;               /* nonzero: solves with WENO5 and fourth-order (or no) dissipative
                                  stencils run batched -- one launch per kernel advances every
                                  solve of a bucket (same precision, reconstruction and viscous
                                  flag; any grid size, 2-D with 3-D), at most 64 per bucket, a
                                  chunk of steps captured once per bucket as a CUDA graph.  Other
                                  solves run alone on their own stream and graph */
  int32_t pad;
} fluid_serve_config;

typedef struct fluid_request {
  uint32_t struct_size;        /* sizeof(fluid_request) */
  int32_t nsteps;              /* RK3 steps */
  fluid_config cfg;            /* the solve */
  const double* U0_host;       /* initial padded state (copied during submit) */
  double* U_out_host;          /* final state written here before the result is ready (may be NULL) */
  double t_end;                /* as in fluid_step (<= 0: no limit) */
} fluid_request;

typedef struct fluid_result {
  int32_t status;              /* fluid_status of the solve (FLUID_ENONFINITE, ...) */
  int32_t steps_done;
  double t_final;              /* solver time at the end */
  double submit_s, start_s, finish_s;   /* server-clock seconds: submitted, admitted, done */
} fluid_result;

typedef struct fluid_serve_stats_t {
  int64_t pending, active, admitted, completed;
  uint64_t bytes_in_use, peak_bytes;
  double cell_updates;         /* interior cells x steps of the completed solves */
  double elapsed_s;
} fluid_serve_stats_t;

/* Start a server (spawns its scheduler thread).  FLUID_EINVAL for a bad config, FLUID_ECUDA when
 * the device is unavailable. */
int fluid_serve_create(const fluid_serve_config* cfg, fluid_server** out);
/* Stop the scheduler (running solves finish with FLUID_EBUSY) and release everything. */
void fluid_serve_destroy(fluid_server* s);
/* Queue a request; never blocks on the GPU.  FLUID_EBUDGET if it can never fit the budget,
 * FLUID_EINVAL for a bad request.  *ticket identifies it for fluid_serve_poll. */
int fluid_serve_submit(fluid_server* s, const fluid_request* req, uint64_t* ticket);
/* Wait up to timeout_ms (0: do not wait) for a result; FLUID_ETIMEOUT if it is not ready.  A
 * delivered result is forgotten by the server (poll each ticket once). */
int fluid_serve_poll(fluid_server* s, uint64_t ticket, fluid_result* out, int timeout_ms);
/* Counters of the server (thread-safe). */
int fluid_serve_stats(fluid_server* s, fluid_serve_stats_t* out);
/* Device bytes a request of this configuration holds while it runs. */
size_t fluid_serve_footprint(const fluid_config* cfg);

/* Library build information: ABI version, and sizeof(fluid_config) expected. */
int fluid_abi_version(void);
size_t fluid_config_size(void);

#ifdef __cplusplus
}
#endif
#endif /* FLUID_H */
