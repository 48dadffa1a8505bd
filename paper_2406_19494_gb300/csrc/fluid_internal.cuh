// Internal definitions shared by the solver's CUDA translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fluid.h"
#include "fast_math.cuh"

struct fluid_solver;

namespace fl {

constexpr int NV = 5;   // conservative variables (rho, rho u, rho v, rho w, E)
constexpr int NW = 6;   // primitive scratch (rho, u, v, w, p, T)
constexpr int NG = 9;   // velocity-gradient scratch, component c * 3 + b = d u_c / d x_b

// flag bits of Ctl::flags
constexpr unsigned FLAG_NONFINITE = 1u;
constexpr unsigned FLAG_GHOST_T = 2u;
constexpr unsigned FLAG_STAGING = 4u;   // a shared-memory staging copy did not complete in time
// the mixed path's y / z face tiles: 4 warps of 3 faces, 11 cells along the face axis
constexpr int kMixedTileWarps = 4, kMixedTileFaces = 3;
constexpr int kMixedTileCells = kMixedTileWarps * kMixedTileFaces - 1;

// Grid geometry: padded sizes, strides and per-axis 1-D metric arrays (device, length p[a]).
struct Geo {
  int ndim;
  int n[3], h[3], p[3];
  int sy, sz;      // strides (cells) of y and z; x stride is 1
  int ncell;       // p0 p1 p2: stride between variables
  const double* xc[3];   // cell centres
  const double* dx[3];   // cell widths
  const double* idx[3];  // 1 / widths
  const double* mc[3];   // d(index)/dx at centres
  const double* mf[3];   // d(index)/dx at face a+1/2
  const float* mf32[3];  // FP32 copy of mf (mixed path only, else null)
  const float* mc32[3];  // FP32 copy of mc (mixed path only, else null)
  const float* idx32[3]; // FP32 copy of idx (mixed path only, else null)
};

struct Phys {
  double gamma, gm1, igm1, R, iR, cp, Pr, lam_fac;
  double mu_ref, T_ref, iT_ref, visc_exp, suth_S;
  int visc_p, visc_q;  // power law: visc_exp = visc_p / visc_q (small integers), else visc_q = 0
  float visc_e32;      // visc_exp in FP32
  int visc_hw_lo, visc_hw_hi;   // high-word bounds of the fast range of fl_pow_rational
  int visc, weno;
  int visc_order;     // central differences of the dissipative fluxes: 4 or 6
  double eps;
  double f[3];
  int has_force;
  double cfl, dt_fixed, dt_visc_k;
};

struct BC {
  int kind[3][2];
  double Tw[3][2];
  const double* inflow[3][2];   // primitive profile [5][T2][T1] (device) or null
  int porous_axis, porous_side, porous_t1;
  const double* vw;             // transpiration velocity per padded index of axis porous_t1
};

// Device-resident step control: solver time, last dt, sticky error flags.
struct Ctl {
  double t, dt;
  unsigned flags;
  unsigned pad;
};

__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff;
}

// Split x = hi + lo + r with |r| <= 2^-48 |x|, using integer operations only: hi keeps the sign,
// the exponent and the leading 23 fraction bits of x (x truncated to FP32 precision, exact), lo the
// remaining 29 fraction bits rounded to FP32.  Below 2^-73 lo is dropped (|r| < 2^-23 |x| <
// 1.2e-29), below 2^-126 both are zero; |x| >= 2^128 or a non-finite x gives NaN, which the
// non-finite check then reports.
__device__ __forceinline__ void split_hi_lo(double x, float& hi, float& lo) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);            // biased FP64 exponent
  if (e < 1023 - 126) { hi = __int_as_float(sign); lo = 0.0f; return; }
  if (e > 1023 + 127) { hi = __int_as_float(0x7fc00000); lo = hi; return; }
  hi = __int_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  // lo = (low 29 fraction bits) * 2^(e - 1075), with 2^(e - 1075) a normal float when e > 948
  const int es = e - 1075 + 127;
  const float m = (float)(lw & 0x1fffffffu);
  lo = es > 0 ? __int_as_float(sign | __float_as_int(m * __int_as_float(es << 23))) : 0.0f;
}

__host__ __device__ __forceinline__ double viscosity(double T, const Phys& ph) {
  if (ph.visc == FLUID_VISC_CONSTANT) return ph.mu_ref;
  const double r = T * ph.iT_ref;
  if (ph.visc == FLUID_VISC_POWER) {
    if (ph.visc_q > 0)
      return ph.mu_ref * fl_pow_rational(r, ph.visc_p, ph.visc_q, ph.visc_e32, ph.visc_hw_lo, ph.visc_hw_hi);
    return ph.mu_ref * exp(ph.visc_exp * log(r));
  }
  // Sutherland
  return ph.mu_ref * (r * fl_sqrt(r)) * (ph.T_ref + ph.suth_S) * fl_rcp(T + ph.suth_S);
}

// d mu / d T of the same laws, given mu = viscosity(T, ph): power law e mu / T; Sutherland
// (mu = C r^{3/2} / (T + S), C = mu_ref (T_ref + S)) mu (1.5 / T - 1 / (T + S))
__host__ __device__ __forceinline__ double viscosity_dT(double T, double mu, const Phys& ph) {
  if (ph.visc == FLUID_VISC_CONSTANT) return 0.0;
  if (ph.visc == FLUID_VISC_POWER) return ph.visc_exp * mu * fl_rcp(T);
  return mu * (1.5 * fl_rcp(T) - fl_rcp(T + ph.suth_S));
}

// The power-law exponent as p / q with 0 < p, q <= 16 when it is one to within a few ulp (0.7 is
// 7/10), for fl_pow_rational; q = 0 otherwise.  Also sets the FP32 copy.
inline void set_power_law(Phys& ph, double e) {
  ph.visc_exp = e;
  ph.visc_e32 = (float)e;
  ph.visc_p = ph.visc_q = 0;
  ph.visc_hw_lo = ph.visc_hw_hi = 0;
  for (int q = 1; q <= 16; ++q) {
    const double pq = e * q;
    const int p = (int)(pq + 0.5);
    if (p >= 1 && p <= 16 && fabs((double)p / q - e) <= 4.0 * 2.220446049250313e-16 * fabs(e)) {
      ph.visc_p = p;
      ph.visc_q = q;
      // |log2 x| < B keeps the FP32 estimate and x^p normal
      int B = 49;
      while (B > 1 && (B * e >= 125.0 || B * p >= 1021)) --B;
      ph.visc_hw_lo = (1023 - B) << 20;
      ph.visc_hw_hi = (1023 + B) << 20;
      return;
    }
  }
}

// Configuration check shared by the entry points: NULL if valid, else a static message.
const char* config_error(const fluid_config* c);

// Kernels the launchers below have enqueued from this host thread (each launch site adds one); the
// solver's profiler counts the kernels of a bracketed call by the difference.
inline thread_local long long t_launches = 0;

// ---- launchers implemented in kernels_fp64.cu --------------------------------------------------
// W32 (mixed path only, else null): exact FP32 (hi, lo) split of the primitives, [2 NW][ncell];
// with it W must hold NW + 1 rows, the last receiving H = E + p
cudaError_t launch_prim_bc(const double* U, double* W, float* W32, const Geo& g, const Phys& ph,
                           const BC& bc, Ctl* ctl, cudaStream_t st);
cudaError_t launch_grad(const double* W, double* G, const Geo& g, const Phys& ph, cudaStream_t st);
// launch shape of the marching FP64 face kernels: block/seg 0 pick the defaults; grid out
void face_shape(int D, const Geo& g, int& block, int& seg, int& grid);
// Seam buffer of the FP64 face kernels: 10 doubles per segment item (lines x segments of a launch),
// cap items; a launch whose segments are shorter than kSeamMinSeg or that does not fit runs without
// it (same result).  {nullptr, 0} turns it off.
struct SeamBuf {
  double* p;
  long long cap;
};
constexpr int kSeamMinSeg = 4;
long long seam_capacity(const Geo& g);   // items for segments of kSeamMinSeg cells on every axis
// the buffer for a launch of segments of `seg` cells along D, or null when it runs without
double* seam_buffer(int D, const Geo& g, int seg, SeamBuf fb);
// the first cells of the segments after each line's first, from the fluxes in FB (fused: the
// TENO kernel's update form fma(-1/dx, F+ - F-, R), else the FP64 kernel's)
cudaError_t launch_face_seam(int D, const double* FB, double* R, const Geo& g, int accumulate,
                             int seg, bool fused, cudaStream_t st);
cudaError_t launch_face(int D, const double* W, const double* G, double* R, const Geo& g,
                        const Phys& ph, int accumulate, int block, int seg, SeamBuf fb,
                        cudaStream_t st);
cudaError_t launch_source(double* R, const double* W, const Geo& g, const Phys& ph, cudaStream_t st);
// dt_arg > 0 replaces the solver's dt (used by the adjoint's stage recomputation)
cudaError_t launch_stage(int stage, const double* Un, const double* Us, const double* R, double* Ud,
                         const double* W, const Geo& g, const Phys& ph, Ctl* ctl, double t_end,
                         cudaStream_t st, double dt_arg = 0.0);
// stage `stage` of RK3 into Ud with the solver's dt, then the primitives of Ud into W (and W32 / H
// when W32 is given) for every padded cell, equal to launch_prim_bc(Ud, ...) on the result
cudaError_t launch_stage_prim(int stage, const double* Un, const double* Us, const double* R,
                              double* Ud, double* W, float* W32, const Geo& g, const Phys& ph,
                              const BC& bc, Ctl* ctl, double t_end, cudaStream_t st);
// the halo cells of W (and W32 / H when W32 is given) from its interior, as launch_stage_prim's
// second pass
cudaError_t launch_halo_prim(double* W, float* W32, const Geo& g, const Phys& ph, const BC& bc, Ctl* ctl,
                             cudaStream_t st);
cudaError_t launch_dt_partial(const double* W, const Geo& g, const Phys& ph, double* partial,
                              int nparts, cudaStream_t st);
cudaError_t launch_dt_final(const double* partial, int nparts, const Phys& ph, Ctl* ctl,
                            double* dt_out, int clip_to_ctl, double t_end, cudaStream_t st);
int dt_partial_count(const Geo& g);
// ---- TENO6-A face kernels implemented in kernels_teno.cu ----------------------------------------
cudaError_t launch_face_teno(int D, const double* W, const double* G, double* R, const Geo& g,
                             const Phys& ph, int accumulate, int block, int seg, SeamBuf fb,
                             cudaStream_t st);
// ---- mixed-precision launchers implemented in kernels_mixed.cu --------------------------------
// seg 1 on the y / z tiles stages their rows by bulk copies; a copy that does not complete within
// its bounded wait sets FLAG_STAGING in *flags (when given) and leaves its tile undone
cudaError_t launch_face_mixed(int D, const double* W, const float* W32, const float* G32, double* R,
                              const Geo& g, const Phys& ph, int accumulate, int block, int seg,
                              cudaStream_t st, unsigned* flags = nullptr);
// Stage output of the last axis's face kernel when the stage is fused into it: Ud = stage `stage`
// of RK3 from Un, Us and the completed right-hand side, and the primitives of Ud (W: NW rows and
// the H row; W32: the split) written to a second buffer pair, since the kernel still reads the
// current one.  prims = false (the last stage of a call) writes Ud only.
struct StageOut {
  int stage;
  int prims;
  const double* Un;
  const double* Us;
  double* Ud;
  double* W;
  float* W32;
  Ctl* ctl;
  double t_end;
};
// whether launch_face_mixed_stage can take the last axis of this grid (the y / z tile kernels)
bool mixed_stage_fusable(const Geo& g, int seg);
// the face kernel of the last axis (ndim - 1) accumulating into R's values of the other axes,
// fused with the stage combination and the primitives of its result (interior cells; the halo
// cells of the new buffer follow with launch_halo_prim)
cudaError_t launch_face_mixed_stage(const double* W, const float* W32, const float* G32,
                                    const double* R, const Geo& g, const Phys& ph, int block, int seg,
                                    const StageOut& so, cudaStream_t st);
cudaError_t launch_grad32(const float* W32, float* G32, const Geo& g, cudaStream_t st);
// check of the bulk-staging helpers (fluid_check_bulk_staging)
cudaError_t launch_bulk_probe(const float* src, float* dst, int nrows, unsigned extra_tx,
                              unsigned* flags, cudaStream_t st);
cudaError_t launch_dt_partial32(const float* W32, const Geo& g, const Phys& ph, double* partial,
                                int nparts, cudaStream_t st);

// ---- adjoint launchers implemented in kernels_adjoint.cu ----------------------------------------
cudaError_t launch_adj_faces(const double* W, const double* G, const double* mu, double* CW,
                             double* CG, double* gW, double* gG, const Geo& g, const Phys& ph,
                             cudaStream_t st);
cudaError_t launch_adj_source(const double* mu, double* gW, const Geo& g, const Phys& ph, cudaStream_t st);
cudaError_t launch_adj_bc(const double* W, double* gW, double* gvw_col, const Geo& g,
                          const Phys& ph, const BC& bc, cudaStream_t st);
cudaError_t launch_adj_prim(const double* U, const double* gW, double* gU, const Geo& g,
                            const Phys& ph, cudaStream_t st);
cudaError_t launch_adj_phi(const double* gvw_col, const double* xc, double* gphi, int p_t1,
                           int h_t1, int ext_t2, int begin, int count, double amp,
                           double two_pi_kappa, cudaStream_t st);
int wall_loss_parts(const Geo& g, int A);
cudaError_t launch_wall_loss(const double* W, double* part, int nparts, double* J, double* gT2,
                             const Geo& g, const Phys& ph, int A, int side, double Tw,
                             cudaStream_t st);
cudaError_t launch_wall_fluxes(const double* W, double* qw, double* tw, const Geo& g, const Phys& ph,
                               int A, int side, double Tw, cudaStream_t st);
cudaError_t launch_wall_loss_grad(const double* U, const double* gT2, double* dJdU, const Geo& g,
                                  const Phys& ph, int A, int side, cudaStream_t st);
cudaError_t launch_lincomb(double* out, double c0, const double* x0, double c1, const double* x1,
                           double c2, const double* x2, double c3, const double* x3, const Geo& g,
                           cudaStream_t st);

cudaError_t launch_prim_to_cons(const double* W, double* U, int ncell, const Phys& ph,
                                cudaStream_t st);
// block decomposition: doubles of one packed halo buffer of axis A, and the copy between the three
// layers next to face (A, side) and the buffer (unpack: buffer -> halo layers; else interior
// layers -> buffer)
size_t halo_count(const Geo& g, int A);
cudaError_t launch_halo_copy(double* U, double* buf, const Geo& g, int A, int side, bool unpack,
                             cudaStream_t st);
cudaError_t launch_wall_velocity(const double* phi, double* vw, const double* xc, int p, int h,
                                 int begin, int count, double amp, double two_pi_kappa,
                                 cudaStream_t st);

// ---- batched launches of the serving loop ------------------------------------------------------
// One launch advances every solve of a bucket: the kernel's blocks walk the "virtual blocks" of all
// solves (each solve's own launch grid of that kernel, laid end to end), and every virtual block
// runs the standalone kernel's body with the solve's data and its own block index and grid size,
// so each solve computes exactly what its standalone launches compute.  Solves of any grid size
// (and 2-D with 3-D) share a bucket; the grids of the launches are fixed, so a chunk of steps is
// captured once per bucket in a CUDA graph and the table below, in device memory, is rewritten
// between chunks as solves are admitted and retire.
constexpr int kBatchMax = 64;   // solves per bucket
enum BatchKernel {
  BK_PRIM = 0, BK_DTP, BK_DTF, BK_GRAD, BK_FACE0, BK_FACE1, BK_FACE2, BK_SEAM0, BK_SEAM1, BK_SEAM2,
  BK_STAGEP, BK_HALO, BK_STAGE, BK_COUNT
};
struct BatchSlot {
  Geo g;
  Phys ph;
  BC bc;
  double* U;          // state (advanced in place)
  double* A;          // stage state
  double* R;          // right-hand side
  double* W;          // primitives (mixed: plus the H row)
  double* G;          // FP64 gradients (FP64 viscous)
  float* W32;         // FP32 split (mixed)
  float* G32;         // FP32 gradients (mixed viscous)
  double* FB[3];      // seam buffer per axis (null: none)
  double* partial;    // CFL partial maxima
  int nparts;         // their count (0 with a fixed dt)
  Ctl* ctl;
  double t_end;
  int seg[3];         // FP64 face segment length per axis
  int steps;          // steps of the current chunk; the solve idles at later steps
  int vgrid[BK_COUNT][3];
};
struct BatchTable {
  int nslots;
  int pad;
  long long prefix[BK_COUNT][kBatchMax + 1];   // virtual blocks before each solve, per kernel
  BatchSlot slot[kBatchMax];
};
// the solve of virtual block vb of kernel k (binary search of the prefix)
__device__ __forceinline__ int batch_slot(const BatchTable* __restrict__ t, int k, long long vb) {
  int lo = 0, hi = t->nslots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t->prefix[k][mid] <= vb) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ uint3 batch_bid(const int vg[3], long long lb) {
  uint3 b;
  b.x = (unsigned)(lb % vg[0]);
  b.y = (unsigned)((lb / vg[0]) % vg[1]);
  b.z = (unsigned)(lb / ((long long)vg[0] * vg[1]));
  return b;
}
// fluid_create with stream-ordered allocations on st (cudaMallocAsync): set-up copies are enqueued
// on st and nothing synchronises; fluid_destroy of such a solver frees on st without waiting
int solver_create_async(const fluid_config* cfg, cudaStream_t st, fluid_solver** out);
// a solver's part of a batch (its geometry, physics, boundaries and scratch, state U, t_end); false
// when its configuration has no batched kernels (TENO6-A, sixth-order stencils, exchange faces)
bool batch_slot_of(fluid_solver* s, double* U, double t_end, BatchSlot& out);
// fill slot.vgrid and the prefixes for the solves of t (their Geo, Phys, seg and FB set)
void batch_plan(BatchTable& t, bool mixed);
// enqueue the batched kernels of `chunk` RK3 steps (what fluid_step(U, chunk) does for every solve)
cudaError_t launch_batch_chunk(const BatchTable* dev, int chunk, bool mixed, int weno, bool visc,
                               cudaStream_t st);
// the mixed path's batched gradient and CFL kernels, and its face kernels (kernels_mixed.cu)
enum { BMX_GRAD = 0, BMX_DTP = 2 };
cudaError_t launch_batch_mixed(const BatchTable* dev, int kind, int D, int step, cudaStream_t st);
cudaError_t launch_batch_mixed_faces(const BatchTable* dev, int D, int step, int weno, bool visc,
                                     cudaStream_t st);

}  // namespace fl
