// C ABI of the solver (declared in include/fluid.h): configuration checks, grid metrics, scratch
// ownership and the launch sequences of the right-hand side and the TVD-RK3 step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "fluid_internal.cuh"

using fl::BC;
using fl::Ctl;
using fl::Geo;
using fl::Phys;

// Device memory of a solver: cudaMalloc (fluid_create), or stream-ordered on one stream for the
// solvers the serving loop owns, so that admitting and retiring a solve never waits for the device.
struct SolverAlloc {
  cudaStream_t st = nullptr;
  bool async = false;
  cudaError_t malloc(void** p, size_t n) const {
    return async ? cudaMallocAsync(p, n, st) : cudaMalloc(p, n);
  }
  void free(void* p) const {
    if (!p) return;
    if (async) cudaFreeAsync(p, st);
    else cudaFree(p);
  }
  cudaError_t h2d(void* d, const void* h, size_t n) const {
    return async ? cudaMemcpyAsync(d, h, n, cudaMemcpyHostToDevice, st)
                 : cudaMemcpy(d, h, n, cudaMemcpyHostToDevice);
  }
  cudaError_t memset(void* d, int v, size_t n) const {
    return async ? cudaMemsetAsync(d, v, n, st) : cudaMemset(d, v, n);
  }
};

struct fluid_solver {
  SolverAlloc alloc;
  fluid_config cfg;
  Geo geo;
  Phys ph;
  BC bc;
  int device = 0;
  double* metric = nullptr;        // 5 arrays x 3 axes, each of length p[a]
  double* W = nullptr;             // primitives, NW * ncell
  double* G = nullptr;             // velocity gradients, NG * ncell (viscous, FP64 path)
  bool mixed = false;              // FLUID_PREC_MIXED: FP32 fluxes, FP64 state
  bool exchange = false;           // some face is FLUID_BC_EXCHANGE (a block of a decomposition)
  float* W32 = nullptr;            // FP32 (hi, lo) primitives, 2 NW * ncell (mixed)
  double* Wb = nullptr;            // mixed: the second pair of primitive buffers (W with its H row,
  float* W32b = nullptr;           // W32), written by a stage fused into the last face kernel
  float* mf32 = nullptr;           // FP32 face metrics, centre metrics and inverse widths of the three axes (mixed)
  float* G32 = nullptr;            // FP32 velocity gradients (mixed, viscous)
  double* A = nullptr;             // RK stage state, NV * ncell
  double* R = nullptr;             // right-hand side accumulator, NV * ncell
  double* FB = nullptr;            // seam buffer of the FP64 face kernels, 10 * fb_cap
  long long fb_cap = 0;
  double* partial = nullptr;       // dt: per-block maxima of the CFL rates
  int nparts = 0;
  Ctl* ctl = nullptr;
  double* vw = nullptr;            // porous transpiration velocities
  double* phi = nullptr;           // porous parameters
  double* inflow[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  size_t inflow_count[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  std::vector<double> host_xc[3], host_dx[3];
  std::string err;
  // kernel timing (fluid_profile_*): event pairs bracketing each launch, resolved on read
  struct ProfEvent {
    int kind;
    cudaEvent_t a, b;
    long long kernels;   // kernels enqueued between the two events
  };
  int face_block = 0, face_seg = 0;   // launch shape of the face kernels (0 = automatic)
  int face_seg_d[3] = {0, 0, 0};      // FP64 path: segment length per axis (0 = automatic)
  int face_block_d[3] = {0, 0, 0};    // FP64 path: threads per block per axis (0 = 128)
  // adjoint scratch (cfg.adjoint != 0)
  double* gW = nullptr;            // cotangent of the primitives, NW * ncell
  double* gG = nullptr;            // cotangent of the velocity gradients, NG * ncell
  double* CW = nullptr;            // per-face contributions (6 slots x 6 primitives), 36 * ncell
  double* CG = nullptr;            // per-face cotangents of the four tangential face gradients, 4 * ncell
  double* S1 = nullptr;            // stage states recomputed by the step adjoint
  double* S2 = nullptr;
  double* MU = nullptr;            // scaled cotangent handed to the right-hand-side adjoint
  double* L1 = nullptr;            // stage adjoints
  double* L2 = nullptr;
  double* GT = nullptr;            // right-hand-side adjoint result
  double* Wn = nullptr;            // primitives and gradients of Un and U1 formed by the step
  double* Gn = nullptr;            // adjoint's stage recomputation, kept for its reverse passes
  double* W1 = nullptr;
  double* G1 = nullptr;
  double* gvw = nullptr;           // porous wall-velocity cotangent per wall column
  size_t gvw_count = 0;
  double* parts = nullptr;         // wall-loss partial sums
  double* gT2 = nullptr;           // wall-loss dJ/dT of the two wall-adjacent cells per column
  int nloss = 0;
  bool prof_on = false;
  std::vector<ProfEvent> prof_pending, prof_pool;
  double prof_ms[FLUID_KERNEL_COUNT] = {0};
  int64_t prof_n[FLUID_KERNEL_COUNT] = {0};
};

namespace {

thread_local std::string g_create_error;

int fail(fluid_solver* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(fluid_solver* s, cudaError_t e, const char* what) {
  return fail(s, e == cudaErrorMemoryAllocation ? FLUID_ENOMEM : FLUID_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define FL_CUDA(s, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
  } while (0)

// face coordinate x(eta) and dx/deta of the axis mapping
void axis_map(int stretch, double beta, double lo, double hi, double eta, double* x, double* dxdeta) {
  const double L = hi - lo;
  if (stretch == FLUID_STRETCH_UNIFORM) {
    *x = lo + L * eta;
    *dxdeta = L;
    return;
  }
  const double tb = std::tanh(beta);
  if (stretch == FLUID_STRETCH_TANH2) {
    const double t = std::tanh(beta * (2.0 * eta - 1.0));
    *x = lo + 0.5 * L * (1.0 + t / tb);
    *dxdeta = L * beta * (1.0 - t * t) / tb;
  } else {
    const double t = std::tanh(beta * (1.0 - eta));
    *x = lo + L * (1.0 - t / tb);
    *dxdeta = L * beta * (1.0 - t * t) / tb;
  }
}

// host metric arrays of one axis: xc, dx, 1/dx, mc, mf over the padded range.  A block of a
// decomposed grid (global_n > 0) evaluates the global mapping at its global cell indices, so every
// value is bitwise the global grid's at the same cell.
void axis_metrics(const fluid_config& c, int a, int h, std::vector<double> out[5]) {
  const int p = c.n[a] + 2 * h;
  const int n = c.global_n[a] > 0 ? c.global_n[a] : c.n[a];
  const int off = c.global_n[a] > 0 ? c.offset[a] : 0;
  for (int k = 0; k < 5; ++k) out[k].assign(p, 0.0);
  if (c.stretch[a] == FLUID_STRETCH_UNIFORM) {
    const double d = (c.hi[a] - c.lo[a]) / n;
    for (int i = 0; i < p; ++i) {
      const double ai = (double)(i + off - h);
      out[0][i] = c.lo[a] + (ai + 0.5) * d;
      out[1][i] = d;
      out[2][i] = 1.0 / d;
      out[3][i] = 1.0 / d;
      out[4][i] = 1.0 / d;
    }
    return;
  }
  std::vector<double> xf(p + 1);
  double dd;
  for (int k = 0; k <= p; ++k)
    axis_map(c.stretch[a], c.beta[a], c.lo[a], c.hi[a], (double)(k + off - h) / n, &xf[k], &dd);
  for (int i = 0; i < p; ++i) {
    const double ai = (double)(i + off - h);
    double x, dc, df;
    out[1][i] = xf[i + 1] - xf[i];
    out[0][i] = 0.5 * (xf[i + 1] + xf[i]);
    out[2][i] = 1.0 / out[1][i];
    axis_map(c.stretch[a], c.beta[a], c.lo[a], c.hi[a], (ai + 0.5) / n, &x, &dc);
    axis_map(c.stretch[a], c.beta[a], c.lo[a], c.hi[a], (ai + 1.0) / n, &x, &df);
    out[3][i] = n / dc;
    out[4][i] = n / df;
  }
}


const char* validate(const fluid_config* c) {
  if (!c) return "cfg is NULL";
  if (c->struct_size != sizeof(fluid_config)) return "cfg->struct_size != sizeof(fluid_config)";
  if (c->ndim < 1 || c->ndim > 3) return "ndim must be 1, 2 or 3";
  long long cells = 1;
  for (int a = 0; a < 3; ++a) {
    const bool act = a < c->ndim;
    if (act && (c->n[a] < 3 || c->n[a] > (1 << 20))) return "active axes need 3 <= n <= 2^20 cells";
    if (!act && c->n[a] != 1) return "inactive axes must have n == 1";
    if (!(c->hi[a] > c->lo[a])) return "hi must exceed lo on every axis";
    if (c->stretch[a] < 0 || c->stretch[a] > 2) return "unknown stretch kind";
    if (c->stretch[a] != FLUID_STRETCH_UNIFORM && !(c->beta[a] > 0)) return "tanh stretching needs beta > 0";
    if (!act && c->stretch[a] != FLUID_STRETCH_UNIFORM) return "inactive axes must be uniform";
    cells *= c->n[a] + (act ? 2 * FLUID_HALO : 0);
    if (!act) continue;
    for (int s = 0; s < 2; ++s) {
      const int k = c->bc[a][s];
      if (k < 0 || k > FLUID_BC_EXCHANGE) return "unknown boundary kind";
      if ((k == FLUID_BC_WALL || k == FLUID_BC_POROUS) && !(c->t_wall[a][s] > 0))
        return "isothermal walls need t_wall > 0";
    }
    if ((c->bc[a][0] == FLUID_BC_PERIODIC) != (c->bc[a][1] == FLUID_BC_PERIODIC))
      return "periodic boundaries must pair";
  }
  for (int a = 0; a < 3; ++a) {
    if (c->global_n[a] < 0) return "global_n must be >= 0";
    if (c->global_n[a] == 0 && c->offset[a] != 0) return "offset needs global_n > 0 on its axis";
    if (c->global_n[a] > 0) {
      if (a >= c->ndim) return "inactive axes cannot be split (global_n must be 0)";
      if (c->global_n[a] > (1 << 20)) return "global_n must be <= 2^20";
      if (c->offset[a] < 0 || c->offset[a] + c->n[a] > c->global_n[a])
        return "the block (offset, n) must lie inside the global grid";
    }
  }
  // the kernels index arrays of R rows of padded cells with 32-bit row * ncell + cell: 9 rows on
  // the FP64 path (the velocity gradients), 12 on the mixed one (the FP32 split of the
  // primitives), 36 for the adjoint (its per-face slots)
  if (cells >= (1LL << 31) / 9) return "grid too large for 32-bit cell indexing";
  if (c->precision == FLUID_PREC_MIXED && cells >= (1LL << 31) / 12)
    return "grid too large for 32-bit cell indexing of the mixed path (12 FP32 rows per cell)";
  if (c->adjoint && cells >= (1LL << 31) / 36)
    return "grid too large for 32-bit cell indexing of the adjoint (36 per-face slots per cell)";
  if (!(c->gamma > 1.0) || !(c->gas_R > 0) || !(c->prandtl > 0)) return "need gamma > 1, R > 0, Pr > 0";
  if (c->visc_law < 0 || c->visc_law > 3) return "unknown viscosity law";
  if (c->visc_law != FLUID_VISC_NONE && !(c->mu_ref > 0)) return "viscous runs need mu_ref > 0";
  if (c->visc_law != FLUID_VISC_NONE && c->visc_law != FLUID_VISC_CONSTANT && !(c->T_ref > 0))
    return "T_ref must be > 0";
  if (c->visc_law == FLUID_VISC_SUTHERLAND && !(c->suth_S >= 0)) return "suth_S must be >= 0";
  if (c->weno != FLUID_WENO_JS && c->weno != FLUID_WENO_Z && c->weno != FLUID_TENO6A)
    return "unknown reconstruction (weno)";
  if (c->visc_order != 0 && c->visc_order != 4 && c->visc_order != 6) return "visc_order must be 0, 4 or 6";
  if ((c->weno == FLUID_TENO6A || c->visc_order == 6) && c->precision != FLUID_PREC_FP64)
    return "TENO6-A and sixth-order dissipative fluxes run in FP64 only";
  if ((c->weno == FLUID_TENO6A || c->visc_order == 6) && c->adjoint)
    return "the adjoint covers WENO5 with fourth-order dissipative fluxes only";
  if (c->precision != FLUID_PREC_FP64 && c->precision != FLUID_PREC_MIXED) return "unknown precision";
  if (!(c->dt_fixed > 0) && !(c->cfl > 0)) return "need cfl > 0 or dt_fixed > 0";
  bool exch = false;
  for (int a = 0; a < c->ndim; ++a)
    for (int s = 0; s < 2; ++s) exch |= c->bc[a][s] == FLUID_BC_EXCHANGE;
  if (exch && c->adjoint) return "the adjoint does not cover sub-domain (exchange) faces";
  int nporous = 0;
  for (int a = 0; a < c->ndim; ++a)
    for (int s = 0; s < 2; ++s) nporous += c->bc[a][s] == FLUID_BC_POROUS;
  if (nporous > 1) return "at most one porous face";
  if (nporous == 1) {
    const int a = c->porous_axis, s = c->porous_side;
    if (a < 0 || a >= c->ndim || s < 0 || s > 1 || c->bc[a][s] != FLUID_BC_POROUS)
      return "porous_axis/porous_side must name the porous face";
    if (c->ndim < 2) return "a porous wall needs ndim >= 2";
    const int t1 = a == 0 ? 1 : 0;
    // a block's strip may reach into its exchange halos along the wall (the neighbours' wall cells)
    const int lo = c->bc[t1][0] == FLUID_BC_EXCHANGE ? -FLUID_HALO : 0;
    const int hi = c->n[t1] + (c->bc[t1][1] == FLUID_BC_EXCHANGE ? FLUID_HALO : 0);
    if (c->porous_count < 1 || c->porous_begin < lo || c->porous_begin + c->porous_count > hi)
      return "porous strip outside the wall";
    if (!(c->porous_phi0 != 0)) return "porous_phi0 must be nonzero";
  }
  return nullptr;
}

cudaStream_t as_stream(void* st) { return reinterpret_cast<cudaStream_t>(st); }

int check_ptr(fluid_solver* s, const void* p, const char* what) {
  if (!p) return fail(s, FLUID_EINVAL, std::string(what) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) % 8 != 0) return fail(s, FLUID_EINVAL, std::string(what) + " is not 8-byte aligned");
  return FLUID_OK;
}

// Run one launch; when profiling is on, bracket it with an event pair on the same stream.
template <class F>
int timed(fluid_solver* s, int kind, cudaStream_t st, const char* what, F&& launch) {
  fluid_solver::ProfEvent ev{kind, nullptr, nullptr, 0};
  const long long before = fl::t_launches;
  if (s->prof_on) {
    if (!s->prof_pool.empty()) {
      ev.a = s->prof_pool.back().a;
      ev.b = s->prof_pool.back().b;
      s->prof_pool.pop_back();
    } else {
      FL_CUDA(s, cudaEventCreate(&ev.a));
      FL_CUDA(s, cudaEventCreate(&ev.b));
    }
    FL_CUDA(s, cudaEventRecord(ev.a, st));
  }
  const cudaError_t e = launch();
  if (e != cudaSuccess) return cuda_fail(s, e, what);
  if (s->prof_on) {
    FL_CUDA(s, cudaEventRecord(ev.b, st));
    ev.kernels = fl::t_launches - before;
    s->prof_pending.push_back(ev);
  }
  return FLUID_OK;
}

#define FL_TIMED(s, kind, st, call)                                           \
  do {                                                                       \
    if (int r_ = timed((s), (kind), (st), #call, [&]() { return (call); })) \
      return r_;                                                             \
  } while (0)

// velocity gradients and the per-axis face kernels of one right-hand side (primitives ready)
int grad_faces(fluid_solver* s, double* R, cudaStream_t st) {
  const Geo& g = s->geo;
  if (s->mixed) {
    if (s->ph.visc != FLUID_VISC_NONE)
      FL_TIMED(s, FLUID_KERNEL_GRAD, st, fl::launch_grad32(s->W32, s->G32, g, st));
    for (int d = 0; d < g.ndim; ++d)
      FL_TIMED(s, FLUID_KERNEL_FACE_X + d, st,
               fl::launch_face_mixed(d, s->W, s->W32, s->G32, R, g, s->ph, d > 0, s->face_block,
                                     s->face_seg, st, &s->ctl->flags));
    return FLUID_OK;
  }
  if (s->ph.visc != FLUID_VISC_NONE)
    FL_TIMED(s, FLUID_KERNEL_GRAD, st, fl::launch_grad(s->W, s->G, g, s->ph, st));
  for (int d = 0; d < g.ndim; ++d)
    FL_TIMED(s, FLUID_KERNEL_FACE_X + d, st,
             fl::launch_face(d, s->W, s->G, R, g, s->ph, d > 0, s->face_block_d[d], s->face_seg_d[d],
                             fl::SeamBuf{s->FB, s->fb_cap}, st));
  return FLUID_OK;
}

int rhs_into(fluid_solver* s, const double* U, double* R, cudaStream_t st) {
  const Geo& g = s->geo;
  FL_TIMED(s, FLUID_KERNEL_PRIM_BC, st, fl::launch_prim_bc(U, s->W, s->W32, g, s->ph, s->bc, s->ctl, st));
  return grad_faces(s, R, st);
}

int dt_into(fluid_solver* s, double* dt_out, int clip, double t_end, cudaStream_t st) {
  if (s->ph.dt_fixed <= 0.0) {
    if (s->mixed)
      FL_TIMED(s, FLUID_KERNEL_DT, st, fl::launch_dt_partial32(s->W32, s->geo, s->ph, s->partial, s->nparts, st));
    else
      FL_TIMED(s, FLUID_KERNEL_DT, st, fl::launch_dt_partial(s->W, s->geo, s->ph, s->partial, s->nparts, st));
  }
  FL_TIMED(s, FLUID_KERNEL_DT, st,
           fl::launch_dt_final(s->partial, s->nparts, s->ph, s->ctl, dt_out, clip, t_end, st));
  return FLUID_OK;
}

int stage_into(fluid_solver* s, int stage, const double* Un, const double* Us, double* Ud,
               double t_end, cudaStream_t st) {
  FL_TIMED(s, FLUID_KERNEL_STAGE, st,
           fl::launch_stage(stage, Un, Us, s->R, Ud, s->W, s->geo, s->ph, s->ctl, t_end, st));
  return FLUID_OK;
}

// stage_into followed by the primitives of Ud (what rhs_into(Ud) computes first)
int stage_prim_into(fluid_solver* s, int stage, const double* Un, const double* Us, double* Ud,
                    double t_end, cudaStream_t st) {
  FL_TIMED(s, FLUID_KERNEL_STAGE, st,
           fl::launch_stage_prim(stage, Un, Us, s->R, Ud, s->W, s->W32, s->geo, s->ph, s->bc,
                                 s->ctl, t_end, st));
  return FLUID_OK;
}

// Mixed path, one RK3 stage from the primitives of its input (in W / W32): the face kernels of the
// axes before the last into R, then the last axis's face kernel fused with the stage combination
// into Ud and the primitives of Ud into the second buffer pair (prims), whose halo cells follow;
// the pairs then swap, so W / W32 hold the primitives of Ud.  Without prims (the last stage of a
// call) only Ud is written.
int stage_fused_into(fluid_solver* s, int stage, const double* Un, const double* Us, double* Ud,
                     bool prims, double t_end, cudaStream_t st) {
  const Geo& g = s->geo;
  if (s->ph.visc != FLUID_VISC_NONE)
    FL_TIMED(s, FLUID_KERNEL_GRAD, st, fl::launch_grad32(s->W32, s->G32, g, st));
  for (int d = 0; d + 1 < g.ndim; ++d)
    FL_TIMED(s, FLUID_KERNEL_FACE_X + d, st,
             fl::launch_face_mixed(d, s->W, s->W32, s->G32, s->R, g, s->ph, d > 0, s->face_block,
                                   s->face_seg, st, &s->ctl->flags));
  const fl::StageOut so{stage, prims ? 1 : 0, Un, Us, Ud, s->Wb, s->W32b, s->ctl, t_end};
  FL_TIMED(s, FLUID_KERNEL_FACE_X + g.ndim - 1, st,
           fl::launch_face_mixed_stage(s->W, s->W32, s->G32, s->R, g, s->ph, s->face_block, s->face_seg,
                                       so, st));
  if (prims) {
    FL_TIMED(s, FLUID_KERNEL_STAGE, st, fl::launch_halo_prim(s->Wb, s->W32b, g, s->ph, s->bc, s->ctl, st));
    std::swap(s->W, s->Wb);
    std::swap(s->W32, s->W32b);
  }
  return FLUID_OK;
}

// (dR/dX)^T mu on the interior into gX; (dR/dphi)^T mu added to gphi when given.  Wx / Gx: the
// primitives and gradients of X when already formed (else computed into the solver's W / G).
int rhs_vjp(fluid_solver* s, const double* X, const double* mu, double* gX, double* gphi,
            cudaStream_t st, double* Wx = nullptr, double* Gx = nullptr) {
  const Geo& g = s->geo;
  const bool visc = s->ph.visc != FLUID_VISC_NONE;
  double* W = Wx ? Wx : s->W;
  double* G = Wx ? Gx : s->G;
  if (!Wx) {
    FL_TIMED(s, FLUID_KERNEL_PRIM_BC, st, fl::launch_prim_bc(X, W, nullptr, g, s->ph, s->bc, s->ctl, st));
    if (visc) FL_TIMED(s, FLUID_KERNEL_GRAD, st, fl::launch_grad(W, G, g, s->ph, st));
  }
  FL_CUDA(s, cudaMemsetAsync(s->gW, 0, fl::NW * (size_t)g.ncell * sizeof(double), st));
  if (visc) FL_CUDA(s, cudaMemsetAsync(s->gG, 0, fl::NG * (size_t)g.ncell * sizeof(double), st));
  FL_CUDA(s, cudaMemsetAsync(s->gvw, 0, s->gvw_count * sizeof(double), st));
  FL_TIMED(s, FLUID_KERNEL_ADJ_FACE, st,
           fl::launch_adj_faces(W, G, mu, s->CW, s->CG, s->gW, s->gG, g, s->ph, st));
  if (s->ph.has_force) FL_TIMED(s, FLUID_KERNEL_ADJ_CELL, st, fl::launch_adj_source(mu, s->gW, g, s->ph, st));
  FL_TIMED(s, FLUID_KERNEL_ADJ_CELL, st, fl::launch_adj_bc(W, s->gW, s->gvw, g, s->ph, s->bc, st));
  FL_TIMED(s, FLUID_KERNEL_ADJ_CELL, st, fl::launch_adj_prim(X, s->gW, gX, g, s->ph, st));
  if (gphi && s->bc.porous_axis >= 0) {
    const int A = s->bc.porous_axis, t1 = s->bc.porous_t1, t2 = 3 - A - t1;
    FL_TIMED(s, FLUID_KERNEL_ADJ_CELL, st,
             fl::launch_adj_phi(s->gvw, g.xc[t1], gphi, g.p[t1], g.h[t1], g.p[t2], s->cfg.porous_begin,
                                s->cfg.porous_count, s->cfg.porous_A / s->cfg.porous_phi0,
                                2.0 * M_PI * s->cfg.porous_kappa, st));
  }
  return FLUID_OK;
}

int need_adjoint(fluid_solver* s) {
  if (!s->gW) return fail(s, FLUID_EINVAL, "create the solver with cfg.adjoint != 0");
  return FLUID_OK;
}

// entry points that run several right-hand sides without returning to the caller cannot refresh
// exchange halos in between
int no_exchange(fluid_solver* s, const char* what) {
  if (s->exchange)
    return fail(s, FLUID_EINVAL, std::string(what) +
                                     " cannot refresh exchange halos between stages: advance a "
                                     "sub-domain solver with fluid_rk3_stage");
  return FLUID_OK;
}

}  // namespace

namespace fl {
const char* config_error(const fluid_config* c) { return validate(c); }

bool batch_slot_of(fluid_solver* s, double* U, double t_end, BatchSlot& out) {
  if (!s || s->exchange || s->ph.weno == FLUID_TENO6A || s->ph.visc_order == 6) return false;
  out = BatchSlot{};
  out.g = s->geo;
  out.ph = s->ph;
  out.bc = s->bc;
  out.U = U;
  out.A = s->A;
  out.R = s->R;
  out.W = s->W;
  out.G = s->G;
  out.W32 = s->W32;
  out.G32 = s->G32;
  out.partial = s->partial;
  out.nparts = s->ph.dt_fixed > 0.0 ? 0 : s->nparts;
  out.ctl = s->ctl;
  out.t_end = t_end;
  for (int D = 0; D < 3; ++D) {
    out.seg[D] = 1;
    out.FB[D] = nullptr;
    if (D >= s->geo.ndim || s->mixed) continue;
    int block = 128, seg = s->face_seg_d[D], grid = 0;
    face_shape(D, s->geo, block, seg, grid);
    out.seg[D] = seg;
    out.FB[D] = seam_buffer(D, s->geo, seg, SeamBuf{s->FB, s->fb_cap});
  }
  return true;
}
}  // namespace fl

extern "C" {

int fluid_abi_version(void) { return FLUID_ABI_VERSION; }
size_t fluid_config_size(void) { return sizeof(fluid_config); }

const char* fluid_last_error(const fluid_solver* s) {
  return s ? s->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

namespace {
int create_impl(const fluid_config* cfg, fluid_solver** out, SolverAlloc al) {
  if (!out) return fail(nullptr, FLUID_EINVAL, "out is NULL");
  *out = nullptr;
  if (const char* why = validate(cfg)) return fail(nullptr, FLUID_EINVAL, why);
  fluid_solver* s = new (std::nothrow) fluid_solver();
  if (!s) return fail(nullptr, FLUID_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  s->alloc = al;
  const fluid_config& c = *cfg;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    delete s;
    return fail(nullptr, FLUID_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  Geo& g = s->geo;
  g.ndim = c.ndim;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = c.n[a];
    g.h[a] = a < c.ndim ? FLUID_HALO : 0;
    g.p[a] = g.n[a] + 2 * g.h[a];
  }
  g.sy = g.p[0];
  g.sz = g.p[0] * g.p[1];
  g.ncell = g.p[0] * g.p[1] * g.p[2];

  Phys& ph = s->ph;
  ph.gamma = c.gamma;
  ph.gm1 = c.gamma - 1.0;
  ph.igm1 = 1.0 / (c.gamma - 1.0);
  ph.R = c.gas_R;
  ph.iR = 1.0 / c.gas_R;
  ph.cp = c.gamma * c.gas_R / (c.gamma - 1.0);
  ph.Pr = c.prandtl;
  ph.lam_fac = ph.cp / c.prandtl;
  ph.mu_ref = c.mu_ref;
  ph.T_ref = c.T_ref;
  ph.iT_ref = c.T_ref > 0 ? 1.0 / c.T_ref : 1.0;
  set_power_law(ph, c.visc_exp);
  ph.suth_S = c.suth_S;
  ph.visc = c.visc_law;
  ph.weno = c.weno;
  ph.visc_order = c.visc_order == 6 ? 6 : 4;
  ph.eps = c.weno_eps > 0 ? c.weno_eps : (c.weno == FLUID_WENO_JS ? 1e-6 : 1e-40);
  ph.has_force = 0;
  for (int a = 0; a < 3; ++a) {
    ph.f[a] = c.body_force[a];
    ph.has_force |= c.body_force[a] != 0.0;
  }
  ph.cfl = c.cfl;
  ph.dt_fixed = c.dt_fixed;
  ph.dt_visc_k = 2.0 * std::fmax(4.0 / 3.0, c.gamma / c.prandtl);

  // device scratch
  const size_t nc = (size_t)g.ncell;
  size_t nmetric = 0;
  for (int a = 0; a < 3; ++a) nmetric += 5 * (size_t)g.p[a];
  s->nparts = fl::dt_partial_count(g);
  auto bail = [&](cudaError_t err, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(err);
    fluid_destroy(s);
    return fail(nullptr, err == cudaErrorMemoryAllocation ? FLUID_ENOMEM : FLUID_ECUDA, m);
  };
  if ((e = al.malloc((void**)&s->metric, nmetric * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc metric");
  s->mixed = c.precision == FLUID_PREC_MIXED;
  // the mixed path keeps H = E + p in one more FP64 row of W
  if ((e = al.malloc((void**)&s->W, (fl::NW + (s->mixed ? 1 : 0)) * nc * sizeof(double))) != cudaSuccess)
    return bail(e, "cudaMalloc W");
  if (s->mixed) {
    // W32 buffers: 64 floats of slack past the end for the aligned tails of bulk-staged rows
    if ((e = al.malloc((void**)&s->W32, (2 * fl::NW * nc + 64) * sizeof(float))) != cudaSuccess) return bail(e, "cudaMalloc W32");
    if ((e = al.malloc((void**)&s->Wb, (fl::NW + 1) * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc Wb");
    if ((e = al.malloc((void**)&s->W32b, (2 * fl::NW * nc + 64) * sizeof(float))) != cudaSuccess) return bail(e, "cudaMalloc W32b");
    if ((e = al.malloc((void**)&s->mf32, 3 * (nmetric / 5) * sizeof(float))) != cudaSuccess) return bail(e, "cudaMalloc mf32");
    if (c.visc_law != FLUID_VISC_NONE)
      if ((e = al.malloc((void**)&s->G32, fl::NG * nc * sizeof(float))) != cudaSuccess) return bail(e, "cudaMalloc G32");
  } else if (c.visc_law != FLUID_VISC_NONE) {
    if ((e = al.malloc((void**)&s->G, fl::NG * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc G");
  }
  if ((e = al.malloc((void**)&s->A, fl::NV * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc A");
  if ((e = al.malloc((void**)&s->R, fl::NV * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc R");
  if (!s->mixed) {
    s->fb_cap = fl::seam_capacity(g);
    if ((e = al.malloc((void**)&s->FB, 10 * (size_t)s->fb_cap * sizeof(double))) != cudaSuccess)
      return bail(e, "cudaMalloc FB");
  }
  if ((e = al.malloc((void**)&s->partial, s->nparts * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc partial");
  if ((e = al.malloc((void**)&s->ctl, sizeof(Ctl))) != cudaSuccess) return bail(e, "cudaMalloc ctl");
  Ctl c0{};
  if ((e = al.h2d(s->ctl, &c0, sizeof(Ctl))) != cudaSuccess) return bail(e, "ctl init");

  std::vector<double> all;
  all.reserve(nmetric);
  size_t off[3][5];
  for (int a = 0; a < 3; ++a) {
    std::vector<double> m[5];
    axis_metrics(c, a, g.h[a], m);
    s->host_xc[a] = m[0];
    s->host_dx[a] = m[1];
    for (int k = 0; k < 5; ++k) {
      off[a][k] = all.size();
      all.insert(all.end(), m[k].begin(), m[k].end());
    }
  }
  if ((e = al.h2d(s->metric, all.data(), all.size() * sizeof(double))) != cudaSuccess)
    return bail(e, "metric upload");
  if (s->mixed) {
    // FP32 copies (rounded to nearest, as the device conversion rounds) of the face metrics, the
    // centre metrics and the inverse widths, so that the FP32 kernels convert nothing per cell
    std::vector<float> m32;
    size_t off32[3][3];
    const int src[3] = {4, 3, 2};            // mf, mc, idx
    for (int q = 0; q < 3; ++q)
      for (int a = 0; a < 3; ++a) {
        off32[q][a] = m32.size();
        for (int k = 0; k < g.p[a]; ++k) m32.push_back((float)all[off[a][src[q]] + k]);
      }
    if ((e = al.h2d(s->mf32, m32.data(), m32.size() * sizeof(float))) != cudaSuccess)
      return bail(e, "metric upload");
    for (int a = 0; a < 3; ++a) {
      g.mf32[a] = s->mf32 + off32[0][a];
      g.mc32[a] = s->mf32 + off32[1][a];
      g.idx32[a] = s->mf32 + off32[2][a];
    }
  }
  for (int a = 0; a < 3; ++a) {
    g.xc[a] = s->metric + off[a][0];
    g.dx[a] = s->metric + off[a][1];
    g.idx[a] = s->metric + off[a][2];
    g.mc[a] = s->metric + off[a][3];
    g.mf[a] = s->metric + off[a][4];
  }

  BC& bc = s->bc;
  bc.porous_axis = -1;
  bc.porous_side = 0;
  bc.porous_t1 = 0;
  bc.vw = nullptr;
  for (int a = 0; a < 3; ++a)
    for (int sd = 0; sd < 2; ++sd) {
      bc.kind[a][sd] = a < c.ndim ? c.bc[a][sd] : FLUID_BC_PERIODIC;
      bc.Tw[a][sd] = c.t_wall[a][sd];
      bc.inflow[a][sd] = nullptr;
      if (a < c.ndim && c.bc[a][sd] == FLUID_BC_INFLOW) {
        const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
        const size_t cnt = 5 * (size_t)g.p[t1] * g.p[t2];
        if ((e = al.malloc((void**)&s->inflow[a][sd], cnt * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc inflow");
        if ((e = al.memset(s->inflow[a][sd], 0, cnt * sizeof(double))) != cudaSuccess) return bail(e, "inflow init");
        s->inflow_count[a][sd] = cnt;
        bc.inflow[a][sd] = s->inflow[a][sd];
      }
    }
  for (int a = 0; a < c.ndim; ++a)
    for (int sd = 0; sd < 2; ++sd) s->exchange |= c.bc[a][sd] == FLUID_BC_EXCHANGE;
  for (int a = 0; a < c.ndim; ++a)
    for (int sd = 0; sd < 2; ++sd)
      if (c.bc[a][sd] == FLUID_BC_POROUS) {
        bc.porous_axis = a;
        bc.porous_side = sd;
        bc.porous_t1 = a == 0 ? 1 : 0;
        const int t1 = bc.porous_t1;
        if ((e = al.malloc((void**)&s->vw, g.p[t1] * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc vw");
        if ((e = al.malloc((void**)&s->phi, c.porous_count * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc phi");
        std::vector<double> phi0(c.porous_count, c.porous_phi0);
        if ((e = al.h2d(s->phi, phi0.data(), phi0.size() * sizeof(double))) != cudaSuccess)
          return bail(e, "phi init");
        bc.vw = s->vw;
        if ((e = fl::launch_wall_velocity(s->phi, s->vw, g.xc[t1], g.p[t1], g.h[t1], c.porous_begin,
                                          c.porous_count, c.porous_A / c.porous_phi0,
                                          2.0 * M_PI * c.porous_kappa, al.st)) != cudaSuccess)
          return bail(e, "wall velocity");
        if (!al.async && (e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "wall velocity sync");
      }
  if (c.adjoint) {
    if (c.precision != FLUID_PREC_FP64) {
      fluid_destroy(s);
      return fail(nullptr, FLUID_ENOTSUP, "the adjoint is built for FLUID_PREC_FP64");
    }
    const bool visc = c.visc_law != FLUID_VISC_NONE;
    if ((e = al.malloc((void**)&s->gW, fl::NW * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc gW");
    if ((e = al.malloc((void**)&s->CW, 36 * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc CW");
    if (visc) {
      if ((e = al.malloc((void**)&s->gG, fl::NG * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc gG");
      if ((e = al.malloc((void**)&s->CG, 4 * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc CG");
    }
    if ((e = al.malloc((void**)&s->Wn, fl::NW * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc Wn");
    if ((e = al.malloc((void**)&s->W1, fl::NW * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc W1");
    if (visc) {
      if ((e = al.malloc((void**)&s->Gn, fl::NG * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc Gn");
      if ((e = al.malloc((void**)&s->G1, fl::NG * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc G1");
    }
    double** bufs[] = {&s->S1, &s->S2, &s->MU, &s->L1, &s->L2, &s->GT};
    for (double** b : bufs) {
      if ((e = al.malloc((void**)b, fl::NV * nc * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc adjoint state");
      if ((e = al.memset(*b, 0, fl::NV * nc * sizeof(double))) != cudaSuccess) return bail(e, "adjoint init");
    }
    // wall columns: every face plane of the grid is covered by the largest padded plane
    size_t plane = 0;
    for (int a = 0; a < 3; ++a) {
      const int t1 = a == 0 ? 1 : 0, t2 = 3 - a - t1;
      plane = std::max(plane, (size_t)g.p[t1] * g.p[t2]);
    }
    s->gvw_count = plane;
    if ((e = al.malloc((void**)&s->gvw, plane * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc gvw");
    if ((e = al.malloc((void**)&s->gT2, 2 * plane * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc gT2");
    s->nloss = 1024;
    if ((e = al.malloc((void**)&s->parts, s->nloss * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc parts");
  }
  *out = s;
  return FLUID_OK;
}
}  // namespace

namespace fl {
int solver_create_async(const fluid_config* cfg, cudaStream_t st, fluid_solver** out) {
  return create_impl(cfg, out, SolverAlloc{st, true});
}
}  // namespace fl

extern "C" {

int fluid_create(const fluid_config* cfg, fluid_solver** out) {
  return create_impl(cfg, out, SolverAlloc{});
}

void fluid_destroy(fluid_solver* s) {
  if (!s) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  // stream-ordered memory is released after the work already on its stream, without waiting
  if (!s->alloc.async) cudaDeviceSynchronize();
  const SolverAlloc& al = s->alloc;
  al.free(s->metric);
  al.free(s->W);
  al.free(s->G);
  al.free(s->W32);
  al.free(s->Wb);
  al.free(s->W32b);
  al.free(s->mf32);
  al.free(s->G32);
  for (double* p : {s->gW, s->gG, s->CW, s->CG, s->S1, s->S2, s->MU, s->L1, s->L2, s->GT, s->gvw,
                    s->parts, s->gT2, s->Wn, s->Gn, s->W1, s->G1})
    al.free(p);
  al.free(s->A);
  al.free(s->R);
  al.free(s->FB);
  al.free(s->partial);
  al.free(s->ctl);
  al.free(s->vw);
  al.free(s->phi);
  for (int a = 0; a < 3; ++a)
    for (int sd = 0; sd < 2; ++sd) al.free(s->inflow[a][sd]);
  for (auto* v : {&s->prof_pending, &s->prof_pool})
    for (auto& ev : *v) {
      cudaEventDestroy(ev.a);
      cudaEventDestroy(ev.b);
    }
  cudaSetDevice(cur);
  delete s;
}

int fluid_padded_dims(const fluid_solver* s, int32_t p[3]) {
  if (!s || !p) return FLUID_EINVAL;
  for (int a = 0; a < 3; ++a) p[a] = s->geo.p[a];
  return FLUID_OK;
}

int fluid_get_grid(const fluid_solver* s, int axis, double* xc, double* dx) {
  if (!s || axis < 0 || axis > 2) return FLUID_EINVAL;
  const size_t p = s->geo.p[axis];
  if (xc) std::memcpy(xc, s->host_xc[axis].data(), p * sizeof(double));
  if (dx) std::memcpy(dx, s->host_dx[axis].data(), p * sizeof(double));
  return FLUID_OK;
}

int fluid_set_wall_params(fluid_solver* s, const double* phi_dev, int n, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (s->bc.porous_axis < 0) return fail(s, FLUID_EINVAL, "no porous face in this configuration");
  if (n != s->cfg.porous_count) return fail(s, FLUID_EINVAL, "n must equal porous_count");
  if (int r = check_ptr(s, phi_dev, "phi_dev")) return r;
  cudaStream_t st = as_stream(stream);
  FL_CUDA(s, cudaMemcpyAsync(s->phi, phi_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const int t1 = s->bc.porous_t1;
  FL_CUDA(s, fl::launch_wall_velocity(s->phi, s->vw, s->geo.xc[t1], s->geo.p[t1], s->geo.h[t1],
                                      s->cfg.porous_begin, s->cfg.porous_count,
                                      s->cfg.porous_A / s->cfg.porous_phi0,
                                      2.0 * M_PI * s->cfg.porous_kappa, st));
  return FLUID_OK;
}

int fluid_set_inflow(fluid_solver* s, int axis, int side, const double* W_dev, size_t count,
                     void* stream) {
  if (!s) return FLUID_EINVAL;
  if (axis < 0 || axis > 2 || side < 0 || side > 1 || !s->inflow[axis][side])
    return fail(s, FLUID_EINVAL, "face is not an inflow face");
  if (count != s->inflow_count[axis][side]) return fail(s, FLUID_EINVAL, "inflow count mismatch");
  if (int r = check_ptr(s, W_dev, "W_dev")) return r;
  FL_CUDA(s, cudaMemcpyAsync(s->inflow[axis][side], W_dev, count * sizeof(double),
                             cudaMemcpyDeviceToDevice, as_stream(stream)));
  return FLUID_OK;
}

int fluid_prim_to_cons(fluid_solver* s, const double* W_dev, double* U_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = check_ptr(s, W_dev, "W_dev")) return r;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  FL_CUDA(s, fl::launch_prim_to_cons(W_dev, U_dev, s->geo.ncell, s->ph, as_stream(stream)));
  return FLUID_OK;
}

int fluid_rhs(fluid_solver* s, const double* U_dev, double* R_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (int r = check_ptr(s, R_dev, "R_dev")) return r;
  if (U_dev == R_dev) return fail(s, FLUID_EINVAL, "U and R must not alias");
  cudaStream_t st = as_stream(stream);
  if (int r = rhs_into(s, U_dev, R_dev, st)) return r;
  if (s->ph.has_force)
    FL_TIMED(s, FLUID_KERNEL_SOURCE, st, fl::launch_source(R_dev, s->W, s->geo, s->ph, st));
  return FLUID_OK;
}

int fluid_compute_dt(fluid_solver* s, const double* U_dev, double* dt_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (int r = check_ptr(s, dt_dev, "dt_dev")) return r;
  cudaStream_t st = as_stream(stream);
  FL_TIMED(s, FLUID_KERNEL_PRIM_BC, st, fl::launch_prim_bc(U_dev, s->W, s->W32, s->geo, s->ph, s->bc, s->ctl, st));
  return dt_into(s, dt_dev, 0, 0.0, st);
}

int fluid_step(fluid_solver* s, double* U_dev, int nsteps, double t_end, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = no_exchange(s, "fluid_step")) return r;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (nsteps < 0) return fail(s, FLUID_EINVAL, "nsteps < 0");
  cudaStream_t st = as_stream(stream);
  // Each stage's combination also writes the primitives of its result (stage_prim_into), so the
  // next right-hand side starts at its gradients; only the first step of a call converts U here,
  // and the call's last stage, whose primitives nothing reads, is the plain combination.
  if (nsteps > 0)
    FL_TIMED(s, FLUID_KERNEL_PRIM_BC, st, fl::launch_prim_bc(U_dev, s->W, s->W32, s->geo, s->ph, s->bc, s->ctl, st));
  // the mixed path on the y / z tile kernels folds each stage into the last axis's face kernel
  const bool fused = s->mixed && fl::mixed_stage_fusable(s->geo, s->face_seg);
  for (int k = 0; k < nsteps; ++k) {
    if (fused) {
      if (int r = dt_into(s, nullptr, 1, t_end, st)) return r;
      if (int r = stage_fused_into(s, 1, U_dev, U_dev, s->A, true, t_end, st)) return r;
      if (int r = stage_fused_into(s, 2, U_dev, s->A, s->A, true, t_end, st)) return r;
      if (int r = stage_fused_into(s, 3, U_dev, s->A, U_dev, k + 1 < nsteps, t_end, st)) return r;
      continue;
    }
    // stage 1: U1 = Un + dt R(Un) into A; dt from the primitives of Un
    if (int r = dt_into(s, nullptr, 1, t_end, st)) return r;
    if (int r = grad_faces(s, s->R, st)) return r;
    if (int r = stage_prim_into(s, 1, U_dev, U_dev, s->A, t_end, st)) return r;
    // stage 2: U2 = 3/4 Un + 1/4 (U1 + dt R(U1)) into A
    if (int r = grad_faces(s, s->R, st)) return r;
    if (int r = stage_prim_into(s, 2, U_dev, s->A, s->A, t_end, st)) return r;
    // stage 3: Un+1 = 1/3 Un + 2/3 (U2 + dt R(U2)) into U
    if (int r = grad_faces(s, s->R, st)) return r;
    if (k + 1 < nsteps) {
      if (int r = stage_prim_into(s, 3, U_dev, s->A, U_dev, t_end, st)) return r;
    } else if (int r = stage_into(s, 3, U_dev, s->A, U_dev, t_end, st)) {
      return r;
    }
  }
  return FLUID_OK;
}

int fluid_step_stages(fluid_solver* s, double* U_dev, double* U1_dev, double* U2_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = no_exchange(s, "fluid_step_stages")) return r;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (int r = check_ptr(s, U1_dev, "U1_dev")) return r;
  if (int r = check_ptr(s, U2_dev, "U2_dev")) return r;
  cudaStream_t st = as_stream(stream);
  FL_TIMED(s, FLUID_KERNEL_PRIM_BC, st, fl::launch_prim_bc(U_dev, s->W, s->W32, s->geo, s->ph, s->bc, s->ctl, st));
  if (int r = dt_into(s, nullptr, 1, 0.0, st)) return r;
  if (int r = grad_faces(s, s->R, st)) return r;
  if (int r = stage_into(s, 1, U_dev, U_dev, U1_dev, 0.0, st)) return r;
  if (int r = rhs_into(s, U1_dev, s->R, st)) return r;
  if (int r = stage_into(s, 2, U_dev, U1_dev, U2_dev, 0.0, st)) return r;
  if (int r = rhs_into(s, U2_dev, s->R, st)) return r;
  return stage_into(s, 3, U_dev, U2_dev, U_dev, 0.0, st);
}

int fluid_adjoint_rhs(fluid_solver* s, const double* U_dev, const double* mu_dev, double* gU_dev,
                      double* gphi_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = need_adjoint(s)) return r;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (int r = check_ptr(s, mu_dev, "mu_dev")) return r;
  if (int r = check_ptr(s, gU_dev, "gU_dev")) return r;
  return rhs_vjp(s, U_dev, mu_dev, gU_dev, gphi_dev, as_stream(stream));
}

int fluid_adjoint_step(fluid_solver* s, const double* Un_dev, const double* U1_dev,
                       const double* U2_dev, double* lam_dev, double* gphi_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = need_adjoint(s)) return r;
  if (!(s->ph.dt_fixed > 0.0)) return fail(s, FLUID_EINVAL, "the step adjoint needs a frozen dt (cfg.dt_fixed > 0)");
  if (int r = check_ptr(s, Un_dev, "Un_dev")) return r;
  if (int r = check_ptr(s, lam_dev, "lam_dev")) return r;
  if ((U1_dev == nullptr) != (U2_dev == nullptr)) return fail(s, FLUID_EINVAL, "pass both stage states or neither");
  const double dt = s->ph.dt_fixed;
  const Geo& g = s->geo;
  cudaStream_t st = as_stream(stream);
  const double* X1 = U1_dev;
  const double* X2 = U2_dev;
  const bool recompute = !X1;
  if (recompute) {
    // recompute the stage states of the step; the primitives and gradients of Un and U1 go to
    // Wn / Gn and W1 / G1, where the reverse passes of those stages find them
    struct Restore {
      fluid_solver* s;
      double *W, *G;
      ~Restore() { s->W = W; s->G = G; }
    } restore{s, s->W, s->G};
    s->W = s->Wn;
    s->G = s->Gn;
    if (int r = rhs_into(s, Un_dev, s->R, st)) return r;
    FL_TIMED(s, FLUID_KERNEL_STAGE, st, fl::launch_stage(1, Un_dev, Un_dev, s->R, s->S1, s->W, g, s->ph, s->ctl, 0.0, st, dt));
    s->W = s->W1;
    s->G = s->G1;
    if (int r = rhs_into(s, s->S1, s->R, st)) return r;
    FL_TIMED(s, FLUID_KERNEL_STAGE, st, fl::launch_stage(2, Un_dev, s->S1, s->R, s->S2, s->W, g, s->ph, s->ctl, 0.0, st, dt));
    X1 = s->S1;
    X2 = s->S2;
  }
  // Un+1 = 1/3 Un + 2/3 U2 + 2/3 dt R(U2)
  FL_CUDA(s, fl::launch_lincomb(s->MU, 2.0 / 3.0 * dt, lam_dev, 0, nullptr, 0, nullptr, 0, nullptr, g, st));
  if (int r = rhs_vjp(s, X2, s->MU, s->GT, gphi_dev, st)) return r;
  FL_CUDA(s, fl::launch_lincomb(s->L2, 2.0 / 3.0, lam_dev, 1.0, s->GT, 0, nullptr, 0, nullptr, g, st));
  // U2 = 3/4 Un + 1/4 U1 + 1/4 dt R(U1)
  FL_CUDA(s, fl::launch_lincomb(s->MU, 0.25 * dt, s->L2, 0, nullptr, 0, nullptr, 0, nullptr, g, st));
  if (int r = rhs_vjp(s, X1, s->MU, s->GT, gphi_dev, st, recompute ? s->W1 : nullptr, s->G1)) return r;
  FL_CUDA(s, fl::launch_lincomb(s->L1, 0.25, s->L2, 1.0, s->GT, 0, nullptr, 0, nullptr, g, st));
  // U1 = Un + dt R(Un)
  FL_CUDA(s, fl::launch_lincomb(s->MU, dt, s->L1, 0, nullptr, 0, nullptr, 0, nullptr, g, st));
  if (int r = rhs_vjp(s, Un_dev, s->MU, s->GT, gphi_dev, st, recompute ? s->Wn : nullptr, s->Gn)) return r;
  FL_CUDA(s, fl::launch_lincomb(lam_dev, 1.0 / 3.0, lam_dev, 0.75, s->L2, 1.0, s->L1, 1.0, s->GT, g, st));
  return FLUID_OK;
}

int fluid_wall_fluxes(fluid_solver* s, const double* U_dev, int axis, int side, double* qw_dev,
                      double* tw_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (!qw_dev && !tw_dev) return fail(s, FLUID_EINVAL, "qw_dev and tw_dev are both NULL");
  if (axis < 0 || axis >= s->geo.ndim || side < 0 || side > 1 || s->geo.ndim < 2)
    return fail(s, FLUID_EINVAL, "bad wall face");
  const int kind = s->bc.kind[axis][side];
  if (kind != FLUID_BC_WALL && kind != FLUID_BC_POROUS)
    return fail(s, FLUID_EINVAL, "wall fluxes need an isothermal or porous face");
  cudaStream_t st = as_stream(stream);
  FL_TIMED(s, FLUID_KERNEL_PRIM_BC, st, fl::launch_prim_bc(U_dev, s->W, s->W32, s->geo, s->ph, s->bc, s->ctl, st));
  FL_CUDA(s, fl::launch_wall_fluxes(s->W, qw_dev, tw_dev, s->geo, s->ph, axis, side, s->bc.Tw[axis][side], st));
  return FLUID_OK;
}

int fluid_wall_heat_loss(fluid_solver* s, const double* U_dev, int axis, int side, double* J_dev,
                         double* dJdU_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = no_exchange(s, "fluid_wall_heat_loss")) return r;
  if (int r = need_adjoint(s)) return r;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (int r = check_ptr(s, J_dev, "J_dev")) return r;
  if (axis < 0 || axis >= s->geo.ndim || side < 0 || side > 1) return fail(s, FLUID_EINVAL, "bad wall face");
  const int kind = s->bc.kind[axis][side];
  if (kind != FLUID_BC_WALL && kind != FLUID_BC_POROUS)
    return fail(s, FLUID_EINVAL, "the wall heat flux needs an isothermal or porous face");
  cudaStream_t st = as_stream(stream);
  const Geo& g = s->geo;
  const int nparts = std::min(s->nloss, fl::wall_loss_parts(g, axis));
  FL_CUDA(s, fl::launch_prim_bc(U_dev, s->W, nullptr, g, s->ph, s->bc, s->ctl, st));
  FL_CUDA(s, fl::launch_wall_loss(s->W, s->parts, nparts, J_dev, dJdU_dev ? s->gT2 : nullptr, g, s->ph,
                                  axis, side, s->bc.Tw[axis][side], st));
  if (dJdU_dev) {
    FL_CUDA(s, cudaMemsetAsync(dJdU_dev, 0, fl::NV * (size_t)g.ncell * sizeof(double), st));
    FL_CUDA(s, fl::launch_wall_loss_grad(U_dev, s->gT2, dJdU_dev, g, s->ph, axis, side, st));
  }
  return FLUID_OK;
}

int fluid_halo_count(const fluid_solver* s, int axis, size_t* count) {
  if (!s || !count || axis < 0 || axis >= s->geo.ndim) return FLUID_EINVAL;
  *count = fl::halo_count(s->geo, axis);
  return FLUID_OK;
}

int fluid_pack_halo(fluid_solver* s, const double* U_dev, int axis, int side, double* buf_dev,
                    void* stream) {
  if (!s) return FLUID_EINVAL;
  if (axis < 0 || axis >= s->geo.ndim || side < 0 || side > 1) return fail(s, FLUID_EINVAL, "bad face");
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (int r = check_ptr(s, buf_dev, "buf_dev")) return r;
  FL_CUDA(s, fl::launch_halo_copy(const_cast<double*>(U_dev), buf_dev, s->geo, axis, side, false,
                                  as_stream(stream)));
  return FLUID_OK;
}

int fluid_unpack_halo(fluid_solver* s, double* U_dev, int axis, int side, const double* buf_dev,
                      void* stream) {
  if (!s) return FLUID_EINVAL;
  if (axis < 0 || axis >= s->geo.ndim || side < 0 || side > 1) return fail(s, FLUID_EINVAL, "bad face");
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (int r = check_ptr(s, buf_dev, "buf_dev")) return r;
  FL_CUDA(s, fl::launch_halo_copy(U_dev, const_cast<double*>(buf_dev), s->geo, axis, side, true,
                                  as_stream(stream)));
  return FLUID_OK;
}

int fluid_rk3_stage(fluid_solver* s, int stage, const double* Un_dev, const double* Us_dev,
                    double* Ud_dev, double dt, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (stage < 1 || stage > 3) return fail(s, FLUID_EINVAL, "stage must be 1, 2 or 3");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(s, FLUID_EINVAL, "dt must be finite and > 0");
  if (int r = check_ptr(s, Un_dev, "Un_dev")) return r;
  if (int r = check_ptr(s, Us_dev, "Us_dev")) return r;
  if (int r = check_ptr(s, Ud_dev, "Ud_dev")) return r;
  if (stage == 1 && Us_dev != Un_dev) return fail(s, FLUID_EINVAL, "stage 1 needs Us == Un");
  cudaStream_t st = as_stream(stream);
  if (int r = rhs_into(s, Us_dev, s->R, st)) return r;
  FL_TIMED(s, FLUID_KERNEL_STAGE, st,
           fl::launch_stage(stage, Un_dev, Us_dev, s->R, Ud_dev, s->W, s->geo, s->ph, s->ctl, 0.0,
                            st, dt));
  return FLUID_OK;
}

int fluid_get_time(fluid_solver* s, double* t, double* last_dt, void* stream) {
  if (!s) return FLUID_EINVAL;
  Ctl h;
  cudaStream_t st = as_stream(stream);
  FL_CUDA(s, cudaMemcpyAsync(&h, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  FL_CUDA(s, cudaStreamSynchronize(st));
  if (t) *t = h.t;
  if (last_dt) *last_dt = h.dt;
  return FLUID_OK;
}

int fluid_set_time(fluid_solver* s, double t, void* stream) {
  if (!s) return FLUID_EINVAL;
  cudaStream_t st = as_stream(stream);
  FL_CUDA(s, cudaMemcpyAsync(&s->ctl->t, &t, sizeof(double), cudaMemcpyHostToDevice, st));
  FL_CUDA(s, cudaStreamSynchronize(st));
  return FLUID_OK;
}

int fluid_check(fluid_solver* s, void* stream) {
  if (!s) return FLUID_EINVAL;
  cudaStream_t st = as_stream(stream);
  unsigned flags = 0;
  FL_CUDA(s, cudaStreamSynchronize(st));
  FL_CUDA(s, cudaGetLastError());
  FL_CUDA(s, cudaMemcpy(&flags, &s->ctl->flags, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (flags) {
    const unsigned zero = 0;
    FL_CUDA(s, cudaMemcpy(&s->ctl->flags, &zero, sizeof(unsigned), cudaMemcpyHostToDevice));
    if (flags & fl::FLAG_STAGING)
      return fail(s, FLUID_ECUDA, "a bulk copy into shared memory did not complete within its wait limit");
    return fail(s, FLUID_ENONFINITE,
                (flags & fl::FLAG_GHOST_T) ? "non-positive ghost temperature at an isothermal wall"
                                           : "non-finite value in the state");
  }
  return FLUID_OK;
}

int fluid_tune_faces(fluid_solver* s, int block, int seg) {
  if (!s) return FLUID_EINVAL;
  if (block != 0 && (block < 32 || block > 128 || block % 32 != 0))
    return fail(s, FLUID_EINVAL, "block must be 0 or a multiple of 32 in [32, 128]");
  if (seg < 0 && !s->mixed) return fail(s, FLUID_EINVAL, "seg must be >= 0 for the FP64 path");
  s->face_block = block;
  s->face_seg = seg;
  for (int d = 0; d < 3; ++d) {
    s->face_seg_d[d] = seg;
    s->face_block_d[d] = block;
  }
  return FLUID_OK;
}

int fluid_autotune_faces(fluid_solver* s, const double* U_dev, void* stream) {
  if (!s) return FLUID_EINVAL;
  if (int r = check_ptr(s, U_dev, "U_dev")) return r;
  if (s->mixed) return FLUID_OK;
  cudaStream_t st = as_stream(stream);
  const Geo& g = s->geo;
  FL_CUDA(s, fl::launch_prim_bc(U_dev, s->W, s->W32, g, s->ph, s->bc, s->ctl, st));
  if (s->ph.visc != FLUID_VISC_NONE) FL_CUDA(s, fl::launch_grad(s->W, s->G, g, s->ph, st));
  cudaEvent_t e0, e1;
  FL_CUDA(s, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(s, FLUID_ECUDA, "cudaEventCreate");
  }
  // candidates: the automatic rule (0) and segments of 8 to 32 cells with blocks of 128 threads,
  // then blocks of 64 and 32 threads with the fastest segment length
  static const int kCand[] = {0, 8, 10, 12, 14, 16, 17, 18, 19, 20, 22, 24, 28, 32};
  cudaError_t e = cudaSuccess;
  for (int d = 0; d < g.ndim && e == cudaSuccess; ++d) {
    int best_seg = 0, best_block = 128;
    float best_ms = 0.0f;
    bool have = false;
    auto trial = [&](int block, int seg) {
      auto launch = [&]() {
        return fl::launch_face(d, s->W, s->G, s->R, g, s->ph, 0, block, seg, fl::SeamBuf{s->FB, s->fb_cap}, st);
      };
      if ((e = launch()) != cudaSuccess) return;                      // warm-up
      if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return;
      for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch();
      if (e != cudaSuccess || (e = cudaEventRecord(e1, st)) != cudaSuccess) return;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return;
      float ms = 0.0f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return;
      if (!have || ms < best_ms) {
        have = true;
        best_ms = ms;
        best_seg = seg;
        best_block = block;
      }
    };
    for (int c : kCand) {
      if (c > g.n[d]) continue;
      trial(128, c);
      if (e != cudaSuccess) break;
    }
    for (int b : {64, 32}) {
      if (e != cudaSuccess) break;
      trial(b, best_seg);
    }
    if (e == cudaSuccess) {
      s->face_seg_d[d] = best_seg;
      s->face_block_d[d] = best_block;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(s, e, "fluid_autotune_faces");
  return FLUID_OK;
}

int fluid_profile_enable(fluid_solver* s, int enable) {
  if (!s) return FLUID_EINVAL;
  s->prof_on = enable != 0;
  return FLUID_OK;
}

int fluid_profile_read(fluid_solver* s, int kind, double* total_ms, int64_t* launches, int reset) {
  if (!s || kind < 0 || kind >= FLUID_KERNEL_COUNT) return FLUID_EINVAL;
  for (auto& ev : s->prof_pending) {
    FL_CUDA(s, cudaEventSynchronize(ev.b));
    float ms = 0.f;
    FL_CUDA(s, cudaEventElapsedTime(&ms, ev.a, ev.b));
    s->prof_ms[ev.kind] += ms;
    s->prof_n[ev.kind] += ev.kernels;
    s->prof_pool.push_back(ev);
  }
  s->prof_pending.clear();
  if (total_ms) *total_ms = s->prof_ms[kind];
  if (launches) *launches = s->prof_n[kind];
  if (reset)
    for (int k = 0; k < FLUID_KERNEL_COUNT; ++k) {
      s->prof_ms[k] = 0.0;
      s->prof_n[k] = 0;
    }
  return FLUID_OK;
}

}  // extern "C"
