// Internal definitions shared by the solver's CUDA translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fluid.h"

namespace fl {

constexpr int NV = 5;   // conservative variables (rho, rho u, rho v, rho w, E)
constexpr int NW = 6;   // primitive scratch (rho, u, v, w, p, T)
constexpr int NG = 9;   // velocity-gradient scratch, component c * 3 + b = d u_c / d x_b

// flag bits of Ctl::flags
constexpr unsigned FLAG_NONFINITE = 1u;
constexpr unsigned FLAG_GHOST_T = 2u;

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
};

struct Phys {
  double gamma, gm1, igm1, R, iR, cp, Pr, lam_fac;
  double mu_ref, T_ref, iT_ref, visc_exp, suth_S;
  int visc, weno;
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

__device__ __forceinline__ double viscosity(double T, const Phys& ph) {
  if (ph.visc == FLUID_VISC_CONSTANT) return ph.mu_ref;
  const double r = T * ph.iT_ref;
  if (ph.visc == FLUID_VISC_POWER) return ph.mu_ref * exp(ph.visc_exp * log(r));
  // Sutherland
  return ph.mu_ref * (r * sqrt(r)) * (ph.T_ref + ph.suth_S) / (T + ph.suth_S);
}

// Configuration check shared by the entry points: NULL if valid, else a static message.
const char* config_error(const fluid_config* c);

// ---- launchers implemented in kernels_fp64.cu --------------------------------------------------
// W32 (optional, may be null): FP32 copy of the primitives for the mixed-precision path
cudaError_t launch_prim_bc(const double* U, double* W, float* W32, const Geo& g, const Phys& ph,
                           const BC& bc, Ctl* ctl, cudaStream_t st);
cudaError_t launch_grad(const double* W, double* G, const Geo& g, cudaStream_t st);
cudaError_t launch_face(int D, const double* W, const double* G, double* R, const Geo& g,
                        const Phys& ph, int accumulate, int block, int seg, cudaStream_t st);
cudaError_t launch_source(double* R, const double* W, const Geo& g, const Phys& ph, cudaStream_t st);
cudaError_t launch_stage(int stage, const double* Un, const double* Us, const double* R, double* Ud,
                         const double* W, const Geo& g, const Phys& ph, Ctl* ctl, double t_end,
                         cudaStream_t st);
cudaError_t launch_dt_partial(const double* W, const Geo& g, const Phys& ph, double* partial,
                              int nparts, cudaStream_t st);
cudaError_t launch_dt_final(const double* partial, int nparts, const Phys& ph, Ctl* ctl,
                            double* dt_out, int clip_to_ctl, double t_end, cudaStream_t st);
int dt_partial_count(const Geo& g);
// ---- mixed-precision launchers implemented in kernels_mixed.cu --------------------------------
cudaError_t launch_face_mixed(int D, const double* W, const float* W32, const float* G32, double* R,
                              const Geo& g, const Phys& ph, int accumulate, int block, int seg,
                              cudaStream_t st);
cudaError_t launch_grad32(const float* W32, float* G32, const Geo& g, cudaStream_t st);
cudaError_t launch_dt_partial32(const float* W32, const Geo& g, const Phys& ph, double* partial,
                                int nparts, cudaStream_t st);

cudaError_t launch_prim_to_cons(const double* W, double* U, int ncell, const Phys& ph,
                                cudaStream_t st);
cudaError_t launch_wall_velocity(const double* phi, double* vw, const double* xc, int p, int h,
                                 int begin, int count, double amp, double two_pi_kappa,
                                 cudaStream_t st);

}  // namespace fl
