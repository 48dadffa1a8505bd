// fluid_rhs_noalloc: the right-hand side of fluid_rhs for callers that cannot allocate device
// memory, with all scratch in one fixed, file-scope device array.
//
// Who needs it: a host whose device memory belongs to its own pool or arena and which forbids
// allocations behind its back, or a latency-critical caller that cannot afford cudaMalloc's
// implicit device synchronisation.  fluid_create allocates its scratch with cudaMalloc; this entry
// point takes the configuration directly and allocates nothing, on the device or the host.
//
// The scratch array below is reserved in every process that loads the library, on every GPU the
// process uses, until the process exits.  Host code must not use its name as a device pointer
// (in host code the symbol is only a host-side shadow); the device address is looked up once per
// device with cudaGetSymbolAddress and cached.  The cache belongs to the device's primary context:
// after cudaDeviceReset the array has a new address, which the cache does not know, so a process
// that resets a device must not call this entry point on it again.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fluid_internal.cuh"

namespace {

// 2^21 doubles = 16 MiB: primitives (6), velocity gradients (9), grid metrics and flags.
constexpr size_t kScratchDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

void put_msg(char* buf, size_t len, const char* msg) {
  if (buf && len > 0) {
    std::strncpy(buf, msg, len - 1);
    buf[len - 1] = '\0';
  }
}

size_t align32(size_t n) { return (n + 31) & ~size_t(31); }

// grid metrics of one axis over its padded range (same mapping as the solver's grid set-up):
// xc, dx, 1/dx, d(index)/dx at centres and at faces a+1/2
__device__ void axis_map(int stretch, double beta, double lo, double hi, double eta, double* x,
                         double* dxdeta) {
  const double L = hi - lo;
  if (stretch == FLUID_STRETCH_UNIFORM) {
    *x = lo + L * eta;
    *dxdeta = L;
    return;
  }
  const double tb = tanh(beta);
  const double t = stretch == FLUID_STRETCH_TANH2 ? tanh(beta * (2.0 * eta - 1.0)) : tanh(beta * (1.0 - eta));
  *x = stretch == FLUID_STRETCH_TANH2 ? lo + 0.5 * L * (1.0 + t / tb) : lo + L * (1.0 - t / tb);
  *dxdeta = L * beta * (1.0 - t * t) / tb;
}

struct AxisArgs {
  int n[3], h[3], p[3], stretch[3];
  double lo[3], hi[3], beta[3];
  double* out[3];          // 5 consecutive arrays of length p[a]
  double* vw;              // porous velocities (length p[t1]) or null
  int t1, begin, count;
  double amp, phi0, two_pi_kappa;
};

__global__ void k_noalloc_metrics(AxisArgs A) {
  for (int a = 0; a < 3; ++a) {
    const int p = A.p[a], n = A.n[a], h = A.h[a];
    double* xc = A.out[a];
    double* dx = xc + p;
    double* idx = dx + p;
    double* mc = idx + p;
    double* mf = mc + p;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p; i += gridDim.x * blockDim.x) {
      const double ai = (double)(i - h);
      if (A.stretch[a] == FLUID_STRETCH_UNIFORM) {
        const double d = (A.hi[a] - A.lo[a]) / n;
        xc[i] = A.lo[a] + (ai + 0.5) * d;
        dx[i] = d;
        idx[i] = 1.0 / d;
        mc[i] = 1.0 / d;
        mf[i] = 1.0 / d;
      } else {
        double x0, x1, dd, dc, df;
        axis_map(A.stretch[a], A.beta[a], A.lo[a], A.hi[a], (double)(i - h) / n, &x0, &dd);
        axis_map(A.stretch[a], A.beta[a], A.lo[a], A.hi[a], (double)(i + 1 - h) / n, &x1, &dd);
        axis_map(A.stretch[a], A.beta[a], A.lo[a], A.hi[a], (ai + 0.5) / n, &dd, &dc);
        axis_map(A.stretch[a], A.beta[a], A.lo[a], A.hi[a], (ai + 1.0) / n, &dd, &df);
        dx[i] = x1 - x0;
        xc[i] = 0.5 * (x1 + x0);
        idx[i] = 1.0 / dx[i];
        mc[i] = n / dc;
        mf[i] = n / df;
      }
    }
  }
}

// porous-wall velocities with every parameter at its reference value (phi_i = phi0); needs the
// centres written by k_noalloc_metrics, hence a second launch
__global__ void k_noalloc_wall(AxisArgs A) {
  const double* xc = A.out[A.t1];
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < A.p[A.t1]; a += gridDim.x * blockDim.x) {
    const int i = a - A.h[A.t1] - A.begin;
    A.vw[a] = (i >= 0 && i < A.count) ? A.amp * A.phi0 * sin(A.two_pi_kappa * xc[a]) : 0.0;
  }
}

// Device address of g_scratch on the current device, looked up once per device.
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int fluid_rhs_noalloc(const fluid_config* cfg, const double* U_dev, double* R_dev,
                                 void* stream, char* errbuf, size_t errlen) {
  if (const char* why = fl::config_error(cfg)) {
    put_msg(errbuf, errlen, why);
    return FLUID_EINVAL;
  }
  const fluid_config& c = *cfg;
  if (!U_dev || !R_dev || reinterpret_cast<uintptr_t>(U_dev) % 8 || reinterpret_cast<uintptr_t>(R_dev) % 8) {
    put_msg(errbuf, errlen, "U_dev and R_dev must be non-NULL and 8-byte aligned");
    return FLUID_EINVAL;
  }
  if (U_dev == R_dev) {
    put_msg(errbuf, errlen, "U and R must not alias");
    return FLUID_EINVAL;
  }
  if (c.precision != FLUID_PREC_FP64) {
    put_msg(errbuf, errlen, "the allocation-free entry point computes in FP64 only");
    return FLUID_ENOTSUP;
  }
  for (int a = 0; a < c.ndim; ++a)
    for (int s = 0; s < 2; ++s) {
      if (c.bc[a][s] == FLUID_BC_INFLOW) {
        put_msg(errbuf, errlen, "inflow faces need a profile: use fluid_create/fluid_set_inflow");
        return FLUID_ENOTSUP;
      }
      if (c.bc[a][s] == FLUID_BC_EXCHANGE) {
        put_msg(errbuf, errlen, "sub-domain (exchange) faces need fluid_create");
        return FLUID_ENOTSUP;
      }
    }
  for (int a = 0; a < 3; ++a)
    if (c.global_n[a] != 0) {
      put_msg(errbuf, errlen, "blocks of a decomposed grid (global_n) need fluid_create");
      return FLUID_ENOTSUP;
    }

  fl::Geo g{};
  g.ndim = c.ndim;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = c.n[a];
    g.h[a] = a < c.ndim ? FLUID_HALO : 0;
    g.p[a] = g.n[a] + 2 * g.h[a];
  }
  g.sy = g.p[0];
  g.sz = g.p[0] * g.p[1];
  g.ncell = g.p[0] * g.p[1] * g.p[2];
  const bool visc = c.visc_law != FLUID_VISC_NONE;
  const int porous_t1 = c.porous_axis == 0 ? 1 : 0;
  bool porous = false;
  for (int a = 0; a < c.ndim; ++a)
    for (int s = 0; s < 2; ++s) porous |= c.bc[a][s] == FLUID_BC_POROUS;

  // layout of the scratch: W | G | metrics (x, y, z) | vw | control block
  const size_t nc = (size_t)g.ncell;
  const size_t offW = 0;
  const size_t offG = offW + align32(fl::NW * nc);
  size_t off = offG + (visc ? align32(fl::NG * nc) : 0);
  size_t offM[3];
  for (int a = 0; a < 3; ++a) {
    offM[a] = off;
    off += align32(5 * (size_t)g.p[a]);
  }
  const size_t offV = off;
  off += porous ? align32(g.p[porous_t1]) : 0;
  const size_t offC = off;
  off += align32((sizeof(fl::Ctl) + 7) / 8);
  if (off > kScratchDoubles) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "grid needs %zu scratch doubles (%d per padded cell for %zu padded cells, plus "
                  "metrics), the fixed array holds %zu (16 MiB)",
                  off, fl::NW + (visc ? fl::NG : 0), nc, kScratchDoubles);
    put_msg(errbuf, errlen, msg);
    return FLUID_EINVAL;
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices)) e = cudaErrorInvalidDevice;
  double* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) {
    put_msg(errbuf, errlen, cudaGetErrorString(e));
    return FLUID_ECUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* W = base + offW;
  double* G = visc ? base + offG : nullptr;
  fl::Ctl* ctl = reinterpret_cast<fl::Ctl*>(base + offC);

  fl::Phys ph{};
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

  AxisArgs A{};
  for (int a = 0; a < 3; ++a) {
    A.n[a] = g.n[a];
    A.h[a] = g.h[a];
    A.p[a] = g.p[a];
    A.stretch[a] = c.stretch[a];
    A.lo[a] = c.lo[a];
    A.hi[a] = c.hi[a];
    A.beta[a] = c.beta[a];
    A.out[a] = base + offM[a];
    g.xc[a] = A.out[a];
    g.dx[a] = A.out[a] + g.p[a];
    g.idx[a] = A.out[a] + 2 * g.p[a];
    g.mc[a] = A.out[a] + 3 * g.p[a];
    g.mf[a] = A.out[a] + 4 * g.p[a];
  }
  fl::BC bc{};
  bc.porous_axis = -1;
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s) {
      bc.kind[a][s] = a < c.ndim ? c.bc[a][s] : FLUID_BC_PERIODIC;
      bc.Tw[a][s] = c.t_wall[a][s];
      bc.inflow[a][s] = nullptr;
    }
  if (porous) {
    bc.porous_axis = c.porous_axis;
    bc.porous_side = c.porous_side;
    bc.porous_t1 = porous_t1;
    bc.vw = base + offV;
    A.vw = base + offV;
    A.t1 = porous_t1;
    A.begin = c.porous_begin;
    A.count = c.porous_count;
    A.amp = c.porous_A / c.porous_phi0;
    A.phi0 = c.porous_phi0;
    A.two_pi_kappa = 2.0 * M_PI * c.porous_kappa;
  }

  // the flags word of the control block must start at zero; W and G are written before read
  e = cudaMemsetAsync(ctl, 0, sizeof(fl::Ctl), st);
  if (e == cudaSuccess) {
    k_noalloc_metrics<<<8, 128, 0, st>>>(A);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && porous) {
    k_noalloc_wall<<<4, 128, 0, st>>>(A);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = fl::launch_prim_bc(U_dev, W, nullptr, g, ph, bc, ctl, st);
  if (e == cudaSuccess && visc) e = fl::launch_grad(W, G, g, ph, st);
  for (int d = 0; e == cudaSuccess && d < g.ndim; ++d)
    e = fl::launch_face(d, W, G, R_dev, g, ph, d > 0, 0, 0, fl::SeamBuf{nullptr, 0}, st);
  if (e == cudaSuccess && ph.has_force) e = fl::launch_source(R_dev, W, g, ph, st);
  if (e != cudaSuccess) {
    put_msg(errbuf, errlen, cudaGetErrorString(e));
    return FLUID_ECUDA;
  }
  return FLUID_OK;
}
