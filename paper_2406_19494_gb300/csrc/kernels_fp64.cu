// FP64 kernels of the finite-volume compressible Navier-Stokes right-hand side (Section 2.1,
// Eq. ODE) and of the TVD-RK3 step.
//
// Pipeline of one right-hand-side evaluation:
//   k_prim_bc   primitives (rho, u, v, w, p, T) of every padded cell; halo cells are built directly
//               from interior cells by composing the boundary maps of the active axes in x, y, z
//               order (Section 3.2: halo cells take values assigned by the boundary conditions)
//   k_grad      fourth-order central velocity gradients at cell centres (tangential derivatives of
//               the dissipative fluxes)
//   k_face<D>   per axis D: WENO5 reconstruction of the primitives, HLLC convective flux, the
//               dissipative flux at the same face, and the flux difference -(F+ - F-)/dx into R.
//               One thread marches along a segment of a grid line so each face is computed once
//               and reused by the two cells that share it.
//   k_source / k_stage   body-force source, RK3 stage combination, non-finite check
//   k_dt_*      CFL time step: per-block minimum, then one block reduces (deterministic)
//
// The state is FP64 structure-of-arrays U[v][z][y][x]; primitives and gradients live in solver
// scratch with the same padded layout.
#include <cuda_runtime.h>

#include "fluid_internal.cuh"

namespace fl {

namespace {

constexpr double kSixth = 1.0 / 6.0;
constexpr double k1312 = 13.0 / 12.0;
constexpr double kTwelfth = 1.0 / 12.0;
constexpr double k24th = 1.0 / 24.0;
constexpr double k16th = 1.0 / 16.0;

int grid_for(long long work, int block) {
  long long b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 152LL * 64) b = 152LL * 64;
  return (int)b;
}

// ------------------------------------------------------------------------------------------------
// boundary maps
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int bc_source(int kind, int side, int a, int n, int h) {
  if (kind == FLUID_BC_PERIODIC) return side == 0 ? a + n : a - n;
  if (kind == FLUID_BC_ZERO_GRADIENT) return side == 0 ? h : h + n - 1;
  return side == 0 ? 2 * h - 1 - a : 2 * (h + n) - 1 - a;   // mirror image across the face
}

__device__ __forceinline__ void prim_of(const double* __restrict__ U, int c, int nc, const Phys& ph,
                                        double w[NW]) {
  const double r = U[c];
  const double mx = U[nc + c], my = U[2 * nc + c], mz = U[3 * nc + c], E = U[4 * nc + c];
  const double ir = 1.0 / r;
  const double u = mx * ir, v = my * ir, ww = mz * ir;
  const double p = ph.gm1 * (E - 0.5 * r * (u * u + v * v + ww * ww));
  w[0] = r; w[1] = u; w[2] = v; w[3] = ww; w[4] = p; w[5] = p * ir * ph.iR;
}

// wall map of axis a applied to primitives w (velocity mirrored; isothermal: T_g = 2 T_w - T,
// p_g = p; porous adds the transpiration velocity to the wall-normal component)
__device__ __forceinline__ void wall_map(double w[NW], int kind, double Tw, double vw, int a,
                                         const Phys& ph, unsigned* flags) {
  w[1] = -w[1]; w[2] = -w[2]; w[3] = -w[3];
  if (kind == FLUID_BC_ADIABATIC) return;
  const double Tg = 2.0 * Tw - w[5];
  if (!(Tg > 0.0)) atomicOr(flags, FLAG_GHOST_T);
  w[0] = w[4] / (ph.R * Tg);
  w[5] = Tg;
  if (kind == FLUID_BC_POROUS) w[1 + a] = 2.0 * vw + w[1 + a];
}

__device__ __forceinline__ void inflow_at(const double* __restrict__ prof, int a, const int c[3],
                                          const Geo& g, const Phys& ph, double w[NW]) {
  // tangential axes t1 < t2; profile laid out [5][p_t2][p_t1]
  const int t1 = (a == 0) ? 1 : 0;
  const int t2 = (a == 2) ? 1 : 2;
  const int plane = g.p[t1] * g.p[t2];
  const int o = c[t2] * g.p[t1] + c[t1];
  for (int v = 0; v < 5; ++v) w[v] = prof[v * plane + o];
  w[5] = w[4] / (w[0] * ph.R);
}

__global__ void k_prim_bc(const double* __restrict__ U, double* __restrict__ W,
                          float* __restrict__ W32, Geo g, Phys ph, BC bc, Ctl* ctl) {
  const int total = g.ncell;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < total;
       cell += gridDim.x * blockDim.x) {
    int own[3];
    own[0] = cell % g.p[0];
    const int r = cell / g.p[0];
    own[1] = r % g.p[1];
    own[2] = r / g.p[1];
    bool ghost[3];
    int side[3], src[3];
    bool any = false;
    for (int a = 0; a < 3; ++a) {
      ghost[a] = own[a] < g.h[a] || own[a] >= g.h[a] + g.n[a];
      side[a] = own[a] < g.h[a] ? 0 : 1;
      src[a] = ghost[a] ? bc_source(bc.kind[a][side[a]], side[a], own[a], g.n[a], g.h[a]) : own[a];
      any |= ghost[a];
    }
    double w[NW];
    if (!any) {
      prim_of(U, cell, g.ncell, ph, w);
    } else {
      // Sequential halo passes x -> y -> z, composed: the pass of axis a sees own indices on the
      // axes before it and source indices on the axes after it.
      bool have = false;
      for (int a = 0; a < 3; ++a) {
        if (!ghost[a]) continue;
        const int kind = bc.kind[a][side[a]];
        int c[3];
        for (int b = 0; b < 3; ++b) c[b] = b < a ? own[b] : src[b];
        if (kind == FLUID_BC_INFLOW) {
          inflow_at(bc.inflow[a][side[a]], a, c, g, ph, w);
          have = true;
          continue;
        }
        if (!have) {
          c[a] = src[a];
          prim_of(U, c[0] + c[1] * g.sy + c[2] * g.sz, g.ncell, ph, w);
          have = true;
        }
        if (kind == FLUID_BC_PERIODIC || kind == FLUID_BC_ZERO_GRADIENT) continue;
        double vw = 0.0;
        if (kind == FLUID_BC_POROUS) vw = bc.vw[c[bc.porous_t1]];
        wall_map(w, kind, bc.Tw[a][side[a]], vw, a, ph, &ctl->flags);
      }
    }
    for (int v = 0; v < NW; ++v) W[v * g.ncell + cell] = w[v];
    if (W32)
      for (int v = 0; v < NW; ++v) W32[v * g.ncell + cell] = (float)w[v];
  }
}

// ------------------------------------------------------------------------------------------------
// centre gradients: G[c*3+b] = d u_c / d x_b by ((f[-2] - f[+2]) + 8 (f[+1] - f[-1])) / 12 * mc,
// only where the cell is interior along b (the only places the face fluxes read it)
// ------------------------------------------------------------------------------------------------
__global__ void k_grad(const double* __restrict__ W, double* __restrict__ G, Geo g) {
  int lo[3], ext[3];
  for (int a = 0; a < 3; ++a) {
    const int m = a < g.ndim ? 2 : 0;
    lo[a] = g.h[a] - m;
    ext[a] = g.n[a] + 2 * m;
  }
  const int total = ext[0] * ext[1] * ext[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int c[3];
    c[0] = lo[0] + t % ext[0];
    const int r = t / ext[0];
    c[1] = lo[1] + r % ext[1];
    c[2] = lo[2] + r / ext[1];
    const int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    for (int b = 0; b < 3; ++b) {
      const bool inb = b < g.ndim && c[b] >= g.h[b] && c[b] < g.h[b] + g.n[b];
      const int s = b == 0 ? 1 : (b == 1 ? g.sy : g.sz);
      const double m = inb ? g.mc[b][c[b]] : 0.0;
      for (int comp = 0; comp < 3; ++comp) {
        double d = 0.0;
        if (inb) {
          const double* f = W + (1 + comp) * g.ncell + cell;
          d = ((f[-2 * s] - f[2 * s]) + 8.0 * (f[s] - f[-s])) * kTwelfth * m;
        }
        G[(comp * 3 + b) * g.ncell + cell] = d;
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// WENO5 (Jiang & Shu; Borges et al. Z variant): left-biased value at i+1/2 from q_{i-2..i+2}
// ------------------------------------------------------------------------------------------------
template <int SCHEME>
__device__ __forceinline__ double weno5(double qm2, double qm1, double q0, double qp1, double qp2,
                                        double eps) {
  // candidate values times 6
  const double C0 = 2.0 * qm2 - 7.0 * qm1 + 11.0 * q0;
  const double C1 = -qm1 + 5.0 * q0 + 2.0 * qp1;
  const double C2 = 2.0 * q0 + 5.0 * qp1 - qp2;
  double t = qm2 - 2.0 * qm1 + q0, s = qm2 - 4.0 * qm1 + 3.0 * q0;
  const double b0 = k1312 * t * t + 0.25 * s * s;
  t = qm1 - 2.0 * q0 + qp1; s = qm1 - qp1;
  const double b1 = k1312 * t * t + 0.25 * s * s;
  t = q0 - 2.0 * qp1 + qp2; s = 3.0 * q0 - 4.0 * qp1 + qp2;
  const double b2 = k1312 * t * t + 0.25 * s * s;
  // Weights scaled by a common positive factor so that one division remains.  With
  // e_k = beta_k + eps and Q_k = prod_{j != k} e_j:
  //   JS: d_k / e_k^2                  = d_k Q_k^2 / P^2,              P = e0 e1 e2
  //   Z : d_k (1 + (tau5 / e_k)^2)     = d_k (P^2 + tau5^2 Q_k^2) / P^2
  // The common 1/P^2 cancels in omega_k = alpha_k / sum alpha.  Since e_k >= eps the scaled
  // weights stay normal for eps = 1e-40 (P^2 >= 1e-240) and finite while beta_k < 1e50.
  const double e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps;
  const double Q0 = e1 * e2, Q1 = e0 * e2, Q2 = e0 * e1;
  double a0, a1, a2;
  if (SCHEME == FLUID_WENO_JS) {
    a0 = 0.1 * (Q0 * Q0); a1 = 0.6 * (Q1 * Q1); a2 = 0.3 * (Q2 * Q2);
  } else {
    const double tau = fabs(b0 - b2);
    const double P = e0 * Q0;
    const double PP = P * P, tt = tau * tau;
    a0 = 0.1 * (PP + tt * (Q0 * Q0));
    a1 = 0.6 * (PP + tt * (Q1 * Q1));
    a2 = 0.3 * (PP + tt * (Q2 * Q2));
  }
  return (a0 * C0 + a1 * C1 + a2 * C2) / (6.0 * (a0 + a1 + a2));
}

// ------------------------------------------------------------------------------------------------
// HLLC along axis D (Toro Ch. 10) with Einfeldt/Roe wave-speed bounds.  Branch order:
// S_L >= 0 -> F_L; S* >= 0 -> F*_L; S_R > 0 -> F*_R; else F_R.
// ------------------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void hllc(const double wl[5], const double wr[5], const Phys& ph,
                                     double F[5]) {
  const double rL = wl[0], pL = wl[4], rR = wr[0], pR = wr[4];
  const double unL = wl[1 + D], unR = wr[1 + D];
  const double q2L = wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3];
  const double q2R = wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3];
  const double EL = pL * ph.igm1 + 0.5 * rL * q2L;
  const double ER = pR * ph.igm1 + 0.5 * rR * q2R;
  // 1/sqrt(rho) gives both sqrt(rho) (Roe weights) and 1/rho
  const double qL = rsqrt(rL), qR = rsqrt(rR);
  const double sL = rL * qL, sR = rR * qR;
  const double irL = qL * qL, irR = qR * qR;
  const double cL = sqrt(ph.gamma * pL * irL), cR = sqrt(ph.gamma * pR * irR);
  const double isum = 1.0 / (sL + sR);
  const double ut0 = (sL * wl[1] + sR * wr[1]) * isum;
  const double ut1 = (sL * wl[2] + sR * wr[2]) * isum;
  const double ut2 = (sL * wl[3] + sR * wr[3]) * isum;
  const double HL = (EL + pL) * irL, HR = (ER + pR) * irR;
  const double Ht = (sL * HL + sR * HR) * isum;
  const double ct = sqrt(ph.gm1 * (Ht - 0.5 * (ut0 * ut0 + ut1 * ut1 + ut2 * ut2)));
  const double utn = D == 0 ? ut0 : (D == 1 ? ut1 : ut2);
  const double SL = fmin(unL - cL, utn - ct);
  const double SR = fmax(unR + cR, utn + ct);
  const double mL = rL * (SL - unL), mR = rR * (SR - unR);
  const double Ss = (pR - pL + unL * mL - unR * mR) / (mL - mR);

  const bool left = (SL >= 0.0) || (Ss >= 0.0);
  const bool star = left ? !(SL >= 0.0) : (SR > 0.0);
  const double r = left ? rL : rR;
  const double p = left ? pL : pR;
  const double E = left ? EL : ER;
  const double un = left ? unL : unR;
  const double S = left ? SL : SR;
  const double m = left ? mL : mR;
  const double u0 = left ? wl[1] : wr[1];
  const double u1 = left ? wl[2] : wr[2];
  const double u2 = left ? wl[3] : wr[3];
  // Euler flux of the selected side
  const double mn = r * un;
  F[0] = mn;
  F[1] = mn * u0;
  F[2] = mn * u1;
  F[3] = mn * u2;
  F[1 + D] += p;
  F[4] = un * (E + p);
  if (star) {
    // U*_K = m/(S - S*) [1, S* (normal), tangential u, E/rho + (S* - un)(S* + p/m)]
    const double q = 1.0 / (S - Ss);
    const double fac = m * q;
    const double ir = left ? irL : irR;
    const double dU0 = fac - r;
    double dU[3] = {fac * u0 - r * u0, fac * u1 - r * u1, fac * u2 - r * u2};
    dU[D] = fac * Ss - r * un;
    const double Es = fac * (E * ir) + (Ss - un) * (fac * Ss + p * q);
    F[0] += S * dU0;
    F[1] += S * dU[0];
    F[2] += S * dU[1];
    F[3] += S * dU[2];
    F[4] += S * (Es - E);
  }
}

// ------------------------------------------------------------------------------------------------
// face flux F^c - F^d at face a+1/2 along D; `cell` is the padded index of cell a, s its stride
// ------------------------------------------------------------------------------------------------
template <int D, int SCHEME, bool VISC>
__device__ __forceinline__ void face_flux(const double* __restrict__ W, const double* __restrict__ G,
                                          int cell, int s, int a, const Geo& g, const Phys& ph,
                                          double F[5]) {
  const int nc = g.ncell;
  double q[5][6];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int o = 0; o < 6; ++o) q[v][o] = __ldg(W + v * nc + cell + (o - 2) * s);
  double wl[5], wr[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    wl[v] = weno5<SCHEME>(q[v][0], q[v][1], q[v][2], q[v][3], q[v][4], ph.eps);
    wr[v] = weno5<SCHEME>(q[v][5], q[v][4], q[v][3], q[v][2], q[v][1], ph.eps);
  }
  hllc<D>(wl, wr, ph, F);
  if (!VISC) return;

  // cells a-1 .. a+2 are q[.][1..4]
  const double mfa = g.mf[D][a];
  double T[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) T[o] = __ldg(W + 5 * nc + cell + (o - 1) * s);
  auto interp = [](double fm1, double f0, double f1, double f2) {
    return (9.0 * (f0 + f1) - (fm1 + f2)) * k16th;
  };
  auto dn = [&](double fm1, double f0, double f1, double f2) {
    return ((fm1 - f2) + 27.0 * (f1 - f0)) * k24th * mfa;
  };
  double vf[3], Gf[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vf[c] = interp(q[1 + c][1], q[1 + c][2], q[1 + c][3], q[1 + c][4]);
    Gf[c][D] = dn(q[1 + c][1], q[1 + c][2], q[1 + c][3], q[1 + c][4]);
  }
  const double Tf = interp(T[0], T[1], T[2], T[3]);
  const double dT = dn(T[0], T[1], T[2], T[3]);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (b == D) continue;
    if (b < g.ndim) {
      const double* gd = G + (D * 3 + b) * nc + cell;   // d u_D / d x_b
      const double* gb = G + (b * 3 + b) * nc + cell;   // d u_b / d x_b
      Gf[D][b] = interp(__ldg(gd - s), __ldg(gd), __ldg(gd + s), __ldg(gd + 2 * s));
      Gf[b][b] = interp(__ldg(gb - s), __ldg(gb), __ldg(gb + s), __ldg(gb + 2 * s));
    } else {
      Gf[D][b] = 0.0;
      Gf[b][b] = 0.0;
    }
  }
  const double div = Gf[0][0] + Gf[1][1] + Gf[2][2];
  const double mu = viscosity(Tf, ph);
  const double lam = mu * ph.lam_fac;
  double tau[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (c == D) tau[c] = mu * (Gf[D][D] + Gf[D][D]) - (2.0 / 3.0) * mu * div;
    else tau[c] = mu * (Gf[c][D] + Gf[D][c]);
  }
  const double en = vf[0] * tau[0] + vf[1] * tau[1] + vf[2] * tau[2] + lam * dT;
  F[1] -= tau[0];
  F[2] -= tau[1];
  F[3] -= tau[2];
  F[4] -= en;
}

template <int D, int SCHEME, bool VISC>
__global__ void __launch_bounds__(128) k_face(const double* __restrict__ W,
                                              const double* __restrict__ G, double* __restrict__ R,
                                              Geo g, Phys ph, int accumulate, int seg) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const int n1 = g.n[A1], n2 = g.n[A2], nd = g.n[D];
  const int nseg = (nd + seg - 1) / seg;
  const long long total = (long long)n1 * n2 * nseg;
  const int s = D == 0 ? 1 : (D == 1 ? g.sy : g.sz);
  const int nc = g.ncell;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i1 = (int)(t % n1);
    const long long r = t / n1;
    const int i2 = (int)(r % n2);
    const int sg = (int)(r / n2);
    int c[3];
    c[A1] = i1 + g.h[A1];
    c[A2] = i2 + g.h[A2];
    const int a0 = g.h[D] + sg * seg;
    const int a1 = min(a0 + seg, g.h[D] + nd);
    c[D] = a0 - 1;
    int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    double Fp[5], F[5];
    face_flux<D, SCHEME, VISC>(W, G, cell, s, a0 - 1, g, ph, Fp);
    for (int a = a0; a < a1; ++a) {
      cell += s;
      face_flux<D, SCHEME, VISC>(W, G, cell, s, a, g, ph, F);
      const double id = g.idx[D][a];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double val = -(F[v] - Fp[v]) * id;
        double* dst = R + v * nc + cell;
        *dst = accumulate ? *dst + val : val;
        Fp[v] = F[v];
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// source, stage combination, dt
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int interior_cell(int t, const Geo& g) {
  const int i = t % g.n[0];
  const int r = t / g.n[0];
  const int j = r % g.n[1];
  const int k = r / g.n[1];
  return (i + g.h[0]) + (j + g.h[1]) * g.sy + (k + g.h[2]) * g.sz;
}

__global__ void k_source(double* __restrict__ R, const double* __restrict__ W, Geo g, Phys ph) {
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int c = interior_cell(t, g);
    const double u = W[nc + c], v = W[2 * nc + c], w = W[3 * nc + c];
    R[nc + c] += ph.f[0];
    R[2 * nc + c] += ph.f[1];
    R[3 * nc + c] += ph.f[2];
    R[4 * nc + c] += ph.f[0] * u + ph.f[1] * v + ph.f[2] * w;
  }
}

// stage 1: Ud = Un + dt r; stage 2: Ud = 3/4 Un + 1/4 (Us + dt r); stage 3: Ud = 1/3 Un + 2/3 (Us + dt r)
__global__ void k_stage(int stage, const double* Un, const double* Us, const double* __restrict__ R,
                        double* Ud, const double* __restrict__ W, Geo g, Phys ph, Ctl* ctl,
                        double t_end) {
  const double dt = ctl->dt;
  if (stage == 3 && blockIdx.x == 0 && threadIdx.x == 0 && dt > 0.0) {
    const double tn = ctl->t + dt;
    ctl->t = (t_end > 0.0 && !(tn < t_end)) ? t_end : tn;
  }
  if (stage == 3 && !(dt > 0.0)) return;
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  bool bad = false;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int c = interior_cell(t, g);
    double r[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v] = R[v * nc + c];
    if (ph.has_force) {
      const double u = W[nc + c], v = W[2 * nc + c], w = W[3 * nc + c];
      r[1] += ph.f[0];
      r[2] += ph.f[1];
      r[3] += ph.f[2];
      r[4] += ph.f[0] * u + ph.f[1] * v + ph.f[2] * w;
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double un = Un[v * nc + c];
      double out;
      if (stage == 1) {
        out = un + dt * r[v];
      } else {
        const double us = Us[v * nc + c];
        out = stage == 2 ? 0.75 * un + 0.25 * (us + dt * r[v])
                         : (1.0 / 3.0) * un + (2.0 / 3.0) * (us + dt * r[v]);
      }
      bad |= !finite_bits(out);
      Ud[v * nc + c] = out;
    }
  }
  if (bad) atomicOr(&ctl->flags, FLAG_NONFINITE);
}

constexpr int kDtBlock = 256;

__global__ void __launch_bounds__(kDtBlock) k_dt_partial(const double* __restrict__ W, Geo g, Phys ph,
                                                         double* __restrict__ partial) {
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  double best = __longlong_as_double(0x7ff0000000000000LL);   // +inf
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int i = t % g.n[0];
    const int r = t / g.n[0];
    const int j = r % g.n[1];
    const int k = r / g.n[1];
    const int ci[3] = {i + g.h[0], j + g.h[1], k + g.h[2]};
    const int c = ci[0] + ci[1] * g.sy + ci[2] * g.sz;
    const double rho = W[c], p = W[4 * nc + c];
    const double cs = sqrt(ph.gamma * p / rho);
    double nu = 0.0;
    if (ph.visc != FLUID_VISC_NONE) nu = viscosity(W[5 * nc + c], ph) / rho;
    for (int d = 0; d < g.ndim; ++d) {
      const double dx = g.dx[d][ci[d]];
      best = fmin(best, dx / (fabs(W[(1 + d) * nc + c]) + cs));
      if (ph.visc != FLUID_VISC_NONE) best = fmin(best, dx * dx / (ph.dt_visc_k * nu));
    }
  }
  __shared__ double sm[kDtBlock / 32];
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < kDtBlock / 32 ? sm[threadIdx.x] : __longlong_as_double(0x7ff0000000000000LL);
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_down_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) partial[blockIdx.x] = best;
  }
}

// dt = cfl * min(partials) (or dt_fixed); clip_to_ctl: clip so that t does not pass t_end and store
// in ctl->dt; otherwise write *dt_out.
__global__ void __launch_bounds__(kDtBlock) k_dt_final(const double* __restrict__ partial, int nparts,
                                                       Phys ph, Ctl* ctl, double* dt_out, int clip,
                                                       double t_end) {
  double best = __longlong_as_double(0x7ff0000000000000LL);
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) best = fmin(best, partial[i]);
  __shared__ double sm[kDtBlock / 32];
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kDtBlock / 32; ++i) best = fmin(best, sm[i]);
    sm[0] = best;
    double dt = ph.dt_fixed > 0.0 ? ph.dt_fixed : ph.cfl * sm[0];
    if (!clip) {
      *dt_out = dt;
      return;
    }
    if (t_end > 0.0) {
      if (ctl->t >= t_end) dt = 0.0;
      else if (ctl->t + dt > t_end) dt = t_end - ctl->t;
    }
    ctl->dt = dt;
  }
}

__global__ void k_prim_to_cons(const double* W, double* U, int nc, Phys ph) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const double r = W[c], u = W[nc + c], v = W[2 * nc + c], w = W[3 * nc + c], p = W[4 * nc + c];
    const double E = p * ph.igm1 + 0.5 * r * (u * u + v * v + w * w);
    U[c] = r;
    U[nc + c] = r * u;
    U[2 * nc + c] = r * v;
    U[3 * nc + c] = r * w;
    U[4 * nc + c] = E;
  }
}

__global__ void k_wall_velocity(const double* __restrict__ phi, double* __restrict__ vw,
                                const double* __restrict__ xc, int p, int h, int begin, int count,
                                double amp, double two_pi_kappa) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < p; a += gridDim.x * blockDim.x) {
    const int i = a - h - begin;
    vw[a] = (i >= 0 && i < count) ? amp * phi[i] * sin(two_pi_kappa * xc[a]) : 0.0;
  }
}

template <int D, int SCHEME, bool VISC>
cudaError_t launch_face_t(const double* W, const double* G, double* R, const Geo& g,
                          const Phys& ph, int accumulate, int block, int seg, cudaStream_t st) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const long long lines = (long long)g.n[A1] * g.n[A2];
  if (block <= 0) block = 128;
  if (seg <= 0) {
    // longest segment (fewest redundant faces) that still gives >= 4 blocks of 128 per SM
    seg = 64;
    while (seg > 8 && lines * ((g.n[D] + seg - 1) / seg) < 152LL * 4 * 128) seg >>= 1;
  }
  const long long total = lines * ((g.n[D] + seg - 1) / seg);
  k_face<D, SCHEME, VISC><<<grid_for(total, block), block, 0, st>>>(W, G, R, g, ph, accumulate, seg);
  return cudaGetLastError();
}

template <int SCHEME, bool VISC>
cudaError_t launch_face_sv(int D, const double* W, const double* G, double* R, const Geo& g,
                           const Phys& ph, int accumulate, int block, int seg, cudaStream_t st) {
  if (D == 0) return launch_face_t<0, SCHEME, VISC>(W, G, R, g, ph, accumulate, block, seg, st);
  if (D == 1) return launch_face_t<1, SCHEME, VISC>(W, G, R, g, ph, accumulate, block, seg, st);
  return launch_face_t<2, SCHEME, VISC>(W, G, R, g, ph, accumulate, block, seg, st);
}

}  // namespace

cudaError_t launch_prim_bc(const double* U, double* W, float* W32, const Geo& g, const Phys& ph,
                           const BC& bc, Ctl* ctl, cudaStream_t st) {
  k_prim_bc<<<grid_for(g.ncell, 256), 256, 0, st>>>(U, W, W32, g, ph, bc, ctl);
  return cudaGetLastError();
}

cudaError_t launch_grad(const double* W, double* G, const Geo& g, cudaStream_t st) {
  long long total = 1;
  for (int a = 0; a < 3; ++a) total *= g.n[a] + (a < g.ndim ? 4 : 0);
  k_grad<<<grid_for(total, 256), 256, 0, st>>>(W, G, g);
  return cudaGetLastError();
}

cudaError_t launch_face(int D, const double* W, const double* G, double* R, const Geo& g,
                        const Phys& ph, int accumulate, int block, int seg, cudaStream_t st) {
  const bool visc = ph.visc != FLUID_VISC_NONE;
  if (ph.weno == FLUID_WENO_JS)
    return visc ? launch_face_sv<FLUID_WENO_JS, true>(D, W, G, R, g, ph, accumulate, block, seg, st)
                : launch_face_sv<FLUID_WENO_JS, false>(D, W, G, R, g, ph, accumulate, block, seg, st);
  return visc ? launch_face_sv<FLUID_WENO_Z, true>(D, W, G, R, g, ph, accumulate, block, seg, st)
              : launch_face_sv<FLUID_WENO_Z, false>(D, W, G, R, g, ph, accumulate, block, seg, st);
}

cudaError_t launch_source(double* R, const double* W, const Geo& g, const Phys& ph, cudaStream_t st) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  k_source<<<grid_for(total, 256), 256, 0, st>>>(R, W, g, ph);
  return cudaGetLastError();
}

cudaError_t launch_stage(int stage, const double* Un, const double* Us, const double* R, double* Ud,
                         const double* W, const Geo& g, const Phys& ph, Ctl* ctl, double t_end,
                         cudaStream_t st) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  k_stage<<<grid_for(total, 256), 256, 0, st>>>(stage, Un, Us, R, Ud, W, g, ph, ctl, t_end);
  return cudaGetLastError();
}

int dt_partial_count(const Geo& g) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  long long b = (total + kDtBlock - 1) / kDtBlock;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_dt_partial(const double* W, const Geo& g, const Phys& ph, double* partial,
                              int nparts, cudaStream_t st) {
  k_dt_partial<<<nparts, kDtBlock, 0, st>>>(W, g, ph, partial);
  return cudaGetLastError();
}

cudaError_t launch_dt_final(const double* partial, int nparts, const Phys& ph, Ctl* ctl,
                            double* dt_out, int clip_to_ctl, double t_end, cudaStream_t st) {
  k_dt_final<<<1, kDtBlock, 0, st>>>(partial, ph.dt_fixed > 0.0 ? 0 : nparts, ph, ctl, dt_out,
                                     clip_to_ctl, t_end);
  return cudaGetLastError();
}

cudaError_t launch_prim_to_cons(const double* W, double* U, int ncell, const Phys& ph,
                                cudaStream_t st) {
  k_prim_to_cons<<<grid_for(ncell, 256), 256, 0, st>>>(W, U, ncell, ph);
  return cudaGetLastError();
}

cudaError_t launch_wall_velocity(const double* phi, double* vw, const double* xc, int p, int h,
                                 int begin, int count, double amp, double two_pi_kappa,
                                 cudaStream_t st) {
  k_wall_velocity<<<grid_for(p, 128), 128, 0, st>>>(phi, vw, xc, p, h, begin, count, amp,
                                                    two_pi_kappa);
  return cudaGetLastError();
}

}  // namespace fl
