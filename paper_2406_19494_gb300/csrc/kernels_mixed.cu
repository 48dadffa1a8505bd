// Mixed-precision face kernels: WENO5 weights and reconstruction, HLLC wave speeds and star
// correction, and the dissipative stencils in FP32; the state, the cell-centre convective flux,
// the face-flux assembly and the flux-difference accumulation in FP64.
//
// Why a delta form.  At low Mach number the pressure (and total enthalpy) is large and nearly
// uniform, so fluxes are large and their differences across a cell small: a flux rounded to FP32
// carries an absolute error ~6e-8 |F| that the divergence divides by dx.  Here every FP32 quantity
// is either a coefficient (used only as a factor) or a small increment that FP32 represents to
// ~6e-8 of its own size:
//   * cell differences D_j = q_{j+1} - q_j of the primitives come from the exact FP32 split
//     q = hi + lo written by the primitive kernel: (hi_{j+1} - hi_j) + (lo_{j+1} - lo_j), each
//     FP32 subtraction rounding relative to its own result, so D_j is within ~1 ulp (FP32) of the
//     FP64 difference, up to 2^-48 |q| from the split;
//   * WENO5 works on offsets delta_k = q_{a+k} - q_a built from the D's (the smoothness
//     indicators and the weights do not depend on the offset, the candidates are affine);
//   * the face flux is F_{a+1/2} = F(q_a) [FP64, from the primitives and H = E + p] + X [FP32],
//     where X is the change of the Euler
//     flux from the cell state q_a to the upwind face state, written as a polynomial in the
//     offsets, plus the HLLC star correction S_K (U*_K - U_K), written through the jumps of the
//     reconstructed states (S* - u_K from the pressure and velocity jumps), minus the
//     dissipative flux;
//   * R += -(F_{a+1/2} - F_{a-1/2}) / dx in FP64, so the face fluxes telescope exactly as in the
//     FP64 path (each face value is computed once and shared by its two cells).
#include <cuda_runtime.h>

#include "flux_math.cuh"
#include "fluid_internal.cuh"

namespace fl {

namespace {

constexpr float k1312f = 13.0f / 12.0f;
constexpr float kZepsF = 1e-20f;      // WENO5-Z epsilon in FP32 (a normal float)
constexpr float kZclampF = 1e18f;     // bound of tau5 / (beta + eps): keeps its square finite

// FP32 reciprocal, square root and reciprocal square root from the hardware approximations
// (PTX rcp.approx / sqrt.approx / rsqrt.approx, each within a few ulp; denormal inputs flush
// to zero). The FP32 increments need ~1e-7 relative accuracy, so the IEEE-rounded division and
// square root, with their refinement steps and slow-path checks, are not needed here.
__device__ __forceinline__ float rcpf(float y) {
  float r; asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y)); return r;
}
__device__ __forceinline__ float sqrtf_a(float y) {
  float r; asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y)); return r;
}
__device__ __forceinline__ float rsqrtf_a(float y) {
  float r; asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y)); return r;
}

// ---- bulk-copy staging: cp.async.bulk (the TMA unit's untiled copy) completing on an mbarrier ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also raises the phase's expected transaction count by `bytes`
__device__ __forceinline__ void mbar_arrive_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte aligned), counted on bar
__device__ __forceinline__ void bulk_to_smem(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}
// Bounded wait for the phase of the given parity: non-blocking tests with a short sleep between
// them, 2^17 of them at most (of the order of 10 ms); false if the phase did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  for (int it = 0; it < (1 << 17); ++it) {
    if (mbar_test(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

int grid_for(long long work, int block) {
  long long b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 152LL * 64) b = 152LL * 64;
  return (int)b;
}

// FP32 copies of the physical constants the increments use (no per-face conversions)
struct PhysF {
  float gamma, gm1, igm1, gg;            // gg = gamma / (gamma - 1)
  float mu_ref, iT_ref, visc_exp, TS, S; // TS = T_ref + S (Sutherland)
  float lam_fac, eps, dt_visc_k;
  int visc;
};

__host__ __device__ inline PhysF phys_f(const Phys& ph) {
  PhysF f;
  f.gamma = (float)ph.gamma; f.gm1 = (float)ph.gm1; f.igm1 = (float)ph.igm1;
  f.gg = (float)(ph.gamma * ph.igm1);
  f.mu_ref = (float)ph.mu_ref; f.iT_ref = (float)ph.iT_ref; f.visc_exp = (float)ph.visc_exp;
  f.TS = (float)(ph.T_ref + ph.suth_S); f.S = (float)ph.suth_S;
  f.lam_fac = (float)ph.lam_fac; f.eps = (float)ph.eps; f.dt_visc_k = (float)ph.dt_visc_k;
  f.visc = ph.visc;
  return f;
}

// inputs of the face kernels: FP64 primitives with the H = E + p row, their FP32 split, gradients
struct MixedIn {
  const double* W;     // [NW + 1][ncell]
  const float* hi;     // [NW][ncell]
  const float* lo;     // [NW][ncell]
  const float* G32;    // [NG][ncell] (viscous only)
};

// WENO5 value at i+1/2 relative to an arbitrary offset, from offsets of q_{i-2..i+2}
template <int SCHEME>
__device__ __forceinline__ float weno5f(float qm2, float qm1, float q0, float qp1, float qp2, float eps) {
  const float p0 = 2.0f * qm2 - 7.0f * qm1 + 11.0f * q0;
  const float p1 = -qm1 + 5.0f * q0 + 2.0f * qp1;
  const float p2 = 2.0f * q0 + 5.0f * qp1 - qp2;
  float t = qm2 - 2.0f * qm1 + q0, s = qm2 - 4.0f * qm1 + 3.0f * q0;
  const float b0 = k1312f * t * t + 0.25f * s * s;
  t = qm1 - 2.0f * q0 + qp1; s = qm1 - qp1;
  const float b1 = k1312f * t * t + 0.25f * s * s;
  t = q0 - 2.0f * qp1 + qp2; s = 3.0f * q0 - 4.0f * qp1 + qp2;
  const float b2 = k1312f * t * t + 0.25f * s * s;
  float a0, a1, a2;
  if (SCHEME == FLUID_WENO_JS) {
    const float r0 = rcpf(eps + b0), r1 = rcpf(eps + b1), r2 = rcpf(eps + b2);
    a0 = 0.1f * r0 * r0; a1 = 0.6f * r1 * r1; a2 = 0.3f * r2 * r2;
  } else {
    const float tau = fabsf(b0 - b2);
    const float r0 = fminf(tau * rcpf(b0 + kZepsF), kZclampF);
    const float r1 = fminf(tau * rcpf(b1 + kZepsF), kZclampF);
    const float r2 = fminf(tau * rcpf(b2 + kZepsF), kZclampF);
    a0 = 0.1f * (1.0f + r0 * r0); a1 = 0.6f * (1.0f + r1 * r1); a2 = 0.3f * (1.0f + r2 * r2);
  }
  return (a0 * p0 + a1 * p1 + a2 * p2) * rcpf(6.0f * (a0 + a1 + a2));
}

__device__ __forceinline__ float viscosity_f(float T, const PhysF& pf) {
  if (pf.visc == FLUID_VISC_CONSTANT) return pf.mu_ref;
  const float r = T * pf.iT_ref;
  if (pf.visc == FLUID_VISC_POWER) return pf.mu_ref * __powf(r, pf.visc_exp);
  return pf.mu_ref * (r * sqrtf_a(r)) * pf.TS * rcpf(T + pf.S);
}

// X: change of the face flux relative to F(q_a), in FP32 (see the file comment).
//   b        FP32 cell state q_a (rho, u, v, w, p)
//   dL, dR   offsets of the reconstructed left and right face states from q_a
template <int D>
__device__ __forceinline__ void hllc_delta(const float b[5], const float dL[5], const float dR[5],
                                           const PhysF& pf, float X[5]) {
  const float g = pf.gamma, gm1 = pf.gm1, igm1 = pf.igm1;
  float wl[5], wr[5], J[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    wl[v] = b[v] + dL[v];
    wr[v] = b[v] + dR[v];
    J[v] = dR[v] - dL[v];                         // jumps, accurate to FP32 relative to themselves
  }
  const float rL = wl[0], pL = wl[4], rR = wr[0], pR = wr[4];
  const float unL = wl[1 + D], unR = wr[1 + D];
  const float q2L = wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3];
  const float q2R = wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3];
  const float EL = pL * igm1 + 0.5f * rL * q2L, ER = pR * igm1 + 0.5f * rR * q2R;
  const float isL = rsqrtf_a(rL), isR = rsqrtf_a(rR);        // 1/sqrt(rho)
  const float irL = isL * isL, irR = isR * isR;               // 1/rho
  const float cL = sqrtf_a(g * pL * irL), cR = sqrtf_a(g * pR * irR);
  const float sL = rL * isL, sR = rR * isR;                   // sqrt(rho)
  const float is = rcpf(sL + sR);
  const float ut0 = (sL * wl[1] + sR * wr[1]) * is;
  const float ut1 = (sL * wl[2] + sR * wr[2]) * is;
  const float ut2 = (sL * wl[3] + sR * wr[3]) * is;
  const float Ht = ((EL + pL) * isL + (ER + pR) * isR) * is;   // sqrt(rho) (E+p)/rho
  const float ct = sqrtf_a(gm1 * (Ht - 0.5f * (ut0 * ut0 + ut1 * ut1 + ut2 * ut2)));
  const float utn = D == 0 ? ut0 : (D == 1 ? ut1 : ut2);
  const float SL = fminf(unL - cL, utn - ct);
  const float SR = fmaxf(unR + cR, utn + ct);
  const float mL = rL * (SL - unL), mR = rR * (SR - unR);
  const float iden = rcpf(mL - mR);
  // S* - u_L and S* - u_R from the jumps: (dp - m_{R|L} du_n) / (m_L - m_R)
  const float sigL = (J[4] - mR * J[1 + D]) * iden;
  const float sigR = (J[4] - mL * J[1 + D]) * iden;
  const float Ss = unL + sigL;

  const bool left = (SL >= 0.0f) || (Ss >= 0.0f);
  const bool star = left ? !(SL >= 0.0f) : (SR > 0.0f);
  // the upwind side's offsets and state, selected value by value so that both arrays stay
  // in registers
  float d[5], w[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) { d[v] = left ? dL[v] : dR[v]; w[v] = left ? wl[v] : wr[v]; }

  // Euler-flux change from q_a to the face state K = b + d
  const float un = b[1 + D], unK = w[1 + D];
  const float mn = b[0] * un;
  const float dm = b[0] * d[1 + D] + d[0] * unK;          // rho' u_n' - rho u_n
  X[0] = dm;
#pragma unroll
  for (int c = 0; c < 3; ++c) X[1 + c] = dm * w[1 + c] + mn * d[1 + c];
  X[1 + D] += d[4];
  const float q2b = b[1] * b[1] + b[2] * b[2] + b[3] * b[3];
  const float dq2 = d[1] * (2.0f * b[1] + d[1]) + d[2] * (2.0f * b[2] + d[2]) + d[3] * (2.0f * b[3] + d[3]);
  const float gg = pf.gg;
  const float Hv = gg * b[4] + 0.5f * b[0] * q2b;         // E + p of q_a
  const float dHv = gg * d[4] + 0.5f * (d[0] * (q2b + dq2) + b[0] * dq2);
  X[4] = d[1 + D] * (Hv + dHv) + un * dHv;

  if (star) {
    // S_K (U*_K - U_K) with theta = (S* - u_K)/(S_K - S*), chi = 1 + theta
    const float S = left ? SL : SR;
    const float sig = left ? sigL : sigR;
    const float rK = w[0], pK = w[4];
    const float EK = left ? EL : ER;
    const float theta = sig * rcpf(S - Ss);
    const float chi = 1.0f + theta;
    float dU[5];
    dU[0] = rK * theta;
#pragma unroll
    for (int c = 0; c < 3; ++c) dU[1 + c] = rK * theta * w[1 + c];
    dU[1 + D] = rK * (theta * unK + chi * sig);
    dU[4] = theta * EK + chi * sig * (rK * Ss + pK * rcpf(S - unK));
#pragma unroll
    for (int v = 0; v < 5; ++v) X[v] += S * dU[v];
  }
}

// D-window entry: difference of one primitive between consecutive cells from its (hi, lo) split
__device__ __forceinline__ float diff32(const float* __restrict__ hi, const float* __restrict__ lo,
                                        int cell, int s) {
  return (__ldg(hi + cell + s) - __ldg(hi + cell)) + (__ldg(lo + cell + s) - __ldg(lo + cell));
}

// Face flux F_{a+1/2} (FP64) along D.  `cell` is cell a; Dw[v][k] holds D_{a-2+k}, k = 0..4.
template <int D, int SCHEME, bool VISC>
__device__ __forceinline__ void face_flux_mixed(const MixedIn& in, int cell, int s, int a,
                                                const float Dw[6][5], const Geo& g, const PhysF& pf,
                                                double F[5]) {
  const int nc = g.ncell;
  const float eps = pf.eps;
  float b[5], dL[5], dR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    b[v] = __ldg(in.hi + v * nc + cell);
    // offsets from q_a of cells a-2 .. a+3
    const float om1 = -Dw[v][1], om2 = -(Dw[v][0] + Dw[v][1]);
    const float op1 = Dw[v][2], op2 = Dw[v][2] + Dw[v][3], op3 = op2 + Dw[v][4];
    dL[v] = weno5f<SCHEME>(om2, om1, 0.0f, op1, op2, eps);
    dR[v] = weno5f<SCHEME>(op3, op2, op1, 0.0f, om1, eps);
  }
  float X[5];
  hllc_delta<D>(b, dL, dR, pf, X);

  if (VISC) {
    // u, v, w, T at cells a-1..a+2 through the D window (entries 1, 2, 3 = D_{a-1}, D_a, D_{a+1})
    const float mfa = __ldg(g.mf32[D] + a);
    float vf[3], Gf[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float d0 = Dw[1 + c][1], d1 = Dw[1 + c][2], d2 = Dw[1 + c][3];
      vf[c] = b[1 + c] + (8.0f * d1 + d0 - d2) * (1.0f / 16.0f);
      Gf[c][D] = (26.0f * d1 - d0 - d2) * (1.0f / 24.0f) * mfa;
    }
    const float Tb = __ldg(in.hi + 5 * nc + cell);
    const float Tf = Tb + (8.0f * Dw[5][2] + Dw[5][1] - Dw[5][3]) * (1.0f / 16.0f);
    const float dT = (26.0f * Dw[5][2] - Dw[5][1] - Dw[5][3]) * (1.0f / 24.0f) * mfa;
    auto interp = [](float fm1, float f0, float f1, float f2) {
      return (9.0f * (f0 + f1) - (fm1 + f2)) * (1.0f / 16.0f);
    };
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
      if (bb == D) continue;
      if (bb < g.ndim) {
        const float* gd = in.G32 + (D * 3 + bb) * nc + cell;
        const float* gb = in.G32 + (bb * 3 + bb) * nc + cell;
        Gf[D][bb] = interp(__ldg(gd - s), __ldg(gd), __ldg(gd + s), __ldg(gd + 2 * s));
        Gf[bb][bb] = interp(__ldg(gb - s), __ldg(gb), __ldg(gb + s), __ldg(gb + 2 * s));
      } else {
        Gf[D][bb] = 0.0f;
        Gf[bb][bb] = 0.0f;
      }
    }
    const float div = Gf[0][0] + Gf[1][1] + Gf[2][2];
    const float mu = viscosity_f(Tf, pf);
    const float lam = mu * pf.lam_fac;
    float tau[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c == D) tau[c] = mu * (Gf[D][D] + Gf[D][D]) - (2.0f / 3.0f) * mu * div;
      else tau[c] = mu * (Gf[c][D] + Gf[D][c]);
    }
    X[1] -= tau[0];
    X[2] -= tau[1];
    X[3] -= tau[2];
    X[4] -= vf[0] * tau[0] + vf[1] * tau[1] + vf[2] * tau[2] + lam * dT;
  }

  // FP64 cell-centre Euler flux of q_a plus the FP32 change (widened on the integer pipe)
  const double* W = in.W;
  const double r = W[cell], u0 = W[nc + cell], u1 = W[2 * nc + cell], u2 = W[3 * nc + cell];
  const double p = W[4 * nc + cell], H = W[NW * nc + cell];
  const double un = D == 0 ? u0 : (D == 1 ? u1 : u2);
  const double mn = r * un;
  F[0] = mn + fl_widen(X[0]);
  F[1] = fma(mn, u0, fl_widen(X[1]));
  F[2] = fma(mn, u1, fl_widen(X[2]));
  F[3] = fma(mn, u2, fl_widen(X[3]));
  F[1 + D] += p;
  F[4] = fma(un, H, fl_widen(X[4]));
}

// R_v (+)= -(F_v - Fp_v) / dx in FP64
__device__ __forceinline__ void divergence(double* __restrict__ R, int nc, int cell, double id,
                                           const double F[5], const double Fp[5], int accumulate) {
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double dF = F[v] - Fp[v];
    double* dst = R + v * nc + cell;
    *dst = accumulate ? fma(-id, dF, *dst) : -id * dF;
  }
}

// The stage of one interior cell once its right-hand side is complete: R_v = its value from the
// other axes' kernels minus this axis's flux difference (the FP64 accumulation of divergence()),
// then the arithmetic of k_stage_prim -- body force, the RK3 combination into Ud, the primitives of
// Ud, their split and H = E + p -- into the second buffer pair.  Wold: the current primitives (the
// body-force velocities of the stage's input state).
__device__ __forceinline__ void stage_cell(const StageOut& so, const double* __restrict__ R,
                                           const double* __restrict__ Wold, int nc, int cell, double id,
                                           const double F[5], const double Fp[5], double dt, bool hold,
                                           const Phys& ph, bool& bad) {
  double u[5];
  if (hold) {
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = so.Un[v * nc + cell];
  } else {
    double r[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v] = fma(-id, F[v] - Fp[v], R[v * nc + cell]);
    if (ph.has_force) {
      const double vx = Wold[nc + cell], vy = Wold[2 * nc + cell], vz = Wold[3 * nc + cell];
      r[1] += ph.f[0];
      r[2] += ph.f[1];
      r[3] += ph.f[2];
      r[4] += fma(ph.f[0], vx, fma(ph.f[1], vy, ph.f[2] * vz));
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double un = so.Un[v * nc + cell];
      double out;
      if (so.stage == 1) {
        out = fma(dt, r[v], un);
      } else {
        const double us = so.Us[v * nc + cell];
        out = so.stage == 2 ? fma(0.75, un, 0.25 * fma(dt, r[v], us))
                            : fma(1.0 / 3.0, un, (2.0 / 3.0) * fma(dt, r[v], us));
      }
      bad |= !finite_bits(out);
      so.Ud[v * nc + cell] = out;
      u[v] = out;
    }
  }
  if (!so.prims) return;
  double w[NW];
  prim_from_cons(u, ph, w);
#pragma unroll
  for (int v = 0; v < NW; ++v) {
    so.W[v * nc + cell] = w[v];
    split_hi_lo(w[v], so.W32[v * nc + cell], so.W32[(NW + v) * nc + cell]);
  }
  so.W[NW * nc + cell] = u[4] + w[4];
}

template <int D, int SCHEME, bool VISC>
__global__ void __launch_bounds__(128) k_face_mixed(MixedIn in, double* __restrict__ R, Geo g,
                                                    PhysF pf, int accumulate, int seg) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  constexpr int NVW = VISC ? 6 : 5;          // windowed primitives (T only for the heat flux)
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
    int cell = c[0] + c[1] * g.sy + c[2] * g.sz;   // cell a = a0 - 1
    // window D_{a-2 .. a+2} for the first face a0 - 1/2
    float Dw[6][5];
#pragma unroll
    for (int v = 0; v < NVW; ++v)
#pragma unroll
      for (int k = 0; k < 5; ++k) Dw[v][k] = diff32(in.hi + v * nc, in.lo + v * nc, cell + (k - 2) * s, s);
    double Fp[5], F[5];
    face_flux_mixed<D, SCHEME, VISC>(in, cell, s, a0 - 1, Dw, g, pf, Fp);
    for (int a = a0; a < a1; ++a) {
      cell += s;
#pragma unroll
      for (int v = 0; v < NVW; ++v) {
#pragma unroll
        for (int k = 0; k < 4; ++k) Dw[v][k] = Dw[v][k + 1];
        Dw[v][4] = diff32(in.hi + v * nc, in.lo + v * nc, cell + 2 * s, s);
      }
      face_flux_mixed<D, SCHEME, VISC>(in, cell, s, a, Dw, g, pf, F);
      divergence(R, nc, cell, g.idx[D][a], F, Fp, accumulate);
#pragma unroll
      for (int v = 0; v < 5; ++v) Fp[v] = F[v];
    }
  }
}

// x-direction variant: lanes map to consecutive faces of one grid row so that every global load is
// coalesced.  A warp covers 31 cells (32 faces) of a row; the cell differences D_j of the tile
// (36 per primitive) are formed once in shared memory, each lane builds its face from that window,
// and the flux difference takes the neighbouring face's flux from shared memory.
constexpr int kXCells = 31;
constexpr int kXRows = 4;

template <int SCHEME, bool VISC>
__device__ __forceinline__ void k_face_mixed_x_body(MixedIn in, double* __restrict__ R,
                                                              Geo g, PhysF pf, int accumulate,
    uint3 bid, uint3 gdim) {
  constexpr int NVW = VISC ? 6 : 5;
  constexpr int ND = kXCells + 5;               // D_j for j in [x0-3, x0+kXCells+1]
  __shared__ float sD[kXRows][6][ND];
  __shared__ double sF[kXRows][5][kXCells + 1];
  const int lane = threadIdx.x, row = threadIdx.y;
  const int n0 = g.n[0], h0 = g.h[0];
  const int line = bid.y * kXRows + row;
  const bool live = line < g.n[1] * g.n[2];
  const int j1 = live ? line % g.n[1] : 0, j2 = live ? line / g.n[1] : 0;
  const int x0 = h0 + bid.x * kXCells;      // first interior cell of the tile (padded index)
  const int nc = g.ncell;
  const int rowbase = (j1 + g.h[1]) * g.sy + (j2 + g.h[2]) * g.sz;
  const int xend = h0 + n0;                      // one past the last interior cell
  if (live) {
    for (int k = lane; k < ND; k += 32) {
      const int j = x0 - 3 + k;
      const bool ok = j + 1 <= xend + 2;         // W index j + 1 stays inside the padded row
#pragma unroll
      for (int v = 0; v < NVW; ++v)
        sD[row][v][k] = ok ? diff32(in.hi + v * nc, in.lo + v * nc, rowbase + j, 1) : 0.0f;
    }
  }
  // each warp reads only the shared rows it wrote: a warp barrier suffices
  __syncwarp();
  const int a = x0 - 1 + lane;                   // this lane's face is a + 1/2
  if (live && a < xend) {
    float Dw[6][5];
#pragma unroll
    for (int v = 0; v < NVW; ++v)
#pragma unroll
      for (int k = 0; k < 5; ++k) Dw[v][k] = sD[row][v][lane + k];
    double F[5];
    face_flux_mixed<0, SCHEME, VISC>(in, rowbase + a, 1, a, Dw, g, pf, F);
#pragma unroll
    for (int v = 0; v < 5; ++v) sF[row][v][lane] = F[v];
  }
  __syncwarp();
  const int cx = x0 + lane;                      // cell of the divergence
  if (live && lane < kXCells && cx < xend) {
    double F[5], Fp[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) { F[v] = sF[row][v][lane + 1]; Fp[v] = sF[row][v][lane]; }
    divergence(R, nc, rowbase + cx, g.idx[0][cx], F, Fp, accumulate);
  }
}

template <int SCHEME, bool VISC>
__global__ void __launch_bounds__(32 * kXRows) k_face_mixed_x(MixedIn in, double* __restrict__ R,
                                                              Geo g, PhysF pf, int accumulate) {
  k_face_mixed_x_body<SCHEME, VISC>(in, R, g, pf, accumulate, blockIdx, gridDim);
}

// y / z variant: lanes map to 32 consecutive x columns (coalesced loads); a block of NWARP warps
// covers FPW NWARP - 1 cells along the face axis D (FPW NWARP faces) of those columns at one index
// of the remaining axis.  The cell differences along D are staged in shared memory; warp w computes
// the FPW consecutive faces FPW w .. FPW w + FPW - 1, keeps the previous face flux in registers for
// the divergence of the cells between them and takes the flux of face FPW (w + 1) from the next
// warp through shared memory.  Registers are capped at 64 so that 32 / NWARP blocks (32 warps)
// fit an SM.
template <int NWARP, int FPW>
constexpr size_t t_smem() {
  return sizeof(float) * 6 * (FPW * NWARP + 4) * 32 + sizeof(double) * NWARP * 5 * 32;
}

// Bulk-staged tiles: the (hi, lo) rows a tile's cell differences need, staged into shared memory
// by cp.async.bulk.  Per row 36 floats: the 32 columns of the tile from the 16-byte boundary at or
// below the first, so that both addresses of the copy are aligned (the rows' own alignment varies
// with the row); the W32 buffers carry 64 floats of slack past their end for the last rows' tails.
constexpr int kBulkRow = 36;

template <int NWARP, int FPW, int NVW>
constexpr size_t t_smem_bulk() {
  return sizeof(float) * 2 * NVW * (FPW * NWARP + 5) * kBulkRow + t_smem<NWARP, FPW>();
}

template <int D, int SCHEME, bool VISC, int NWARP, int FPW, bool STAGE = false, bool BULK = false>
__device__ __forceinline__ void k_face_mixed_t_body(MixedIn in, double* __restrict__ R,
                                                                       Geo g, PhysF pf, int accumulate,
    uint3 bid, uint3 gdim, const StageOut* sop = nullptr, const Phys* php = nullptr,
    unsigned* flags = nullptr) {
  static_assert(D == 1 || D == 2, "tiles along y or z");
  constexpr int kTFaces = FPW;
  constexpr int kTCells = kTFaces * NWARP - 1;
  constexpr int kTWarps = NWARP;
  constexpr int NVW = VISC ? 6 : 5;
  constexpr int ND = kTCells + 5;
  constexpr int OTHER = D == 1 ? 2 : 1;                     // the axis that is neither x nor D
  constexpr int NA = 2 * NVW;                               // staged arrays: hi and lo of each primitive
  constexpr int NR = ND + 1;                                // staged rows: cells d0 - 3 .. d0 + kTCells + 2
  constexpr size_t kRawBytes = BULK ? sizeof(float) * NA * NR * kBulkRow : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* raw = reinterpret_cast<float*>(smem_raw);                                      // [NA][NR][36]
  float (*sD)[ND][32] = reinterpret_cast<float (*)[ND][32]>(smem_raw + kRawBytes);      // [6][ND][32]
  double (*sF)[5][32] =
      reinterpret_cast<double (*)[5][32]>(smem_raw + kRawBytes + sizeof(float) * 6 * ND * 32);  // [NWARP][5][32]
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int x = g.h[0] + bid.x * 32 + lane;
  const bool xok = x < g.h[0] + g.n[0];
  const int d0 = g.h[D] + bid.y * kTCells;             // first cell of the tile along D
  const int dend = g.h[D] + g.n[D];
  const int o = g.h[OTHER] + bid.z;
  const int s = D == 1 ? g.sy : g.sz;
  const int so = OTHER == 1 ? g.sy : g.sz;
  const int nc = g.ncell;
  const int colbase = x + o * so;                           // cell index with D coordinate 0
  // fused stage: dt of the step, the third stage's hold (dt <= 0) and its clock update
  double dt = 0.0;
  bool hold = false, bad = false;
  if (STAGE) {
    dt = sop->ctl->dt;
    hold = sop->stage == 3 && !(dt > 0.0);
    if (sop->stage == 3 && !hold && bid.x == 0 && bid.y == 0 && bid.z == 0 && lane == 0 && warp == 0) {
      const double tn = sop->ctl->t + dt;
      sop->ctl->t = (sop->t_end > 0.0 && !(tn < sop->t_end)) ? sop->t_end : tn;
    }
  }
  if (BULK) {
    // stage the rows: warp 0 issues one bulk copy per (array, row) inside the padded grid, all
    // counted on one mbarrier; every thread then waits for the phase (bounded)
    __shared__ __align__(8) unsigned long long s_bar;
    const unsigned bar = smem_u32(&s_bar);
    const int nvalid = min(NR, g.p[D] - (d0 - 3));
    const int colbase0 = g.h[0] + bid.x * 32 + o * so;      // column of lane 0
    if (lane == 0 && warp == 0) mbar_init(bar, 1);
    __syncthreads();
    if (warp == 0) {
      if (lane == 0) mbar_arrive_expect(bar, (unsigned)(NA * nvalid * kBulkRow * sizeof(float)));
      __syncwarp();
      for (int q = lane; q < NA * nvalid; q += 32) {
        const int ar = q / nvalid, k = q - ar * nvalid;
        const float* src = (ar < NVW ? in.hi + (size_t)ar * nc : in.lo + (size_t)(ar - NVW) * nc) +
                           colbase0 + (d0 - 3 + k) * s;
        const uintptr_t a16 = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
        bulk_to_smem(smem_u32(raw + (ar * NR + k) * kBulkRow), reinterpret_cast<const void*>(a16),
                     kBulkRow * sizeof(float), bar);
      }
    }
    const bool late = !mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(late)) {
      // the copies did not complete in time: report it, give copies still in flight into this
      // block's shared memory one more bounded wait, and leave the tile undone
      if (lane == 0 && warp == 0 && flags) atomicOr(flags, FLAG_STAGING);
      if (late) mbar_wait_bounded(bar, 0);
      return;
    }
    // cell differences from the staged rows, in the order diff32 forms them
    auto at = [&](int ar, int k) {
      const float* src = (ar < NVW ? in.hi + (size_t)ar * nc : in.lo + (size_t)(ar - NVW) * nc) +
                         colbase0 + (d0 - 3 + k) * s;
      const int sh = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
      return raw[(ar * NR + k) * kBulkRow + sh + lane];
    };
    for (int k = warp; k < ND; k += kTWarps) {
      const int j = d0 - 3 + k;
      const bool ok = xok && j + 1 <= dend + 2;
#pragma unroll
      for (int v = 0; v < NVW; ++v)
        sD[v][k][lane] = ok ? (at(v, k + 1) - at(v, k)) + (at(NVW + v, k + 1) - at(NVW + v, k)) : 0.0f;
    }
  } else {
    // each warp takes a run of consecutive rows and keeps the previous row's (hi, lo) in
    // registers, so every value is loaded once (the differences are those diff32 forms; the
    // rows' second loads missed L1, which holds about 11 KB per tile beside the shared memory:
    // on TGV 128^3 the y tile 4.5 % faster, the z tile with the stage 1.3 %)
    constexpr int KPW = (ND + kTWarps - 1) / kTWarps;
    const int k0 = warp * KPW, k1 = min(ND, k0 + KPW);
    const int jmax = dend + 2;                              // last padded index along D
#pragma unroll
    for (int v = 0; v < NVW; ++v) {
      const float* hp = in.hi + v * nc + colbase;
      const float* lp = in.lo + v * nc + colbase;
      float h0 = 0.0f, l0 = 0.0f;
      if (xok && k0 < k1 && d0 - 3 + k0 <= jmax) {
        h0 = __ldg(hp + (d0 - 3 + k0) * s);
        l0 = __ldg(lp + (d0 - 3 + k0) * s);
      }
      for (int k = k0; k < k1; ++k) {
        const int j = d0 - 3 + k;
        const bool ok = xok && j + 1 <= jmax;
        float h1 = 0.0f, l1 = 0.0f;
        if (ok) {
          h1 = __ldg(hp + (j + 1) * s);
          l1 = __ldg(lp + (j + 1) * s);
        }
        sD[v][k][lane] = ok ? (h1 - h0) + (l1 - l0) : 0.0f;
        h0 = h1;
        l0 = l1;
      }
    }
  }
  __syncthreads();
  const int f0 = warp * kTFaces;                            // face a + 1/2, a = d0 - 1 + f
  double Fp[5];
  for (int f = f0; f < f0 + kTFaces; ++f) {
    const int a = d0 - 1 + f;
    if (!xok || a >= dend) break;
    float Dw[6][5];
#pragma unroll
    for (int v = 0; v < NVW; ++v)
#pragma unroll
      for (int kk = 0; kk < 5; ++kk) Dw[v][kk] = sD[v][f + kk][lane];
    double F[5];
    face_flux_mixed<D, SCHEME, VISC>(in, colbase + a * s, s, a, Dw, g, pf, F);
    if (f == f0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[warp][v][lane] = F[v];
    } else if (STAGE) {
      stage_cell(*sop, R, in.W, nc, colbase + a * s, g.idx[D][a], F, Fp, dt, hold, *php, bad);
    } else {
      divergence(R, nc, colbase + a * s, g.idx[D][a], F, Fp, accumulate);   // cell a, faces a -+ 1/2
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) Fp[v] = F[v];
  }
  __syncthreads();
  // the last cell of this warp's run, d0 - 1 + f0 + kTFaces: right face from the next warp
  const int a = d0 + f0 + kTFaces - 1;
  if (warp + 1 < kTWarps && xok && a < dend) {
    double F[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = sF[warp + 1][v][lane];
    if (STAGE) stage_cell(*sop, R, in.W, nc, colbase + a * s, g.idx[D][a], F, Fp, dt, hold, *php, bad);
    else divergence(R, nc, colbase + a * s, g.idx[D][a], F, Fp, accumulate);
  }
  if (STAGE && bad) atomicOr(&sop->ctl->flags, FLAG_NONFINITE);
}

template <int D, int SCHEME, bool VISC, int NWARP, int FPW>
__global__ void __launch_bounds__(32 * NWARP, 32 / NWARP) k_face_mixed_t(MixedIn in, double* __restrict__ R,
                                                                       Geo g, PhysF pf, int accumulate) {
  k_face_mixed_t_body<D, SCHEME, VISC, NWARP, FPW>(in, R, g, pf, accumulate, blockIdx, gridDim);
}

// bulk-staged tile (4 warps x 4 faces): the y / z face kernel with its rows staged by cp.async.bulk
template <int D, int SCHEME, bool VISC>
__global__ void __launch_bounds__(128, 4) k_face_mixed_tb(MixedIn in, double* __restrict__ R, Geo g,
                                                          PhysF pf, int accumulate, unsigned* flags) {
  k_face_mixed_t_body<D, SCHEME, VISC, 4, 4, false, true>(in, R, g, pf, accumulate, blockIdx, gridDim,
                                                          nullptr, nullptr, flags);
}

// the last axis's tile kernel with the stage fused (StageOut): R is read, not written
template <int D, int SCHEME, bool VISC, int NWARP, int FPW, int MINB, bool BULK = false>
__global__ void __launch_bounds__(32 * NWARP, MINB) k_face_mixed_ts(MixedIn in, const double* __restrict__ R,
                                                                    Geo g, PhysF pf, StageOut so, Phys ph) {
  k_face_mixed_t_body<D, SCHEME, VISC, NWARP, FPW, true, BULK>(in, const_cast<double*>(R), g, pf, 1, blockIdx,
                                                               gridDim, &so, &ph, &so.ctl->flags);
}


// centre velocity gradients in FP32 from the FP32 primitives (fourth-order central)
__device__ __forceinline__ void k_grad32_body(const float* __restrict__ W32, float* __restrict__ G32, Geo g,
    uint3 bid, uint3 gdim) {
  int lo[3], ext[3];
  for (int a = 0; a < 3; ++a) {
    const int m = a < g.ndim ? 2 : 0;
    lo[a] = g.h[a] - m;
    ext[a] = g.n[a] + 2 * m;
  }
  const int total = ext[0] * ext[1] * ext[2];
  for (int t = bid.x * blockDim.x + threadIdx.x; t < total; t += gdim.x * blockDim.x) {
    int c[3];
    c[0] = lo[0] + t % ext[0];
    const int r = t / ext[0];
    c[1] = lo[1] + r % ext[1];
    c[2] = lo[2] + r / ext[1];
    const int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    for (int b = 0; b < 3; ++b) {
      const bool inb = b < g.ndim && c[b] >= g.h[b] && c[b] < g.h[b] + g.n[b];
      const int s = b == 0 ? 1 : (b == 1 ? g.sy : g.sz);
      const float m = inb ? g.mc32[b][c[b]] : 0.0f;
      for (int comp = 0; comp < 3; ++comp) {
        float d = 0.0f;
        if (inb) {
          const float* f = W32 + (1 + comp) * g.ncell + cell;
          d = ((f[-2 * s] - f[2 * s]) + 8.0f * (f[s] - f[-s])) * (1.0f / 12.0f) * m;
        }
        G32[(comp * 3 + b) * g.ncell + cell] = d;
      }
    }
  }
}

__global__ void k_grad32(const float* __restrict__ W32, float* __restrict__ G32, Geo g) {
  k_grad32_body(W32, G32, g, blockIdx, gridDim);
}

constexpr int kDtBlock = 256;

// CFL partial maxima of the rates (|u| + c) / dx and k nu / dx^2 (the inverse time steps, as in
// the FP64 kernel) from the FP32 primitives: the time step needs no more than FP32 accuracy
__device__ __forceinline__ void k_dt_partial32_body(const float* __restrict__ W32, Geo g, PhysF pf,
                                                           double* __restrict__ partial,
    uint3 bid, uint3 gdim) {
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  float best = 0.0f;
  const float gam = pf.gamma, k = pf.dt_visc_k;
  for (int t = bid.x * blockDim.x + threadIdx.x; t < total; t += gdim.x * blockDim.x) {
    const int i = t % g.n[0];
    const int r = t / g.n[0];
    const int j = r % g.n[1];
    const int kk = r / g.n[1];
    const int ci[3] = {i + g.h[0], j + g.h[1], kk + g.h[2]};
    const int c = ci[0] + ci[1] * g.sy + ci[2] * g.sz;
    const float rho = W32[c], p = W32[4 * nc + c];
    const float irho = rcpf(rho);
    const float cs = sqrtf_a(gam * p * irho);
    float knu = 0.0f;
    if (pf.visc != FLUID_VISC_NONE) knu = k * viscosity_f(W32[5 * nc + c], pf) * irho;
    for (int d = 0; d < g.ndim; ++d) {
      const float id = g.idx32[d][ci[d]];
      best = fmaxf(best, (fabsf(W32[(1 + d) * nc + c]) + cs) * id);
      if (pf.visc != FLUID_VISC_NONE) best = fmaxf(best, knu * id * id);
    }
  }
  __shared__ float sm[kDtBlock / 32];
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < kDtBlock / 32 ? sm[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_down_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) partial[bid.x] = (double)best;
  }
}

__global__ void __launch_bounds__(kDtBlock) k_dt_partial32(const float* __restrict__ W32, Geo g, PhysF pf,
                                                           double* __restrict__ partial) {
  k_dt_partial32_body(W32, g, pf, partial, blockIdx, gridDim);
}

// ---- batched kernels of the serving loop (see BatchTable in fluid_internal.cuh) -----------------
#define FL_BATCH_LOOP(K)                                                        \
  const long long total_ = t->prefix[K][t->nslots];                             \
  for (long long vb = blockIdx.x; vb < total_; vb += gridDim.x) {                \
    const int si_ = batch_slot(t, K, vb);                                       \
    const BatchSlot& S = t->slot[si_];                                          \
    const uint3 bid = batch_bid(S.vgrid[K], vb - t->prefix[K][si_]);            \
    const uint3 gdim = make_uint3(S.vgrid[K][0], S.vgrid[K][1], S.vgrid[K][2]);
#define FL_BATCH_END \
    __syncthreads(); \
  }

__device__ __forceinline__ MixedIn batch_in(const BatchSlot& S) {
  return MixedIn{S.W, S.W32, S.W32 + (size_t)NW * S.g.ncell, S.G32};
}

template <int SCHEME, bool VISC>
__global__ void __launch_bounds__(32 * kXRows) kbm_face_x(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_FACE0)
  if (step < S.steps) k_face_mixed_x_body<SCHEME, VISC>(batch_in(S), S.R, S.g, phys_f(S.ph), 0, bid, gdim);
  FL_BATCH_END
}

template <int D, int SCHEME, bool VISC>
__global__ void __launch_bounds__(128, 8) kbm_face_t(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_FACE0 + D)
  if (step < S.steps)
    k_face_mixed_t_body<D, SCHEME, VISC, kMixedTileWarps, kMixedTileFaces>(batch_in(S), S.R, S.g, phys_f(S.ph), 1,
                                                                          bid, gdim);
  FL_BATCH_END
}

__global__ void __launch_bounds__(256) kbm_grad(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_GRAD)
  if (step < S.steps) k_grad32_body(S.W32, S.G32, S.g, bid, gdim);
  FL_BATCH_END
}

__global__ void __launch_bounds__(kDtBlock) kbm_dtp(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_DTP)
  if (step < S.steps) k_dt_partial32_body(S.W32, S.g, phys_f(S.ph), S.partial, bid, gdim);
  FL_BATCH_END
}

template <class K>
int batch_grid_m(K kernel, int block, size_t smem = 0) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

template <int SCHEME, bool VISC>
cudaError_t batch_face_m(const BatchTable* dev, int D, int step, cudaStream_t st) {
  constexpr size_t smem = t_smem<kMixedTileWarps, kMixedTileFaces>();
  if (D == 0) {
    static const int gx = batch_grid_m(kbm_face_x<SCHEME, VISC>, 32 * kXRows);
    (kbm_face_x<SCHEME, VISC><<<gx, dim3(32, kXRows), 0, st>>>(dev, step), ++t_launches);
    return cudaGetLastError();
  }
  static bool init = false;
  static int g1 = 0, g2 = 0;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(kbm_face_t<1, SCHEME, VISC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kbm_face_t<2, SCHEME, VISC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g1 = batch_grid_m(kbm_face_t<1, SCHEME, VISC>, 128, smem);
    g2 = batch_grid_m(kbm_face_t<2, SCHEME, VISC>, 128, smem);
    init = true;
  }
  if (D == 1) (kbm_face_t<1, SCHEME, VISC><<<g1, dim3(32, kMixedTileWarps), smem, st>>>(dev, step), ++t_launches);
  else (kbm_face_t<2, SCHEME, VISC><<<g2, dim3(32, kMixedTileWarps), smem, st>>>(dev, step), ++t_launches);
  return cudaGetLastError();
}

template <int D, int SCHEME, bool VISC>
cudaError_t launch_t(const MixedIn& in, double* R, const Geo& g, const PhysF& pf, int accumulate,
                     int block, int seg, cudaStream_t st) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const long long lines = (long long)g.n[A1] * g.n[A2];
  if (block <= 0) block = 128;
  if (seg <= 0) {
    seg = 64;
    while (seg > 8 && lines * ((g.n[D] + seg - 1) / seg) < 152LL * 4 * 128) seg >>= 1;
  }
  const long long total = lines * ((g.n[D] + seg - 1) / seg);
  (k_face_mixed<D, SCHEME, VISC><<<grid_for(total, block), block, 0, st>>>(in, R, g, pf, accumulate, seg), ++t_launches);
  return cudaGetLastError();
}

template <int SCHEME, bool VISC, int NWARP, int FPW>
cudaError_t launch_tile(int D, const MixedIn& in, double* R, const Geo& g, const PhysF& pf,
                        int accumulate, cudaStream_t st) {
  constexpr int cells = FPW * NWARP - 1;
  constexpr size_t smem = t_smem<NWARP, FPW>();
  const int other = D == 1 ? 2 : 1;
  const dim3 grid((g.n[0] + 31) / 32, (g.n[D] + cells - 1) / cells, g.n[other]);
  // a tile may need more than the default 48 KB of dynamic shared memory (attribute is per device)
  if (D == 1) {
    cudaError_t e = cudaFuncSetAttribute(k_face_mixed_t<1, SCHEME, VISC, NWARP, FPW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (k_face_mixed_t<1, SCHEME, VISC, NWARP, FPW><<<grid, dim3(32, NWARP), smem, st>>>(in, R, g, pf, accumulate), ++t_launches);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_face_mixed_t<2, SCHEME, VISC, NWARP, FPW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (k_face_mixed_t<2, SCHEME, VISC, NWARP, FPW><<<grid, dim3(32, NWARP), smem, st>>>(in, R, g, pf, accumulate), ++t_launches);
  }
  return cudaGetLastError();
}

template <int SCHEME, bool VISC>
cudaError_t launch_tile_bulk(int D, const MixedIn& in, double* R, const Geo& g, const PhysF& pf,
                             int accumulate, unsigned* flags, cudaStream_t st) {
  constexpr size_t smem = t_smem_bulk<4, 4, VISC ? 6 : 5>();
  const int other = D == 1 ? 2 : 1;
  const dim3 grid((g.n[0] + 31) / 32, (g.n[D] + 14) / 15, g.n[other]);
  if (D == 1) {
    cudaError_t e = cudaFuncSetAttribute(k_face_mixed_tb<1, SCHEME, VISC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (k_face_mixed_tb<1, SCHEME, VISC><<<grid, dim3(32, 4), smem, st>>>(in, R, g, pf, accumulate, flags), ++t_launches);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_face_mixed_tb<2, SCHEME, VISC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (k_face_mixed_tb<2, SCHEME, VISC><<<grid, dim3(32, 4), smem, st>>>(in, R, g, pf, accumulate, flags), ++t_launches);
  }
  return cudaGetLastError();
}

template <int SCHEME, bool VISC>
cudaError_t launch_sv(int D, const MixedIn& in, double* R, const Geo& g, const PhysF& pf,
                      int accumulate, int block, int seg, unsigned* flags, cudaStream_t st) {
  if (D == 0) {
    const long long lines = (long long)g.n[1] * g.n[2];
    const dim3 grid((g.n[0] + kXCells - 1) / kXCells, (unsigned)((lines + kXRows - 1) / kXRows));
    (k_face_mixed_x<SCHEME, VISC><<<grid, dim3(32, kXRows), 0, st>>>(in, R, g, pf, accumulate), ++t_launches);
    return cudaGetLastError();
  }
  const int other = D == 1 ? 2 : 1;
  if (seg < 0 || g.n[other] > 65535) {   // register-window marching kernels
    const int sg = seg < 0 ? -seg : 0;
    if (D == 1) return launch_t<1, SCHEME, VISC>(in, R, g, pf, accumulate, block, sg, st);
    return launch_t<2, SCHEME, VISC>(in, R, g, pf, accumulate, block, sg, st);
  }
  // seg 1: the 4 x 4 tile with its rows staged by bulk copies
  if (seg == 1) return launch_tile_bulk<SCHEME, VISC>(D, in, R, g, pf, accumulate, flags, st);
  // tile shape (warps x faces per warp): block 64 -> 2 x 4, otherwise 4 x 3 (on TGV 128^3 the
  // 4 x 4 tile was the fastest of 16 x 1, 8 x 2, 4 x 4 and 2 x 4, and 4 x 3 beat 4 x 4, 4 x 5 and
  // 4 x 2 by 2.5 % or more over the step)
  if (block == 64) return launch_tile<SCHEME, VISC, 2, 4>(D, in, R, g, pf, accumulate, st);
  return launch_tile<SCHEME, VISC, kMixedTileWarps, kMixedTileFaces>(D, in, R, g, pf, accumulate, st);
}

template <int SCHEME, bool VISC, int NWARP, int FPW, int MINB, bool BULK = false>
cudaError_t launch_tile_stage(int D, const MixedIn& in, const double* R, const Geo& g, const PhysF& pf,
                              const Phys& ph, const StageOut& so, cudaStream_t st) {
  constexpr int cells = FPW * NWARP - 1;
  constexpr size_t smem = BULK ? t_smem_bulk<NWARP, FPW, VISC ? 6 : 5>() : t_smem<NWARP, FPW>();
  const int other = D == 1 ? 2 : 1;
  const dim3 grid((g.n[0] + 31) / 32, (g.n[D] + cells - 1) / cells, g.n[other]);
  if (D == 1) {
    cudaError_t e = cudaFuncSetAttribute(k_face_mixed_ts<1, SCHEME, VISC, NWARP, FPW, MINB, BULK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (k_face_mixed_ts<1, SCHEME, VISC, NWARP, FPW, MINB, BULK><<<grid, dim3(32, NWARP), smem, st>>>(in, R, g, pf, so, ph), ++t_launches);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_face_mixed_ts<2, SCHEME, VISC, NWARP, FPW, MINB, BULK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (k_face_mixed_ts<2, SCHEME, VISC, NWARP, FPW, MINB, BULK><<<grid, dim3(32, NWARP), smem, st>>>(in, R, g, pf, so, ph), ++t_launches);
  }
  return cudaGetLastError();
}

template <int SCHEME, bool VISC>
cudaError_t launch_stage_sv(const MixedIn& in, const double* R, const Geo& g, const PhysF& pf, const Phys& ph,
                            int block, int seg, const StageOut& so, cudaStream_t st) {
  const int D = g.ndim - 1;
  if (seg == 1) return launch_tile_stage<SCHEME, VISC, 4, 4, 4, true>(D, in, R, g, pf, ph, so, st);
  if (block == 64) return launch_tile_stage<SCHEME, VISC, 2, 4, 12>(D, in, R, g, pf, ph, so, st);
  // 4 warps x 3 faces, as the unfused tile; 64 registers (a few bytes spilled) so that 8 tiles
  // fit an SM: on TGV 128^3 6 % faster than 72 registers without spills (7 tiles) and 11 % faster
  // than 80 (6 tiles)
  return launch_tile_stage<SCHEME, VISC, kMixedTileWarps, kMixedTileFaces, 8>(D, in, R, g, pf, ph, so, st);
}

}  // namespace

bool mixed_stage_fusable(const Geo& g, int seg) {
  if (g.ndim < 2 || seg < 0) return false;
  const int other = g.ndim - 1 == 1 ? 2 : 1;
  return g.n[other] <= 65535;
}

cudaError_t launch_face_mixed_stage(const double* W, const float* W32, const float* G32,
                                    const double* R, const Geo& g, const Phys& ph, int block, int seg,
                                    const StageOut& so, cudaStream_t st) {
  const bool visc = ph.visc != FLUID_VISC_NONE;
  const MixedIn in{W, W32, W32 + (size_t)NW * g.ncell, G32};
  const PhysF pf = phys_f(ph);
  if (ph.weno == FLUID_WENO_JS)
    return visc ? launch_stage_sv<FLUID_WENO_JS, true>(in, R, g, pf, ph, block, seg, so, st)
                : launch_stage_sv<FLUID_WENO_JS, false>(in, R, g, pf, ph, block, seg, so, st);
  return visc ? launch_stage_sv<FLUID_WENO_Z, true>(in, R, g, pf, ph, block, seg, so, st)
              : launch_stage_sv<FLUID_WENO_Z, false>(in, R, g, pf, ph, block, seg, so, st);
}

cudaError_t launch_face_mixed(int D, const double* W, const float* W32, const float* G32, double* R,
                              const Geo& g, const Phys& ph, int accumulate, int block, int seg,
                              cudaStream_t st, unsigned* flags) {
  const bool visc = ph.visc != FLUID_VISC_NONE;
  const MixedIn in{W, W32, W32 + (size_t)NW * g.ncell, G32};
  const PhysF pf = phys_f(ph);
  if (ph.weno == FLUID_WENO_JS)
    return visc ? launch_sv<FLUID_WENO_JS, true>(D, in, R, g, pf, accumulate, block, seg, flags, st)
                : launch_sv<FLUID_WENO_JS, false>(D, in, R, g, pf, accumulate, block, seg, flags, st);
  return visc ? launch_sv<FLUID_WENO_Z, true>(D, in, R, g, pf, accumulate, block, seg, flags, st)
              : launch_sv<FLUID_WENO_Z, false>(D, in, R, g, pf, accumulate, block, seg, flags, st);
}

namespace {
// Check of the bulk-staging helpers: one warp stages nrows rows of 36 floats (16-byte aligned) from
// src into shared memory on one mbarrier whose expected transaction count is the rows' bytes plus
// extra_tx, waits with the tiles' bounded wait and copies the rows to dst.  With extra_tx > 0 the
// phase cannot complete (every copy lands, the count stays short), so the wait runs out: the block
// sets FLAG_STAGING in *flags, waits once more and returns without writing dst.
constexpr int kProbeRows = 8;
__global__ void k_bulk_probe(const float* __restrict__ src, float* __restrict__ dst, int nrows,
                             unsigned extra_tx, unsigned* flags) {
  __shared__ __align__(16) float rows[kProbeRows * kBulkRow];
  __shared__ __align__(8) unsigned long long s_bar;
  const unsigned bar = smem_u32(&s_bar);
  const int lane = threadIdx.x;
  if (lane == 0) mbar_init(bar, 1);
  __syncthreads();
  if (lane == 0) mbar_arrive_expect(bar, (unsigned)(nrows * kBulkRow * sizeof(float)) + extra_tx);
  __syncwarp();
  if (lane < nrows)
    bulk_to_smem(smem_u32(rows + lane * kBulkRow), src + lane * kBulkRow, kBulkRow * sizeof(float), bar);
  const bool late = !mbar_wait_bounded(bar, 0);
  if (__syncthreads_or(late)) {
    if (lane == 0) atomicOr(flags, FLAG_STAGING);
    if (late) mbar_wait_bounded(bar, 0);
    return;
  }
  for (int i = lane; i < nrows * kBulkRow; i += 32) dst[i] = rows[i];
}
}  // namespace

cudaError_t launch_bulk_probe(const float* src, float* dst, int nrows, unsigned extra_tx,
                              unsigned* flags, cudaStream_t st) {
  if (nrows < 1 || nrows > kProbeRows || (reinterpret_cast<uintptr_t>(src) & 15) != 0)
    return cudaErrorInvalidValue;
  (k_bulk_probe<<<1, 32, 0, st>>>(src, dst, nrows, extra_tx, flags), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_batch_mixed(const BatchTable* dev, int kind, int D, int step, cudaStream_t st) {
  static const int gg = batch_grid_m(kbm_grad, 256);
  static const int gd = batch_grid_m(kbm_dtp, kDtBlock);
  if (kind == BMX_GRAD) {
    (kbm_grad<<<gg, 256, 0, st>>>(dev, step), ++t_launches);
    return cudaGetLastError();
  }
  if (kind == BMX_DTP) {
    (kbm_dtp<<<gd, kDtBlock, 0, st>>>(dev, step), ++t_launches);
    return cudaGetLastError();
  }
  // the bucket key fixes the scheme and the viscosity, read from the first solve on the host side
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch_mixed_faces(const BatchTable* dev, int D, int step, int weno, bool visc,
                                     cudaStream_t st) {
  if (weno == FLUID_WENO_JS)
    return visc ? batch_face_m<FLUID_WENO_JS, true>(dev, D, step, st) : batch_face_m<FLUID_WENO_JS, false>(dev, D, step, st);
  return visc ? batch_face_m<FLUID_WENO_Z, true>(dev, D, step, st) : batch_face_m<FLUID_WENO_Z, false>(dev, D, step, st);
}

cudaError_t launch_grad32(const float* W32, float* G32, const Geo& g, cudaStream_t st) {
  long long total = 1;
  for (int a = 0; a < 3; ++a) total *= g.n[a] + (a < g.ndim ? 4 : 0);
  (k_grad32<<<grid_for(total, 256), 256, 0, st>>>(W32, G32, g), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_dt_partial32(const float* W32, const Geo& g, const Phys& ph, double* partial,
                                int nparts, cudaStream_t st) {
  (k_dt_partial32<<<nparts, kDtBlock, 0, st>>>(W32, g, phys_f(ph), partial), ++t_launches);
  return cudaGetLastError();
}

}  // namespace fl
