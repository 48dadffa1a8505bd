// FP64 kernels of the finite-volume compressible Navier-Stokes right-hand side (Section 2.1,
// Eq. ODE) and of the TVD-RK3 step.
//
// Pipeline of one right-hand-side evaluation:
//   k_prim_bc   primitives (rho, u, v, w, p, T) of every padded cell; halo cells are built directly
//               from interior cells by composing the boundary maps of the active axes in x, y, z
//               order (Section 3.2: halo cells take values assigned by the boundary conditions)
//   k_grad      fourth- or sixth-order central velocity gradients at cell centres (tangential
//               derivatives of the dissipative fluxes)
//   k_face<D>   per axis D: WENO5 reconstruction of the primitives, HLLC convective flux, the
//               dissipative flux at the same face, and the flux difference -(F+ - F-)/dx into R.
//               One thread marches along a segment of a grid line so each face is computed once
//               and reused by the two cells that share it; a segment starts with the carried
//               terms formed by the march's own operations (march_start), so the result is the
//               same for every segment length.
//   k_face_seam<D>   the first cell of every segment after a line's first, from the two fluxes
//               the neighbouring segments hand over in the seam buffer (with the buffer no face
//               is formed twice)
//   k_source / k_stage   body-force source, RK3 stage combination, non-finite check
//   k_stage_prim / k_halo_prim   the stage combination fused with the primitives of its result
//               (interior cells), then the halo cells from those; fluid_step uses this pair in
//               place of k_stage followed by the next right-hand side's k_prim_bc
//   k_dt_*      CFL time step: per-block minimum, then one block reduces (deterministic)
//
// The state is FP64 structure-of-arrays U[v][z][y][x]; primitives and gradients live in solver
// scratch with the same padded layout.
#include <cuda_runtime.h>

#include <algorithm>

#include "flux_math.cuh"
#include "fluid_internal.cuh"

namespace fl {

namespace {

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
  const double u[5] = {U[c], U[nc + c], U[2 * nc + c], U[3 * nc + c], U[4 * nc + c]};
  prim_from_cons(u, ph, w);
}

__device__ __forceinline__ void wall_map(double w[NW], int kind, double Tw, double vw, int a,
                                         const Phys& ph, unsigned* flags) {
  if (!wall_map_prim(w, kind, Tw, vw, a, ph)) atomicOr(flags, FLAG_GHOST_T);
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

// primitives of padded cell own[] (interior: from U; halo: composed boundary maps); E receives the
// total energy per volume of interior cells (halo cells leave it unset).
//
// The halo passes x -> y -> z compose: the pass of axis a sees own indices on the axes before it
// and source indices on the axes after it, so a halo cell starts from the cell at the source index
// on every axis and then takes the maps of its halo axes in order (an inflow axis replaces the
// state by its profile).  Every cell therefore converts exactly one cell's U -- its own or its
// source -- and only wall halos run map arithmetic, so warps that straddle the x halo do not run
// the conversion twice.
// Source cell of padded cell own[]: ghost[a] / side[a] / src[a] per axis; returns whether any axis
// is a halo axis (then src[] is the interior cell the halo maps start from).
// The halo layers of an exchange face (a sub-domain boundary of a block decomposition) hold the
// neighbouring block's cells: along that axis the cell is its own source, like an interior cell.
__device__ __forceinline__ bool halo_source(const int own[3], const Geo& g, const BC& bc,
                                            bool ghost[3], int side[3], int src[3]) {
  bool any = false;
  for (int a = 0; a < 3; ++a) {
    side[a] = own[a] < g.h[a] ? 0 : 1;
    ghost[a] = (own[a] < g.h[a] || own[a] >= g.h[a] + g.n[a]) &&
               bc.kind[a][side[a]] != FLUID_BC_EXCHANGE;
    src[a] = ghost[a] ? bc_source(bc.kind[a][side[a]], side[a], own[a], g.n[a], g.h[a]) : own[a];
    any |= ghost[a];
  }
  return any;
}

// the maps of the halo axes of a cell, in axis order, applied to the primitives w of its source;
// returns whether any of them changes values (a wall or inflow map) rather than only indices
__device__ __forceinline__ bool halo_maps(const int own[3], const bool ghost[3], const int side[3],
                                          const int src[3], const Geo& g, const Phys& ph,
                                          const BC& bc, Ctl* ctl, double w[NW]) {
  bool valued = false;
  for (int a = 0; a < 3; ++a) {
    if (!ghost[a]) continue;
    const int kind = bc.kind[a][side[a]];
    if (kind == FLUID_BC_PERIODIC || kind == FLUID_BC_ZERO_GRADIENT) continue;
    valued = true;
    int c[3];
    for (int b = 0; b < 3; ++b) c[b] = b < a ? own[b] : src[b];
    if (kind == FLUID_BC_INFLOW) {
      inflow_at(bc.inflow[a][side[a]], a, c, g, ph, w);
      continue;
    }
    double vw = 0.0;
    if (kind == FLUID_BC_POROUS) vw = bc.vw[c[bc.porous_t1]];
    wall_map(w, kind, bc.Tw[a][side[a]], vw, a, ph, &ctl->flags);
  }
  return valued;
}

// primitives of padded cell own[] (interior: from U; halo: composed boundary maps); E receives the
// total energy per volume of the source cell (the cell itself when interior) unless a wall or
// inflow map changed the values, which the return value says (then E is left unset).
//
// The halo passes x -> y -> z compose: the pass of axis a sees own indices on the axes before it
// and source indices on the axes after it, so a halo cell starts from the cell at the source index
// on every axis and then takes the maps of its halo axes in order (an inflow axis replaces the
// state by its profile).  Every cell therefore converts exactly one cell's U -- its own or its
// source -- and only wall halos run map arithmetic, so warps that straddle the x halo do not run
// the conversion twice.
__device__ __forceinline__ bool prim_cell(const double* __restrict__ U, const int own[3], int cell,
                                          const Geo& g, const Phys& ph, const BC& bc, Ctl* ctl,
                                          double w[NW], double& E) {
  bool ghost[3];
  int side[3], src[3];
  const bool any = halo_source(own, g, bc, ghost, side, src);
  const int scell = any ? src[0] + src[1] * g.sy + src[2] * g.sz : cell;
  prim_of(U, scell, g.ncell, ph, w);
  E = U[4 * g.ncell + scell];
  if (!any) return false;
  return halo_maps(own, ghost, side, src, g, ph, bc, ctl, w);
}

// One thread per padded cell: x from the thread index, y and z from the block index.
// MIXED: the primitives also go to W32 = [2 NW][ncell] floats as the split (hi, lo) above, and
// H = E + p to the FP64 row W[NW]; the FP32 face kernels form their cell differences from the pairs.
template <bool MIXED>
__device__ __forceinline__ void k_prim_bc_body(const double* __restrict__ U, double* __restrict__ W,
                          float* __restrict__ W32, Geo g, Phys ph, BC bc, Ctl* ctl,
    uint3 bid, uint3 gdim) {
  const int i = bid.x * blockDim.x + threadIdx.x;
  if (i >= g.p[0]) return;
  for (int k = bid.z; k < g.p[2]; k += gdim.z)
    for (int j = bid.y; j < g.p[1]; j += gdim.y) {
      const int own[3] = {i, j, k};
      const int cell = i + j * g.sy + k * g.sz;
      double w[NW];
      double E = 0.0;
      // H = E + p of a halo cell: the source cell's own value when only indices map (periodic,
      // zero gradient, exchange), so that it equals the source's H bitwise; recomputed from the
      // mapped primitives after a wall or inflow map
      const bool valued = prim_cell(U, own, cell, g, ph, bc, ctl, w, E);
      for (int v = 0; v < NW; ++v) W[v * g.ncell + cell] = w[v];
      if (MIXED) {
        for (int v = 0; v < NW; ++v)
          split_hi_lo(w[v], W32[v * g.ncell + cell], W32[(NW + v) * g.ncell + cell]);
        if (valued) E = w[4] * ph.igm1 + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        W[NW * g.ncell + cell] = E + w[4];
      }
    }
}

template <bool MIXED>
__global__ void k_prim_bc(const double* __restrict__ U, double* __restrict__ W,
                          float* __restrict__ W32, Geo g, Phys ph, BC bc, Ctl* ctl) {
  k_prim_bc_body<MIXED>(U, W, W32, g, ph, bc, ctl, blockIdx, gridDim);
}

// ------------------------------------------------------------------------------------------------
// centre gradients G[c*3+b] = d u_c / d x_b, only where the cell is interior along b (the only
// places the face fluxes read it), for the cells the face stencils reach along the other axes:
//   order 4: ((f[-2] - f[+2]) + 8 (f[+1] - f[-1])) * (mc / 12)
//   order 6: (45 (f[+1] - f[-1]) - 9 (f[+2] - f[-2]) + (f[+3] - f[-3])) * (mc / 60)
// ------------------------------------------------------------------------------------------------
template <int ORDER>
__device__ __forceinline__ void k_grad_body(const double* __restrict__ W, double* __restrict__ G, Geo g,
    uint3 bid, uint3 gdim) {
  constexpr int M = ORDER / 2;
  int lo[3], ext[3];
  for (int a = 0; a < 3; ++a) {
    const int m = a < g.ndim ? M : 0;
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
      // the stencil's 1/12 (1/60) and the metric as one factor per axis
      const double cm = inb ? (ORDER == 4 ? kTwelfth : 1.0 / 60.0) * g.mc[b][c[b]] : 0.0;
      for (int comp = 0; comp < 3; ++comp) {
        double d = 0.0;
        if (inb) {
          const double* f = W + (1 + comp) * g.ncell + cell;
          // explicit fused multiply-adds: every kernel inlining this rounds alike
          if (ORDER == 4)
            d = fma(8.0, f[s] - f[-s], f[-2 * s] - f[2 * s]) * cm;
          else
            d = fma(45.0, f[s] - f[-s], fma(-9.0, f[2 * s] - f[-2 * s], f[3 * s] - f[-3 * s])) * cm;
        }
        G[(comp * 3 + b) * g.ncell + cell] = d;
      }
    }
  }
}

template <int ORDER>
__global__ void k_grad(const double* __restrict__ W, double* __restrict__ G, Geo g) {
  k_grad_body<ORDER>(W, G, g, blockIdx, gridDim);
}

// ------------------------------------------------------------------------------------------------
// face flux F^c - F^d at face a+1/2 along D; `cell` is the padded index of cell a, s its stride
// ------------------------------------------------------------------------------------------------
template <int D, int SCHEME, int VORD>
__device__ __forceinline__ void face_flux(const double* __restrict__ W, const double* __restrict__ G,
                                          int cell, int s, int a, const Geo& g, const Phys& ph,
                                          double F[5], double xl[5][3], double k0[5], double k1[5]) {
  // Carried along the march, per primitive: xl, the scaled weights (weno_x) of the left-biased
  // value at this face, whose indicator set (A_{a-1}, B_a, C_{a+1}) was the right-biased set of
  // the previous face; k0, k1 = (13/3) t^2 + 4 eps of the stencils centred at a and a+1 (epsilon
  // enters each indicator through its stencil's carried term).  The right-biased value needs
  // C_{a+2}, B_{a+1}, A_a: one new stencil (centred at a+2) per face.
  // The indicators are taken times 4 (13/3 t^2 + s^2) with epsilon times 4: the weights of
  // either scheme are homogeneous in (beta + eps, tau), so the normalised weights are unchanged.
  const int nc = g.ncell;
  const double eps4 = 4.0 * ph.eps;
  double q[5][6];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int o = 0; o < 6; ++o) q[v][o] = __ldg(W + v * nc + cell + (o - 2) * s);
  double wl[5], wr[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    // cells a-2 .. a+3 are q[v][0..5]; d_j = q[v][j+1] - q[v][j]
    const double d0 = q[v][1] - q[v][0], d1 = q[v][2] - q[v][1], d2 = q[v][3] - q[v][2];
    const double d3 = q[v][4] - q[v][3], d4 = q[v][5] - q[v][4];
    const double t2 = d4 - d3;
    const double k2 = fma((4.0 * k1312) * t2, t2, eps4);   // (13/3) t^2 + 4 eps, cells a+1 .. a+3
    const double sA = fma(3.0, d2, -d1);                   // q_{a-1} - 4 q_a + 3 q_{a+1}
    const double sB = d2 + d3;                             // -(q_a - q_{a+2})
    const double sC = fma(-3.0, d3, d4);                   // 3 q_{a+1} - 4 q_{a+2} + q_{a+3}
    const double An = fma(sA, sA, k0[v]);                  // 4 (A_a + eps)
    const double Bn = fma(sB, sB, k1[v]);                  // 4 (B_{a+1} + eps)
    const double Cn = fma(sC, sC, k2);                     // 4 (C_{a+2} + eps)
    wl[v] = weno_x_value(q[v][2], d0, d1, d2, d3, xl[v]);
    double xr[3];
    weno_x<SCHEME>(Cn, Bn, An, xr);
    // mirrored stencil: centre q_{a+1}, differences -d4, -d3, -d2, -d1
    wr[v] = weno_x_value(q[v][3], -d4, -d3, -d2, -d1, xr);
    xl[v][0] = xr[2];
    xl[v][1] = xr[1];
    xl[v][2] = xr[0];
    k0[v] = k1[v];
    k1[v] = k2;
  }
  hllc<D>(wl, wr, ph, F);
  if (VORD) add_visc_face<D, VORD ? VORD : 4>(W, G, cell, s, a, g, ph, q, F);
}

// The carried terms with which the march arrives at face a+1/2, formed by the operations the
// march itself uses at face a-1/2 from cells a-2 .. a+2 (q[0..4]): the scaled weights xl of the
// left-biased set (A_{a-1}, B_a, C_{a+1}) and k0, k1 = (13/3) t^2 + 4 eps of the stencils centred at
// a and a+1.  A segment start therefore continues bit for bit as if the march had come from
// further back, and the right-hand side does not depend on the segment length.
template <int SCHEME>
__device__ __forceinline__ void march_start(const double q[5], double eps4, double xl[3],
                                            double& k0, double& k1) {
  const double d1 = q[1] - q[0], d2 = q[2] - q[1], d3 = q[3] - q[2], d4 = q[4] - q[3];
  const double c = 4.0 * k1312;
  const double t1 = d2 - d1, t2 = d3 - d2, t3 = d4 - d3;
  const double km = fma(c * t1, t1, eps4);                  // centred at a-1
  k0 = fma(c * t2, t2, eps4);                               // centred at a
  k1 = fma(c * t3, t3, eps4);                               // centred at a+1
  const double sA = fma(3.0, d2, -d1), sB = d2 + d3, sC = fma(-3.0, d3, d4);
  double xr[3];
  weno_x<SCHEME>(fma(sC, sC, k1), fma(sB, sB, k0), fma(sA, sA, km), xr);
  xl[0] = xr[2];
  xl[1] = xr[1];
  xl[2] = xr[0];
}

// R_a (+)= -(F_{a+1/2} - F_{a-1/2}) / dx_a with the product rounded before the sum (no fused
// multiply-add), so that k_face and k_face_seam give the same bits
__device__ __forceinline__ void update_r(double* dst, double F, double Fp, double id, int accumulate) {
  const double val = __dmul_rn(-(F - Fp), id);
  *dst = accumulate ? *dst + val : val;
}

// With a seam buffer FB (2 x 5 doubles per segment, [side][v][item]), a segment after the first
// starts its march at face a0+1/2 instead of a0-1/2: it leaves its first cell a0 to k_face_seam,
// with the flux at a0+1/2 in FB side 0, and its own last flux goes to FB side 1 of the next
// segment, which is the flux at that segment's a0-1/2.  Every face is then formed once; without FB
// each segment forms the face before its first cell as well.  Both give the same bits.
template <int D, int SCHEME, int VORD>
__device__ __forceinline__ void k_face_body(const double* __restrict__ W,
                                              const double* __restrict__ G, double* __restrict__ R,
                                              double* __restrict__ FB, Geo g, Phys ph,
                                              int accumulate, int seg,
    uint3 bid, uint3 gdim) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const int n1 = g.n[A1], n2 = g.n[A2], nd = g.n[D];
  const int nseg = (nd + seg - 1) / seg;
  const long long lines = (long long)n1 * n2;
  const long long total = lines * nseg;
  const int s = D == 0 ? 1 : (D == 1 ? g.sy : g.sz);
  const int nc = g.ncell;
  for (long long t = bid.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gdim.x * blockDim.x) {
    const int i1 = (int)(t % n1);
    const long long r = t / n1;
    const int i2 = (int)(r % n2);
    const int sg = (int)(r / n2);
    int c[3];
    c[A1] = i1 + g.h[A1];
    c[A2] = i2 + g.h[A2];
    const int a0 = g.h[D] + sg * seg;
    const int a1 = min(a0 + seg, g.h[D] + nd);
    const bool seam = FB != nullptr && sg > 0;
    c[D] = seam ? a0 : a0 - 1;
    int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    double Fp[5], F[5], xl[5][3], k0[5], k1[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      // the left-biased set of the march's first face and the stencil terms it carries forward
      const double* f = W + v * nc + cell;
      const double qw[5] = {__ldg(f - 2 * s), __ldg(f - s), __ldg(f), __ldg(f + s), __ldg(f + 2 * s)};
      march_start<SCHEME>(qw, 4.0 * ph.eps, xl[v], k0[v], k1[v]);
    }
    face_flux<D, SCHEME, VORD>(W, G, cell, s, c[D], g, ph, Fp, xl, k0, k1);
    if (seam) {
#pragma unroll
      for (int v = 0; v < 5; ++v) FB[v * total + t] = Fp[v];
    }
    for (int a = seam ? a0 + 1 : a0; a < a1; ++a) {
      cell += s;
      face_flux<D, SCHEME, VORD>(W, G, cell, s, a, g, ph, F, xl, k0, k1);
      const double id = g.idx[D][a];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        update_r(R + v * nc + cell, F[v], Fp[v], id, accumulate);
        Fp[v] = F[v];
      }
    }
    if (FB != nullptr && sg + 1 < nseg) {
#pragma unroll
      for (int v = 0; v < 5; ++v) FB[(5 + v) * total + t + lines] = Fp[v];
    }
  }
}

template <int D, int SCHEME, int VORD>
__global__ void __launch_bounds__(128) k_face(const double* __restrict__ W,
                                              const double* __restrict__ G, double* __restrict__ R,
                                              double* __restrict__ FB, Geo g, Phys ph,
                                              int accumulate, int seg) {
  k_face_body<D, SCHEME, VORD>(W, G, R, FB, g, ph, accumulate, seg, blockIdx, gridDim);
}

// The first cell a0 of every segment after the first: the same update as the face kernel that
// filled FB, from the two fluxes its neighbouring segments left there (FUSED: the TENO kernel's
// form, R = fma(-1/dx, F+ - F-, R))
template <int D, bool FUSED>
__device__ __forceinline__ void k_face_seam_body(const double* __restrict__ FB, double* __restrict__ R, Geo g,
                            int accumulate, int seg,
    uint3 bid, uint3 gdim) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const int n1 = g.n[A1], n2 = g.n[A2], nd = g.n[D];
  const int nseg = (nd + seg - 1) / seg;
  const long long lines = (long long)n1 * n2;
  const long long total = lines * nseg;
  const int nc = g.ncell;
  for (long long t = lines + bid.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gdim.x * blockDim.x) {
    const int i1 = (int)(t % n1);
    const long long r = t / n1;
    const int i2 = (int)(r % n2);
    const int sg = (int)(r / n2);
    int c[3];
    c[A1] = i1 + g.h[A1];
    c[A2] = i2 + g.h[A2];
    c[D] = g.h[D] + sg * seg;
    const int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    const double id = g.idx[D][c[D]];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double Fv = FB[v * total + t], Fpv = FB[(5 + v) * total + t];
      double* dst = R + v * nc + cell;
      if (FUSED) {
        const double dF = Fv - Fpv;
        *dst = accumulate ? fma(-id, dF, *dst) : -id * dF;
      } else {
        update_r(dst, Fv, Fpv, id, accumulate);
      }
    }
  }
}

template <int D, bool FUSED>
__global__ void k_face_seam(const double* __restrict__ FB, double* __restrict__ R, Geo g,
                            int accumulate, int seg) {
  k_face_seam_body<D, FUSED>(FB, R, g, accumulate, seg, blockIdx, gridDim);
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
    R[4 * nc + c] += fma(ph.f[0], u, fma(ph.f[1], v, ph.f[2] * w));
  }
}

// stage 1: Ud = Un + dt r; stage 2: Ud = 3/4 Un + 1/4 (Us + dt r); stage 3: Ud = 1/3 Un + 2/3 (Us + dt r)
__device__ __forceinline__ void k_stage_body(int stage, const double* Un, const double* Us, const double* __restrict__ R,
                        double* Ud, const double* __restrict__ W, Geo g, Phys ph, Ctl* ctl,
                        double t_end, double dt_arg,
    uint3 bid, uint3 gdim) {
  const double dt = dt_arg > 0.0 ? dt_arg : ctl->dt;
  if (stage == 3 && dt_arg <= 0.0 && bid.x == 0 && threadIdx.x == 0 && dt > 0.0) {
    const double tn = ctl->t + dt;
    ctl->t = (t_end > 0.0 && !(tn < t_end)) ? t_end : tn;
  }
  if (stage == 3 && !(dt > 0.0)) return;
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  bool bad = false;
  for (int t = bid.x * blockDim.x + threadIdx.x; t < total; t += gdim.x * blockDim.x) {
    const int c = interior_cell(t, g);
    double r[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v] = R[v * nc + c];
    if (ph.has_force) {
      const double u = W[nc + c], v = W[2 * nc + c], w = W[3 * nc + c];
      r[1] += ph.f[0];
      r[2] += ph.f[1];
      r[3] += ph.f[2];
      r[4] += fma(ph.f[0], u, fma(ph.f[1], v, ph.f[2] * w));
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double un = Un[v * nc + c];
      double out;
      if (stage == 1) {
        out = fma(dt, r[v], un);
      } else {
        const double us = Us[v * nc + c];
        out = stage == 2 ? fma(0.75, un, 0.25 * fma(dt, r[v], us))
                         : fma(1.0 / 3.0, un, (2.0 / 3.0) * fma(dt, r[v], us));
      }
      bad |= !finite_bits(out);
      Ud[v * nc + c] = out;
    }
  }
  if (bad) atomicOr(&ctl->flags, FLAG_NONFINITE);
}

__global__ void k_stage(int stage, const double* Un, const double* Us, const double* __restrict__ R,
                        double* Ud, const double* __restrict__ W, Geo g, Phys ph, Ctl* ctl,
                        double t_end, double dt_arg) {
  k_stage_body(stage, Un, Us, R, Ud, W, g, ph, ctl, t_end, dt_arg, blockIdx, gridDim);
}

// One RK3 stage fused with the primitives of its result (the next right-hand side's first pass):
// interior cell c gets Ud = the stage combination of k_stage, and W (and for MIXED the W32 split and
// H) from Ud by the same conversion k_prim_bc applies, so the halo cells (k_halo_prim, next) and
// the following kernels see exactly what k_prim_bc would have produced.  W is read (body-force
// velocities of the stage's input state) and rewritten only at the thread's own cell.  A third
// stage with dt <= 0 leaves Un unwritten and converts it as it is.
template <bool MIXED>
__device__ __forceinline__ void k_stage_prim_body(int stage, const double* Un, const double* Us, const double* __restrict__ R,
                             double* Ud, double* W, float* __restrict__ W32, Geo g, Phys ph, Ctl* ctl,
                             double t_end,
    uint3 bid, uint3 gdim) {
  const double dt = ctl->dt;
  const bool hold = stage == 3 && !(dt > 0.0);
  if (stage == 3 && !hold && bid.x == 0 && bid.y == 0 && bid.z == 0 && threadIdx.x == 0) {
    const double tn = ctl->t + dt;
    ctl->t = (t_end > 0.0 && !(tn < t_end)) ? t_end : tn;
  }
  const int i = bid.x * blockDim.x + threadIdx.x;
  if (i >= g.n[0]) return;
  const int nc = g.ncell;
  // two cells per thread, rows j and j + J2, with every load of both issued before any store, so
  // that the two conversions' FP64 chains overlap
  const int J2 = (g.n[1] + 1) >> 1;
  bool bad = false;
  for (int k = bid.z; k < g.n[2]; k += gdim.z)
    for (int j = bid.y; j < J2; j += gdim.y) {
      const int base = (i + g.h[0]) + (k + g.h[2]) * g.sz;
      const bool two = j + J2 < g.n[1];
      const int c[2] = {base + (j + g.h[1]) * g.sy, base + (j + J2 + g.h[1]) * g.sy};
      double un[2][5], rs[2][5], us[2][5], vel[2][3];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q == 1 && !two) break;
#pragma unroll
        for (int v = 0; v < 5; ++v) un[q][v] = Un[v * nc + c[q]];
        if (!hold) {
#pragma unroll
          for (int v = 0; v < 5; ++v) rs[q][v] = R[v * nc + c[q]];
          if (stage != 1) {
#pragma unroll
            for (int v = 0; v < 5; ++v) us[q][v] = Us[v * nc + c[q]];
          }
          if (ph.has_force) {
#pragma unroll
            for (int b = 0; b < 3; ++b) vel[q][b] = W[(1 + b) * nc + c[q]];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q == 1 && !two) break;
        double u[5];
        if (hold) {
#pragma unroll
          for (int v = 0; v < 5; ++v) u[v] = un[q][v];
        } else {
          double* r = rs[q];
          if (ph.has_force) {
            r[1] += ph.f[0];
            r[2] += ph.f[1];
            r[3] += ph.f[2];
            r[4] += fma(ph.f[0], vel[q][0], fma(ph.f[1], vel[q][1], ph.f[2] * vel[q][2]));
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            double out;
            if (stage == 1) {
              out = fma(dt, r[v], un[q][v]);
            } else {
              out = stage == 2 ? fma(0.75, un[q][v], 0.25 * fma(dt, r[v], us[q][v]))
                               : fma(1.0 / 3.0, un[q][v], (2.0 / 3.0) * fma(dt, r[v], us[q][v]));
            }
            bad |= !finite_bits(out);
            Ud[v * nc + c[q]] = out;
            u[v] = out;
          }
        }
        double w[NW];
        prim_from_cons(u, ph, w);
#pragma unroll
        for (int v = 0; v < NW; ++v) W[v * nc + c[q]] = w[v];
        if (MIXED) {
#pragma unroll
          for (int v = 0; v < NW; ++v) split_hi_lo(w[v], W32[v * nc + c[q]], W32[(NW + v) * nc + c[q]]);
          W[NW * nc + c[q]] = u[4] + w[4];
        }
      }
    }
  if (bad) atomicOr(&ctl->flags, FLAG_NONFINITE);
}

template <bool MIXED>
__global__ void k_stage_prim(int stage, const double* Un, const double* Us, const double* __restrict__ R,
                             double* Ud, double* W, float* __restrict__ W32, Geo g, Phys ph, Ctl* ctl,
                             double t_end) {
  k_stage_prim_body<MIXED>(stage, Un, Us, R, Ud, W, W32, g, ph, ctl, t_end, blockIdx, gridDim);
}

// Halo cells only, from the interior primitives already in W: the maps of k_prim_bc applied to the
// source cell's primitives.  Cells are enumerated by their highest halo axis a: axes above a
// interior, axis a one of its 2 h[a] halo layers, axes below a anywhere in the padded range.
template <bool MIXED>
__device__ __forceinline__ void k_halo_prim_body(double* __restrict__ W, float* __restrict__ W32, Geo g, Phys ph, BC bc,
                            Ctl* ctl, long long total,
    uint3 bid, uint3 gdim) {
  const int nc = g.ncell;
  for (long long t0 = bid.x * (long long)blockDim.x + threadIdx.x; t0 < total;
       t0 += (long long)gdim.x * blockDim.x) {
    long long t = t0;
    int own[3] = {0, 0, 0};
    for (int a = 2; a >= 0; --a) {
      long long cnt = 2LL * g.h[a];
      for (int b = 0; b < 3; ++b)
        if (b != a) cnt *= b < a ? g.p[b] : g.n[b];
      if (t >= cnt) {
        t -= cnt;
        continue;
      }
      for (int b = 0; b < a; ++b) {
        own[b] = (int)(t % g.p[b]);
        t /= g.p[b];
      }
      const int l = (int)(t % (2 * g.h[a]));
      t /= 2 * g.h[a];
      own[a] = l < g.h[a] ? l : g.n[a] + l;
      for (int b = a + 1; b < 3; ++b) {
        own[b] = g.h[b] + (int)(t % g.n[b]);
        t /= g.n[b];
      }
      break;
    }
    bool ghost[3];
    int side[3], src[3];
    halo_source(own, g, bc, ghost, side, src);
    const int scell = src[0] + src[1] * g.sy + src[2] * g.sz;
    const int cell = own[0] + own[1] * g.sy + own[2] * g.sz;
    double w[NW];
#pragma unroll
    for (int v = 0; v < NW; ++v) w[v] = W[v * nc + scell];
    const bool valued = halo_maps(own, ghost, side, src, g, ph, bc, ctl, w);
#pragma unroll
    for (int v = 0; v < NW; ++v) W[v * nc + cell] = w[v];
    if (MIXED) {
#pragma unroll
      for (int v = 0; v < NW; ++v) split_hi_lo(w[v], W32[v * nc + cell], W32[(NW + v) * nc + cell]);
      // as k_prim_bc: index-only maps keep the source's H, value maps recompute it
      if (valued) {
        const double E = w[4] * ph.igm1 + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        W[NW * nc + cell] = E + w[4];
      } else {
        W[NW * nc + cell] = W[NW * nc + scell];
      }
    }
  }
}

template <bool MIXED>
__global__ void k_halo_prim(double* __restrict__ W, float* __restrict__ W32, Geo g, Phys ph, BC bc,
                            Ctl* ctl, long long total) {
  k_halo_prim_body<MIXED>(W, W32, g, ph, bc, ctl, total, blockIdx, gridDim);
}

constexpr int kDtBlock = 256;

// CFL: dt = cfl * min over cells and axes of dx / (|u| + c) and dx^2 / (k nu), taken as
// cfl / max of the rates (|u| + c) / dx and k nu / dx^2 so that a cell costs no division.
// Per-block maxima of the rate go to `partial`.
__device__ __forceinline__ void k_dt_partial_body(const double* __restrict__ W, Geo g, Phys ph,
                                                         double* __restrict__ partial,
    uint3 bid, uint3 gdim) {
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  double best = 0.0;
  for (int t = bid.x * blockDim.x + threadIdx.x; t < total; t += gdim.x * blockDim.x) {
    const int i = t % g.n[0];
    const int r = t / g.n[0];
    const int j = r % g.n[1];
    const int k = r / g.n[1];
    const int ci[3] = {i + g.h[0], j + g.h[1], k + g.h[2]};
    const int c = ci[0] + ci[1] * g.sy + ci[2] * g.sz;
    const double rho = W[c], p = W[4 * nc + c];
    const double irho = fl_rcp(rho);
    const double cs = fl_sqrt(ph.gamma * p * irho);
    double knu = 0.0;
    if (ph.visc != FLUID_VISC_NONE) knu = ph.dt_visc_k * viscosity(W[5 * nc + c], ph) * irho;
    for (int d = 0; d < g.ndim; ++d) {
      const double id = g.idx[d][ci[d]];
      best = fmax(best, (fabs(W[(1 + d) * nc + c]) + cs) * id);
      if (ph.visc != FLUID_VISC_NONE) best = fmax(best, knu * id * id);
    }
  }
  __shared__ double sm[kDtBlock / 32];
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < kDtBlock / 32 ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) partial[bid.x] = best;
  }
}

__global__ void __launch_bounds__(kDtBlock) k_dt_partial(const double* __restrict__ W, Geo g, Phys ph,
                                                         double* __restrict__ partial) {
  k_dt_partial_body(W, g, ph, partial, blockIdx, gridDim);
}

// dt = cfl / max(partial rates) (or dt_fixed); clip_to_ctl: clip so that t does not pass t_end and
// store in ctl->dt; otherwise write *dt_out.
__device__ __forceinline__ void k_dt_final_body(const double* __restrict__ partial, int nparts,
                                                       Phys ph, Ctl* ctl, double* dt_out, int clip,
                                                       double t_end,
    uint3 bid, uint3 gdim) {
  double best = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) best = fmax(best, partial[i]);
  __shared__ double sm[kDtBlock / 32];
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kDtBlock / 32; ++i) best = fmax(best, sm[i]);
    double dt = ph.dt_fixed > 0.0 ? ph.dt_fixed : ph.cfl / best;
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

__global__ void __launch_bounds__(kDtBlock) k_dt_final(const double* __restrict__ partial, int nparts,
                                                       Phys ph, Ctl* ctl, double* dt_out, int clip,
                                                       double t_end) {
  k_dt_final_body(partial, nparts, ph, ctl, dt_out, clip, t_end, blockIdx, gridDim);
}

// Halo exchange of a block decomposition: element t of the buffer [5][3][e2][e1] (t1 < t2 the axes
// other than A; e_b = p_b below A, n_b above A, starting at 0 resp. h_b) and the padded cell it
// maps to: layer l of face (A, side) is h + l / n + l (interior layers, packed) or l / h + n + l
// (halo layers, unpacked).
__global__ void k_halo_copy(double* __restrict__ U, double* __restrict__ buf, Geo g, int A,
                            int side, int unpack, long long total) {
  const int t1 = A == 0 ? 1 : 0, t2 = A == 2 ? 1 : 2;
  const int e1 = t1 < A ? g.p[t1] : g.n[t1], o1 = t1 < A ? 0 : g.h[t1];
  const int e2 = t2 < A ? g.p[t2] : g.n[t2], o2 = t2 < A ? 0 : g.h[t2];
  const int h = g.h[A], n = g.n[A];
  const int l0 = unpack ? (side == 0 ? 0 : h + n) : (side == 0 ? h : n);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long r = t;
    const int i1 = (int)(r % e1);
    r /= e1;
    const int i2 = (int)(r % e2);
    r /= e2;
    const int l = (int)(r % 3);
    const int v = (int)(r / 3);
    int c[3];
    c[A] = l0 + l;
    c[t1] = o1 + i1;
    c[t2] = o2 + i2;
    const long long cell = (long long)v * g.ncell + c[0] + (long long)c[1] * g.sy + (long long)c[2] * g.sz;
    if (unpack) U[cell] = buf[t];
    else buf[t] = U[cell];
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

template <int D, int SCHEME, int VORD>
cudaError_t launch_face_t(const double* W, const double* G, double* R, const Geo& g,
                          const Phys& ph, int accumulate, int block, int seg, SeamBuf fb,
                          cudaStream_t st) {
  int grid;
  face_shape(D, g, block, seg, grid);
  double* FB = seam_buffer(D, g, seg, fb);
  (k_face<D, SCHEME, VORD><<<grid, block, 0, st>>>(W, G, R, FB, g, ph, accumulate, seg), ++t_launches);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !FB) return e;
  return launch_face_seam(D, FB, R, g, accumulate, seg, false, st);
}

template <int SCHEME, int VORD>
cudaError_t launch_face_sv(int D, const double* W, const double* G, double* R, const Geo& g,
                           const Phys& ph, int accumulate, int block, int seg, SeamBuf fb,
                           cudaStream_t st) {
  if (D == 0) return launch_face_t<0, SCHEME, VORD>(W, G, R, g, ph, accumulate, block, seg, fb, st);
  if (D == 1) return launch_face_t<1, SCHEME, VORD>(W, G, R, g, ph, accumulate, block, seg, fb, st);
  return launch_face_t<2, SCHEME, VORD>(W, G, R, g, ph, accumulate, block, seg, fb, st);
}

template <int SCHEME>
cudaError_t launch_face_s(int D, const double* W, const double* G, double* R, const Geo& g,
                          const Phys& ph, int accumulate, int block, int seg, SeamBuf fb,
                          cudaStream_t st) {
  if (ph.visc == FLUID_VISC_NONE)
    return launch_face_sv<SCHEME, 0>(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
  if (ph.visc_order == 6)
    return launch_face_sv<SCHEME, 6>(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
  return launch_face_sv<SCHEME, 4>(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
}

// ------------------------------------------------------------------------------------------------
// batched kernels of the serving loop (see BatchTable): each block walks virtual blocks of all the
// bucket's solves and runs the standalone body with the solve's data, block index and grid size
// ------------------------------------------------------------------------------------------------
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

template <bool MIXED>
__global__ void __launch_bounds__(128) kb_prim(const BatchTable* __restrict__ t) {
  FL_BATCH_LOOP(BK_PRIM)
  if (S.steps > 0) k_prim_bc_body<MIXED>(S.U, S.W, S.W32, S.g, S.ph, S.bc, S.ctl, bid, gdim);
  FL_BATCH_END
}

__global__ void __launch_bounds__(kDtBlock) kb_dtp(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_DTP)
  if (step < S.steps) k_dt_partial_body(S.W, S.g, S.ph, S.partial, bid, gdim);
  FL_BATCH_END
}

__global__ void __launch_bounds__(kDtBlock) kb_dtf(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_DTF)
  if (step < S.steps) k_dt_final_body(S.partial, S.nparts, S.ph, S.ctl, nullptr, 1, S.t_end, bid, gdim);
  FL_BATCH_END
}

__global__ void __launch_bounds__(256) kb_grad(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_GRAD)
  if (step < S.steps) k_grad_body<4>(S.W, S.G, S.g, bid, gdim);
  FL_BATCH_END
}

template <int D, int SCHEME, int VORD>
__global__ void __launch_bounds__(128) kb_face(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_FACE0 + D)
  if (step < S.steps)
    k_face_body<D, SCHEME, VORD>(S.W, S.G, S.R, S.FB[D], S.g, S.ph, D > 0, S.seg[D], bid, gdim);
  FL_BATCH_END
}

template <int D>
__global__ void __launch_bounds__(256) kb_seam(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_SEAM0 + D)
  if (step < S.steps) k_face_seam_body<D, false>(S.FB[D], S.R, S.g, D > 0, S.seg[D], bid, gdim);
  FL_BATCH_END
}

template <bool MIXED>
__global__ void __launch_bounds__(128) kb_stage_prim(const BatchTable* __restrict__ t, int stage, int step) {
  FL_BATCH_LOOP(BK_STAGEP)
  if (step < S.steps)
    k_stage_prim_body<MIXED>(stage, S.U, stage == 1 ? S.U : S.A, S.R, stage == 3 ? S.U : S.A, S.W,
                             S.W32, S.g, S.ph, S.ctl, S.t_end, bid, gdim);
  FL_BATCH_END
}

template <bool MIXED>
__global__ void __launch_bounds__(256) kb_halo(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_HALO)
  if (step < S.steps) {
    const long long total = (long long)S.g.p[0] * S.g.p[1] * S.g.p[2] -
                            (long long)S.g.n[0] * S.g.n[1] * S.g.n[2];
    k_halo_prim_body<MIXED>(S.W, S.W32, S.g, S.ph, S.bc, S.ctl, total, bid, gdim);
  }
  FL_BATCH_END
}

__global__ void __launch_bounds__(256) kb_stage(const BatchTable* __restrict__ t, int step) {
  FL_BATCH_LOOP(BK_STAGE)
  if (step < S.steps) k_stage_body(3, S.U, S.A, S.R, S.U, S.W, S.g, S.ph, S.ctl, S.t_end, 0.0, bid, gdim);
  FL_BATCH_END
}

// blocks of a batched launch: as many as fit the GPU at once (each walks virtual blocks)
template <class K>
int batch_grid(K kernel, int block, size_t smem = 0) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

template <int SCHEME, int VORD>
cudaError_t launch_batch_faces(const BatchTable* dev, int step, cudaStream_t st) {
  static const int g0 = batch_grid(kb_face<0, SCHEME, VORD>, 128);
  static const int g1 = batch_grid(kb_face<1, SCHEME, VORD>, 128);
  static const int g2 = batch_grid(kb_face<2, SCHEME, VORD>, 128);
  static const int gs = batch_grid(kb_seam<0>, 256);
  (kb_face<0, SCHEME, VORD><<<g0, 128, 0, st>>>(dev, step), ++t_launches);
  (kb_seam<0><<<gs, 256, 0, st>>>(dev, step), ++t_launches);
  (kb_face<1, SCHEME, VORD><<<g1, 128, 0, st>>>(dev, step), ++t_launches);
  (kb_seam<1><<<gs, 256, 0, st>>>(dev, step), ++t_launches);
  (kb_face<2, SCHEME, VORD><<<g2, 128, 0, st>>>(dev, step), ++t_launches);
  (kb_seam<2><<<gs, 256, 0, st>>>(dev, step), ++t_launches);
  return cudaGetLastError();
}

}  // namespace

void batch_plan(BatchTable& t, bool mixed) {
  auto ceil_div = [](long long a, long long b) { return (a + b - 1) / b; };
  for (int k = 0; k < BK_COUNT; ++k) t.prefix[k][0] = 0;
  for (int i = 0; i < t.nslots; ++i) {
    BatchSlot& S = t.slot[i];
    const Geo& g = S.g;
    for (int k = 0; k < BK_COUNT; ++k) S.vgrid[k][0] = S.vgrid[k][1] = S.vgrid[k][2] = 1;
    auto set = [&](int k, long long x, long long y = 1, long long z = 1) {
      S.vgrid[k][0] = (int)x;
      S.vgrid[k][1] = (int)y;
      S.vgrid[k][2] = (int)z;
    };
    const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long npad = (long long)g.p[0] * g.p[1] * g.p[2];
    set(BK_PRIM, ceil_div(g.p[0], 128), std::min(g.p[1], 65535), std::min(g.p[2], 65535));
    set(BK_DTP, S.nparts > 0 ? S.nparts : 0);
    set(BK_DTF, 1);
    const bool visc = S.ph.visc != FLUID_VISC_NONE;
    long long gt = 1;
    for (int a = 0; a < 3; ++a) gt *= g.n[a] + (a < g.ndim ? 4 : 0);   // order-4 stencils, both paths
    set(BK_GRAD, visc ? ceil_div(gt, 256) : 0);
    for (int D = 0; D < 3; ++D) {
      const long long lines = (long long)g.n[D == 0 ? 1 : 0] * g.n[D == 2 ? 1 : 2];
      if (D >= g.ndim) {
        set(BK_FACE0 + D, 0);
        set(BK_SEAM0 + D, 0);
        continue;
      }
      if (mixed) {
        if (D == 0) set(BK_FACE0, ceil_div(g.n[0], 31), ceil_div(lines, 4));
        else set(BK_FACE0 + D, ceil_div(g.n[0], 32), ceil_div(g.n[D], kMixedTileCells), g.n[D == 1 ? 2 : 1]);
        set(BK_SEAM0 + D, 0);
      } else {
        const long long nseg = ceil_div(g.n[D], S.seg[D]);
        set(BK_FACE0 + D, ceil_div(lines * nseg, 128));
        set(BK_SEAM0 + D, S.FB[D] ? ceil_div(lines * (nseg - 1), 256) : 0);
      }
    }
    set(BK_STAGEP, ceil_div(g.n[0], 128), std::min((g.n[1] + 1) / 2, 65535), std::min(g.n[2], 65535));
    set(BK_HALO, ceil_div(npad - nint, 256));
    set(BK_STAGE, ceil_div(nint, 256));
    for (int k = 0; k < BK_COUNT; ++k)
      t.prefix[k][i + 1] = t.prefix[k][i] + (long long)S.vgrid[k][0] * S.vgrid[k][1] * S.vgrid[k][2];
  }
}

cudaError_t launch_batch_chunk(const BatchTable* dev, int chunk, bool mixed, int weno, bool visc,
                               cudaStream_t st) {
  static const int gp = batch_grid(kb_prim<false>, 128), gpm = batch_grid(kb_prim<true>, 128);
  static const int gd = batch_grid(kb_dtp, kDtBlock), gf = batch_grid(kb_dtf, kDtBlock);
  static const int gg = batch_grid(kb_grad, 256);
  static const int gsp = batch_grid(kb_stage_prim<false>, 128), gspm = batch_grid(kb_stage_prim<true>, 128);
  static const int gh = batch_grid(kb_halo<false>, 256), ghm = batch_grid(kb_halo<true>, 256);
  static const int gs = batch_grid(kb_stage, 256);
  cudaError_t e;
  if (mixed) (kb_prim<true><<<gpm, 128, 0, st>>>(dev), ++t_launches);
  else (kb_prim<false><<<gp, 128, 0, st>>>(dev), ++t_launches);
  for (int k = 0; k < chunk; ++k) {
    if (mixed) {
      if ((e = launch_batch_mixed(dev, BMX_DTP, 0, k, st)) != cudaSuccess) return e;
    } else {
      (kb_dtp<<<gd, kDtBlock, 0, st>>>(dev, k), ++t_launches);
    }
    (kb_dtf<<<gf, kDtBlock, 0, st>>>(dev, k), ++t_launches);
    for (int stage = 1; stage <= 3; ++stage) {
      if (mixed) {
        if (visc && (e = launch_batch_mixed(dev, BMX_GRAD, 0, k, st)) != cudaSuccess) return e;
        for (int D = 0; D < 3; ++D)
          if ((e = launch_batch_mixed_faces(dev, D, k, weno, visc, st)) != cudaSuccess) return e;
      } else {
        if (visc) (kb_grad<<<gg, 256, 0, st>>>(dev, k), ++t_launches);
        if (weno == FLUID_WENO_JS)
          e = visc ? launch_batch_faces<FLUID_WENO_JS, 4>(dev, k, st) : launch_batch_faces<FLUID_WENO_JS, 0>(dev, k, st);
        else
          e = visc ? launch_batch_faces<FLUID_WENO_Z, 4>(dev, k, st) : launch_batch_faces<FLUID_WENO_Z, 0>(dev, k, st);
        if (e != cudaSuccess) return e;
      }
      if (stage < 3 || k + 1 < chunk) {
        if (mixed) {
          (kb_stage_prim<true><<<gspm, 128, 0, st>>>(dev, stage, k), ++t_launches);
          (kb_halo<true><<<ghm, 256, 0, st>>>(dev, k), ++t_launches);
        } else {
          (kb_stage_prim<false><<<gsp, 128, 0, st>>>(dev, stage, k), ++t_launches);
          (kb_halo<false><<<gh, 256, 0, st>>>(dev, k), ++t_launches);
        }
      } else {
        (kb_stage<<<gs, 256, 0, st>>>(dev, k), ++t_launches);
      }
    }
  }
  return cudaGetLastError();
}

double* seam_buffer(int D, const Geo& g, int seg, SeamBuf fb) {
  const long long lines = (long long)g.n[D == 0 ? 1 : 0] * g.n[D == 2 ? 1 : 2];
  const long long nseg = (g.n[D] + seg - 1) / seg;
  return (fb.p != nullptr && nseg > 1 && lines * nseg <= fb.cap) ? fb.p : nullptr;
}

cudaError_t launch_face_seam(int D, const double* FB, double* R, const Geo& g, int accumulate,
                             int seg, bool fused, cudaStream_t st) {
  const long long lines = (long long)g.n[D == 0 ? 1 : 0] * g.n[D == 2 ? 1 : 2];
  const long long items = lines * ((g.n[D] + seg - 1) / seg - 1);
  const int grid = grid_for(items, 256);
  if (D == 0) {
    if (fused) (k_face_seam<0, true><<<grid, 256, 0, st>>>(FB, R, g, accumulate, seg), ++t_launches);
    else (k_face_seam<0, false><<<grid, 256, 0, st>>>(FB, R, g, accumulate, seg), ++t_launches);
  } else if (D == 1) {
    if (fused) (k_face_seam<1, true><<<grid, 256, 0, st>>>(FB, R, g, accumulate, seg), ++t_launches);
    else (k_face_seam<1, false><<<grid, 256, 0, st>>>(FB, R, g, accumulate, seg), ++t_launches);
  } else {
    if (fused) (k_face_seam<2, true><<<grid, 256, 0, st>>>(FB, R, g, accumulate, seg), ++t_launches);
    else (k_face_seam<2, false><<<grid, 256, 0, st>>>(FB, R, g, accumulate, seg), ++t_launches);
  }
  return cudaGetLastError();
}

void face_shape(int D, const Geo& g, int& block, int& seg, int& grid) {
  const int A1 = (D == 0) ? 1 : 0;
  const int A2 = (D == 2) ? 1 : 2;
  const long long lines = (long long)g.n[A1] * g.n[A2];
  if (block <= 0) block = 128;
  if (seg <= 0) {
    // longest segment (fewest redundant faces) that still gives >= 4 blocks of 128 per SM, down
    // to 8 cells; 4 cells only where segments of 8 would leave SMs without a block (small 2-D
    // grids such as the 512 x 128 boundary layer: there segments of 4 take 40 % less time than 8,
    // while on TGV 64^3, which 8 already spreads over every SM, they take 14 % more).  The result
    // does not depend on the choice.
    seg = 64;
    auto threads = [&](int sg) { return lines * ((g.n[D] + sg - 1) / sg); };
    while (seg > 8 && threads(seg) < 152LL * 4 * 128) seg >>= 1;
    if (seg == 8 && threads(8) < 152LL * 128) seg = 4;
  }
  grid = grid_for(lines * ((g.n[D] + seg - 1) / seg), block);
}

cudaError_t launch_prim_bc(const double* U, double* W, float* W32, const Geo& g, const Phys& ph,
                           const BC& bc, Ctl* ctl, cudaStream_t st) {
  // a padded row in nb near-equal chunks of whole warps, at most 256 threads each
  const int nb = (g.p[0] + 255) / 256;
  const int block = ((g.p[0] + nb - 1) / nb + 31) / 32 * 32;
  const dim3 grid((g.p[0] + block - 1) / block, g.p[1] < 65535 ? g.p[1] : 65535,
                  g.p[2] < 65535 ? g.p[2] : 65535);
  if (W32) (k_prim_bc<true><<<grid, block, 0, st>>>(U, W, W32, g, ph, bc, ctl), ++t_launches);
  else (k_prim_bc<false><<<grid, block, 0, st>>>(U, W, W32, g, ph, bc, ctl), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_grad(const double* W, double* G, const Geo& g, const Phys& ph, cudaStream_t st) {
  const int m = ph.visc_order == 6 ? 3 : 2;
  long long total = 1;
  for (int a = 0; a < 3; ++a) total *= g.n[a] + (a < g.ndim ? 2 * m : 0);
  if (m == 3) (k_grad<6><<<grid_for(total, 256), 256, 0, st>>>(W, G, g), ++t_launches);
  else (k_grad<4><<<grid_for(total, 256), 256, 0, st>>>(W, G, g), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_face(int D, const double* W, const double* G, double* R, const Geo& g,
                        const Phys& ph, int accumulate, int block, int seg, SeamBuf fb,
                        cudaStream_t st) {
  if (ph.weno == FLUID_TENO6A)
    return launch_face_teno(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
  if (ph.weno == FLUID_WENO_JS)
    return launch_face_s<FLUID_WENO_JS>(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
  return launch_face_s<FLUID_WENO_Z>(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
}

long long seam_capacity(const Geo& g) {
  long long cap = 0;
  for (int D = 0; D < g.ndim; ++D) {
    const long long lines = (long long)g.n[D == 0 ? 1 : 0] * g.n[D == 2 ? 1 : 2];
    const long long items = lines * ((g.n[D] + kSeamMinSeg - 1) / kSeamMinSeg);
    if (items > cap) cap = items;
  }
  return cap;
}

cudaError_t launch_source(double* R, const double* W, const Geo& g, const Phys& ph, cudaStream_t st) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  (k_source<<<grid_for(total, 256), 256, 0, st>>>(R, W, g, ph), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_stage(int stage, const double* Un, const double* Us, const double* R, double* Ud,
                         const double* W, const Geo& g, const Phys& ph, Ctl* ctl, double t_end,
                         cudaStream_t st, double dt_arg) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  (k_stage<<<grid_for(total, 256), 256, 0, st>>>(stage, Un, Us, R, Ud, W, g, ph, ctl, t_end, dt_arg), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_stage_prim(int stage, const double* Un, const double* Us, const double* R,
                              double* Ud, double* W, float* W32, const Geo& g, const Phys& ph,
                              const BC& bc, Ctl* ctl, double t_end, cudaStream_t st) {
  // interior rows in nb near-equal chunks of whole warps, at most 256 threads each
  const int nb = (g.n[0] + 255) / 256;
  const int block = ((g.n[0] + nb - 1) / nb + 31) / 32 * 32;
  const int j2 = (g.n[1] + 1) / 2;                                     // row pairs
  const dim3 grid((g.n[0] + block - 1) / block, j2 < 65535 ? j2 : 65535, g.n[2] < 65535 ? g.n[2] : 65535);
  if (W32) (k_stage_prim<true><<<grid, block, 0, st>>>(stage, Un, Us, R, Ud, W, W32, g, ph, ctl, t_end), ++t_launches);
  else (k_stage_prim<false><<<grid, block, 0, st>>>(stage, Un, Us, R, Ud, W, W32, g, ph, ctl, t_end), ++t_launches);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_halo_prim(W, W32, g, ph, bc, ctl, st);
}

cudaError_t launch_halo_prim(double* W, float* W32, const Geo& g, const Phys& ph, const BC& bc, Ctl* ctl,
                             cudaStream_t st) {
  const long long total = (long long)g.p[0] * g.p[1] * g.p[2] - (long long)g.n[0] * g.n[1] * g.n[2];
  if (total <= 0) return cudaSuccess;
  if (W32) (k_halo_prim<true><<<grid_for(total, 256), 256, 0, st>>>(W, W32, g, ph, bc, ctl, total), ++t_launches);
  else (k_halo_prim<false><<<grid_for(total, 256), 256, 0, st>>>(W, W32, g, ph, bc, ctl, total), ++t_launches);
  return cudaGetLastError();
}

size_t halo_count(const Geo& g, int A) {
  size_t cnt = 5 * 3;
  for (int b = 0; b < 3; ++b)
    if (b != A) cnt *= (size_t)(b < A ? g.p[b] : g.n[b]);
  return cnt;
}

cudaError_t launch_halo_copy(double* U, double* buf, const Geo& g, int A, int side, bool unpack,
                             cudaStream_t st) {
  const long long total = (long long)halo_count(g, A);
  (k_halo_copy<<<grid_for(total, 256), 256, 0, st>>>(U, buf, g, A, side, unpack ? 1 : 0, total),
   ++t_launches);
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
  (k_dt_partial<<<nparts, kDtBlock, 0, st>>>(W, g, ph, partial), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_dt_final(const double* partial, int nparts, const Phys& ph, Ctl* ctl,
                            double* dt_out, int clip_to_ctl, double t_end, cudaStream_t st) {
  (k_dt_final<<<1, kDtBlock, 0, st>>>(partial, ph.dt_fixed > 0.0 ? 0 : nparts, ph, ctl, dt_out,
                                     clip_to_ctl, t_end), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_prim_to_cons(const double* W, double* U, int ncell, const Phys& ph,
                                cudaStream_t st) {
  (k_prim_to_cons<<<grid_for(ncell, 256), 256, 0, st>>>(W, U, ncell, ph), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_wall_velocity(const double* phi, double* vw, const double* xc, int p, int h,
                                 int begin, int count, double amp, double two_pi_kappa,
                                 cudaStream_t st) {
  (k_wall_velocity<<<grid_for(p, 128), 128, 0, st>>>(phi, vw, xc, p, h, begin, count, amp,
                                                    two_pi_kappa), ++t_launches);
  return cudaGetLastError();
}

}  // namespace fl
