// Discrete adjoint (vector-Jacobian product) of the FP64 right-hand side and of the wall heat-flux
// loss.  Given a state X and a cotangent mu of R(X) on the interior cells, the kernels below form
// (dR/dX)^T mu and (dR/dphi)^T mu (phi: porous-wall parameters) in gather form -- every value is
// summed in a fixed order, so the result does not depend on scheduling:
//   k_adj_face<D>     one thread per segment of faces along a grid line: per face the face-flux
//                     cotangent from the two adjacent cells, then the reverse of HLLC, of the ten
//                     WENO5 reconstructions (weights included; the two values reconstructed in one
//                     cell share its indicator set) and of the dissipative flux; the contributions
//                     to the primitives of the six stencil cells (and to the four tangential-
//                     gradient cells: the four cotangents of the face's interpolated tangential
//                     gradients) go to per-face slots
//   k_adj_gather<D>   one thread per cell: sum of the slots of the faces whose stencil contains it
//                     (the tangential-gradient cotangents times the cell's interpolation weight)
//   k_adj_grad        reverse of the centre velocity gradients
//   k_adj_bc<a>       reverse of the halo passes, z then y then x; one thread owns a boundary
//                     column (both sides, all layers), so contributions to a source cell never race
//   k_adj_prim        reverse of the conservative -> primitive conversion on interior cells
//   k_adj_phi         porous-wall parameters: d v_w / d phi_i = (A / phi0) sin(2 pi kappa x_i)
#include <cuda_runtime.h>

#include "adjoint_math.cuh"
#include "fluid_internal.cuh"

namespace fl {

namespace {

int grid_for(long long work, int block) {
  long long b = (work + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 152LL * 64) b = 152LL * 64;
  return (int)b;
}

constexpr int kSlots = 6;     // stencil cells a-2 .. a+3 of face a+1/2
constexpr int kGSlots = 4;    // viscous stencil cells a-1 .. a+2
constexpr int kGComp = 4;     // tangential gradient components read by one face direction

__device__ __forceinline__ int stride_of(const Geo& g, int d) { return d == 0 ? 1 : (d == 1 ? g.sy : g.sz); }

// threads per block of k_adj_face (its WENO gradients sit in shared memory): one warp, so that a
// launch of a few blocks per SM spreads evenly (the registers allow eight warps per SM)
constexpr int kAdjBlock = 32;
constexpr int kAdjWarpsPerSM = 8;

// One thread marches a segment of faces a+1/2 (a = cfirst .. clast) of one grid line along D; the
// step to target cell x (x = cfirst .. clast + 1) forms both WENO5 values of x with their gradients
// from one indicator set (weno5_vjp_cell): the right-biased value at x-1/2, which completes face
// x-1/2, and the left-biased value at x+1/2, which waits for the next step.  The segment's first
// cell forms only its left-biased value and the cell after its last face only its right-biased one,
// so every value is computed once per segment and the result does not depend on the segment length
// except through these two ends.  Face x-1/2 then takes the reverse HLLC and dissipative flux and
// writes its contributions to the six stencil cells (and four tangential-gradient cells) to its
// per-face slots.
template <int D, int SCHEME, bool VISC>
__global__ void __launch_bounds__(kAdjBlock) k_adj_face(const double* __restrict__ W,
                                                  const double* __restrict__ G,
                                                  const double* __restrict__ mu,
                                                  double* __restrict__ CW, double* __restrict__ CG,
                                                  Geo g, Phys ph, int seg) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const int n1 = g.n[A1], n2 = g.n[A2], nd = g.n[D];
  const int nf = nd + 1;                         // faces a + 1/2, a = h - 1 .. h + nd - 1
  const int nseg = (nf + seg - 1) / seg;
  const long long total = (long long)n1 * n2 * nseg;
  const int s = stride_of(g, D);
  const int nc = g.ncell;
  const double eps4 = 4.0 * ph.eps;
  // gradients of the reconstructions: [x & 1] the left-biased value of target cell x (read at the
  // next step), [2] the right-biased value of the current step
  __shared__ double sJ[3][25][kAdjBlock];
  const int tid = threadIdx.x;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    // consecutive threads take consecutive lines (consecutive x for D = y, z)
    const int i1 = (int)(t % n1);
    const long long rr = t / n1;
    const int i2 = (int)(rr % n2);
    const int sg = (int)(rr / n2);
    const int cfirst = g.h[D] - 1 + sg * seg;
    const int clast = g.h[D] - 1 + min((sg + 1) * seg, nf) - 1;
    int c[3];
    c[A1] = i1 + g.h[A1];
    c[A2] = i2 + g.h[A2];
    c[D] = cfirst;
    int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    double wl[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int x = cfirst; x <= clast + 1; ++x, cell += s) {
      const bool up = x <= clast, dn = x > cfirst;
      double q[5][5];                            // cells x-2 .. x+2
#pragma unroll
      for (int v = 0; v < 5; ++v)
#pragma unroll
        for (int o = 0; o < 5; ++o) q[v][o] = __ldg(W + v * nc + cell + (o - 2) * s);
      double wn[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, wr[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double Ju[5], Jd[5];
        weno5_vjp_cell<SCHEME>(q[v], eps4, up, dn, wn[v], Ju, wr[v], Jd);
        if (up) {
#pragma unroll
          for (int k = 0; k < 5; ++k) sJ[x & 1][v * 5 + k][tid] = Ju[k];
        }
        if (dn) {
#pragma unroll
          for (int k = 0; k < 5; ++k) sJ[2][v * 5 + k][tid] = Jd[k];
        }
      }
      if (dn) {
        // face a + 1/2 between cells a = x - 1 and x
        const int a = x - 1;
        const int fcell = cell - s;
        const int af = a - (g.h[D] - 1);
        // face-flux cotangent: R_a = -(F_{a+1/2} - F_{a-1/2}) / dx_a
        double gF[5];
        const bool inL = af > 0, inR = af < nd;
        const double iL = inL ? g.idx[D][a] : 0.0, iR = inR ? g.idx[D][a + 1] : 0.0;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const double mL = inL ? mu[v * nc + fcell] : 0.0;
          const double mR = inR ? mu[v * nc + cell] : 0.0;
          gF[v] = mR * iR - mL * iL;
        }
        double gwl[5], gwr[5];
        hllc_vjp<D>(wl, wr, ph, gF, gwl, gwr);
        // slots k = 0 .. 5 are cells a-2 .. a+3; the left value's stencil is a-2 .. a+2, the
        // right value's a-1 .. a+3
        const int pl = (x - 1) & 1;
        double gcell[6][kSlots];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          gcell[v][0] = gwl[v] * sJ[pl][v * 5][tid];
#pragma unroll
          for (int k = 1; k < 5; ++k)
            gcell[v][k] = fma(gwl[v], sJ[pl][v * 5 + k][tid], gwr[v] * sJ[2][v * 5 + k - 1][tid]);
          gcell[v][5] = gwr[v] * sJ[2][v * 5 + 4][tid];
        }
#pragma unroll
        for (int k = 0; k < kSlots; ++k) gcell[5][k] = 0.0;
        if (VISC) {
          double vel[3][4], T[4], gd[3][4], gb[3][4];
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            vel[0][o] = q[1][o];
            vel[1][o] = q[2][o];
            vel[2][o] = q[3][o];
            T[o] = __ldg(W + 5 * nc + fcell + (o - 1) * s);
          }
#pragma unroll
          for (int b = 0; b < 3; ++b) {
#pragma unroll
            for (int o = 0; o < 4; ++o) {
              gd[b][o] = 0.0;
              gb[b][o] = 0.0;
            }
            if (b == D || b >= g.ndim) continue;
            const double* pd = G + (D * 3 + b) * nc + fcell;
            const double* pb = G + (b * 3 + b) * nc + fcell;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
              gd[b][o] = __ldg(pd + (o - 1) * s);
              gb[b][o] = __ldg(pb + (o - 1) * s);
            }
          }
          const double gFd[4] = {-gF[1], -gF[2], -gF[3], -gF[4]};
          double gvel[3][4], gT[4], gGD[3], gGB[3];
          visc_face_vjp<D>(vel, T, gd, gb, g.ndim, g.mf[D][a], ph, gFd, gvel, gT, gGD, gGB);
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            gcell[1][1 + o] += gvel[0][o];
            gcell[2][1 + o] += gvel[1][o];
            gcell[3][1 + o] += gvel[2][o];
            gcell[5][1 + o] += gT[o];
          }
          CG[0 * nc + fcell] = gGD[A1];
          CG[1 * nc + fcell] = gGB[A1];
          CG[2 * nc + fcell] = gGD[A2];
          CG[3 * nc + fcell] = gGB[A2];
        }
#pragma unroll
        for (int k = 0; k < kSlots; ++k)
#pragma unroll
          for (int v = 0; v < 6; ++v) CW[(k * 6 + v) * nc + fcell] = gcell[v][k];
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) wl[v] = wn[v];
    }
  }
}

// gW (and gG) += contributions of the faces along D whose stencils contain the cell
template <int D, bool VISC>
__global__ void k_adj_gather(const double* __restrict__ CW, const double* __restrict__ CG,
                             double* __restrict__ gW, double* __restrict__ gG, Geo g) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const int n1 = g.n[A1], n2 = g.n[A2], pd = g.p[D];
  const long long total = (long long)n1 * n2 * pd;
  const int s = stride_of(g, D);
  const int nc = g.ncell;
  const int amin = g.h[D] - 1, amax = g.h[D] + g.n[D] - 1;   // faces a + 1/2
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int x, i1, i2;                               // consecutive threads take consecutive x
    if (D == 0) {
      x = (int)(t % pd);
      const long long r = t / pd;
      i1 = (int)(r % n1);
      i2 = (int)(r / n1);
    } else {
      i1 = (int)(t % n1);
      const long long r = t / n1;
      x = (int)(r % pd);
      i2 = (int)(r / pd);
    }
    int c[3];
    c[A1] = i1 + g.h[A1];
    c[A2] = i2 + g.h[A2];
    c[D] = x;
    const int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    double acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      const int a = x + 2 - k;                     // face whose slot k is this cell
      if (a < amin || a > amax) continue;
      const int fcell = cell + (a - x) * s;
#pragma unroll
      for (int v = 0; v < 6; ++v) acc[v] += CW[(k * 6 + v) * nc + fcell];
    }
#pragma unroll
    for (int v = 0; v < 6; ++v) gW[v * nc + cell] += acc[v];
    if (VISC) {
      // face a's four cotangents of its interpolated tangential gradients, times the weight of
      // this cell (stencil point k of a-1 .. a+2) in the interpolation (-1, 9, 9, -1) / 16
      double ag[kGComp] = {0, 0, 0, 0};
#pragma unroll
      for (int k = 0; k < kGSlots; ++k) {
        const int a = x + 1 - k;
        if (a < amin || a > amax) continue;
        const int fcell = cell + (a - x) * s;
        const double wk = (k == 0 || k == 3) ? -k16th : 9.0 * k16th;
#pragma unroll
        for (int m = 0; m < kGComp; ++m) ag[m] = fma(wk, CG[m * nc + fcell], ag[m]);
      }
      // components: (D, A1), (A1, A1), (D, A2), (A2, A2) of d u_c / d x_b
      if (A1 < g.ndim) {
        gG[(D * 3 + A1) * nc + cell] += ag[0];
        gG[(A1 * 3 + A1) * nc + cell] += ag[1];
      }
      if (A2 < g.ndim) {
        gG[(D * 3 + A2) * nc + cell] += ag[2];
        gG[(A2 * 3 + A2) * nc + cell] += ag[3];
      }
    }
  }
}

// reverse of G[c*3+b](y) = ((u_c(y-2b) - u_c(y+2b)) + 8 (u_c(y+b) - u_c(y-b))) / 12 * mc_b(y)
__global__ void k_adj_grad(const double* __restrict__ gG, double* __restrict__ gW, Geo g) {
  const int total = g.ncell;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < total; cell += gridDim.x * blockDim.x) {
    int x[3];
    x[0] = cell % g.p[0];
    const int r = cell / g.p[0];
    x[1] = r % g.p[1];
    x[2] = r / g.p[1];
    for (int b = 0; b < g.ndim; ++b) {
      const int s = stride_of(g, b);
      const int lo = g.h[b], hi = g.h[b] + g.n[b];     // G along b lives on b-interior cells
      const int offs[4] = {2, -2, -1, 1};              // y = x + o b
      const double coef[4] = {1.0, -1.0, 8.0, -8.0};
      for (int comp = 0; comp < 3; ++comp) {
        double acc = 0.0;
        for (int m = 0; m < 4; ++m) {
          const int yb = x[b] + offs[m];
          if (yb < lo || yb >= hi) continue;
          const int y = cell + offs[m] * s;
          acc += coef[m] * g.mc[b][yb] * gG[(comp * 3 + b) * g.ncell + y];
        }
        gW[(1 + comp) * g.ncell + cell] += acc * kTwelfth;
      }
    }
  }
}

__global__ void k_adj_source(const double* __restrict__ mu, double* __restrict__ gW, Geo g, Phys ph) {
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int i = t % g.n[0];
    const int r = t / g.n[0];
    const int c = (i + g.h[0]) + (r % g.n[1] + g.h[1]) * g.sy + (r / g.n[1] + g.h[2]) * g.sz;
    const double m4 = mu[4 * nc + c];
    gW[1 * nc + c] += ph.f[0] * m4;
    gW[2 * nc + c] += ph.f[1] * m4;
    gW[3 * nc + c] += ph.f[2] * m4;
  }
}

__device__ __forceinline__ int bc_src(int kind, int side, int a, int n, int h) {
  if (kind == FLUID_BC_PERIODIC) return side == 0 ? a + n : a - n;
  if (kind == FLUID_BC_ZERO_GRADIENT) return side == 0 ? h : h + n - 1;
  return side == 0 ? 2 * h - 1 - a : 2 * (h + n) - 1 - a;
}

// reverse of the halo pass of axis A: columns over (axes < A: padded, axes > A: interior).  Per side
// all loads of the column's layers come first (ghost cotangents, source primitives, source
// cotangents), then the layers' contributions are added in layer order, as the halo pass wrote
// them (a zero-gradient side adds all layers to one source cell, in the same order).
template <int A>
__global__ void k_adj_bc(const double* __restrict__ W, double* __restrict__ gW,
                         double* __restrict__ gvw_col, Geo g, Phys ph, BC bc) {
  constexpr int H = FLUID_HALO;
  int lo[3], ext[3];
  for (int b = 0; b < 3; ++b) {
    if (b < A) { lo[b] = 0; ext[b] = g.p[b]; }
    else { lo[b] = g.h[b]; ext[b] = g.n[b]; }
  }
  ext[A] = 1;
  const int total = ext[0] * ext[1] * ext[2];
  const int nc = g.ncell;
  const int s = stride_of(g, A);
  const int n = g.n[A];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int c[3];
    c[0] = lo[0] + t % ext[0];
    const int r = t / ext[0];
    c[1] = lo[1] + r % ext[1];
    c[2] = lo[2] + r / ext[1];
    c[A] = 0;
    const int base = c[0] + c[1] * g.sy + c[2] * g.sz;
    double gvw_sum = 0.0;
    for (int side = 0; side < 2; ++side) {
      const int kind = bc.kind[A][side];
      if (kind == FLUID_BC_INFLOW) continue;            // fixed values: no dependence
      const bool copy = kind == FLUID_BC_PERIODIC || kind == FLUID_BC_ZERO_GRADIENT;
      const bool one_source = kind == FLUID_BC_ZERO_GRADIENT;
      int gc[H], sc[H];
      double gg[H][6], w[H][6], gs[H][6];
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int gi = side == 0 ? H - 1 - m : H + n + m;
        gc[m] = base + gi * s;
        sc[m] = base + bc_src(kind, side, gi, n, H) * s;
      }
#pragma unroll
      for (int m = 0; m < H; ++m)
#pragma unroll
        for (int v = 0; v < 6; ++v) {
          gg[m][v] = gW[v * nc + gc[m]];
          w[m][v] = copy ? 0.0 : W[v * nc + sc[m]];
          gs[m][v] = gW[v * nc + sc[m]];
        }
#pragma unroll
      for (int m = 0; m < H; ++m) {
        double gw[6];
        if (copy) {
#pragma unroll
          for (int v = 0; v < 6; ++v) gw[v] = gg[m][v];
        } else {
          double gvw = 0.0;
          wall_map_vjp(w[m], kind, bc.Tw[A][side], A, ph, gg[m], gw, &gvw);
          gvw_sum += gvw;
        }
        const int k = one_source ? 0 : m;
#pragma unroll
        for (int v = 0; v < 6; ++v) gs[k][v] += gw[v];
      }
#pragma unroll
      for (int m = 0; m < H; ++m)
#pragma unroll
        for (int v = 0; v < 6; ++v) {
          if (m == 0 || !one_source) gW[v * nc + sc[m]] = gs[m][v];
          gW[v * nc + gc[m]] = 0.0;
        }
    }
    if (gvw_col && bc.porous_axis == A) {
      // column index over the two tangential axes (t1 fastest)
      const int t1 = bc.porous_t1, t2 = 3 - A - t1;
      gvw_col[c[t2] * g.p[t1] + c[t1]] += gvw_sum;
    }
  }
}

__global__ void k_adj_prim(const double* __restrict__ U, const double* __restrict__ gW,
                           double* __restrict__ gU, Geo g, Phys ph) {
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int i = t % g.n[0];
    const int r = t / g.n[0];
    const int c = (i + g.h[0]) + (r % g.n[1] + g.h[1]) * g.sy + (r / g.n[1] + g.h[2]) * g.sz;
    double u[5], gw[6], gu[5];
    for (int v = 0; v < 5; ++v) u[v] = U[v * nc + c];
    for (int v = 0; v < 6; ++v) gw[v] = gW[v * nc + c];
    prim_vjp(u, ph, gw, gu);
    for (int v = 0; v < 5; ++v) gU[v * nc + c] = gu[v];
  }
}

// gphi_i += sum over the t2 index of gvw_col(t1 = h + begin + i) * (A/phi0) sin(2 pi kappa x_i)
__global__ void k_adj_phi(const double* __restrict__ gvw_col, const double* __restrict__ xc,
                          double* __restrict__ gphi, int p_t1, int h_t1, int ext_t2, int begin,
                          int count, double amp, double two_pi_kappa) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const int a = h_t1 + begin + i;
    double s = 0.0;
    for (int k = 0; k < ext_t2; ++k) s += gvw_col[k * p_t1 + a];
    gphi[i] += s * amp * sin(two_pi_kappa * xc[a]);
  }
}

// wall heat flux q = -lambda(T_w) dT/dn through the mirrored halo (closed form of the normal
// stencil): side 0: dn = (54 T_h - 2 T_{h+1} - 52 T_w) / 24 * mf; side 1 with the mirror image.
// One thread per wall cell: J partial (q * face area) and, optionally, dJ/dT of the two cells.
__global__ void k_wall_loss(const double* __restrict__ W, double* __restrict__ part,
                            double* __restrict__ gT2, Geo g, Phys ph, int A, int side, double Tw,
                            double lam_w) {
  const int t1 = A == 0 ? 1 : 0, t2 = 3 - A - t1;
  const int n1 = g.n[t1], n2 = g.n[t2];
  const int total = n1 * n2;
  const int s = stride_of(g, A);
  const int a0 = side == 0 ? g.h[A] : g.h[A] + g.n[A] - 1;     // wall-adjacent interior cell
  const int a1 = side == 0 ? a0 + 1 : a0 - 1;
  const int af = side == 0 ? g.h[A] - 1 : g.h[A] + g.n[A] - 1;  // the wall face af + 1/2
  const double mf = g.mf[A][af];
  const double sgn = side == 0 ? 1.0 : -1.0;                     // derivative along +axis
  double acc = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int c[3];
    c[t1] = g.h[t1] + t % n1;
    c[t2] = g.h[t2] + t / n1;
    c[A] = a0;
    const int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    const double T0 = W[5 * g.ncell + cell], T1 = W[5 * g.ncell + cell + (a1 - a0) * s];
    const double area = (t1 < g.ndim ? g.dx[t1][c[t1]] : 1.0) * (t2 < g.ndim ? g.dx[t2][c[t2]] : 1.0);
    const double dn = sgn * (54.0 * T0 - 2.0 * T1 - 52.0 * Tw) * k24th * mf;
    acc += -lam_w * dn * area;
    if (gT2) {
      gT2[2 * t] = -lam_w * sgn * 54.0 * k24th * mf * area;
      gT2[2 * t + 1] = lam_w * sgn * 2.0 * k24th * mf * area;
    }
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// Per wall cell of face (A, side): q_w = -lambda(T_w) dT/dn and tau_w = mu(T_w) du_t1/dn by the
// fourth-order face stencil through the mirrored ghost cells (T_g = 2 T_w - T, u_g = -u), which in
// the two wall-adjacent interior cells reads (54 f_0 - 2 f_1 - 52 f_w) / 24 * (d index / dn)
__global__ void k_wall_fluxes(const double* __restrict__ W, double* __restrict__ qw,
                              double* __restrict__ tw, Geo g, int A, int side, double Tw,
                              double mu_w, double lam_w) {
  const int t1 = A == 0 ? 1 : 0, t2 = 3 - A - t1;
  const int n1 = g.n[t1], n2 = g.n[t2];
  const int total = n1 * n2;
  const int s = stride_of(g, A);
  const int a0 = side == 0 ? g.h[A] : g.h[A] + g.n[A] - 1;
  const int a1 = side == 0 ? a0 + 1 : a0 - 1;
  const int af = side == 0 ? g.h[A] - 1 : g.h[A] + g.n[A] - 1;
  const double m = (side == 0 ? 1.0 : -1.0) * k24th * g.mf[A][af];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int c[3];
    c[t1] = g.h[t1] + t % n1;
    c[t2] = g.h[t2] + t / n1;
    c[A] = a0;
    const int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    const int cell1 = cell + (a1 - a0) * s;
    const double T0 = W[5 * g.ncell + cell], T1 = W[5 * g.ncell + cell1];
    const double u0 = W[(1 + t1) * g.ncell + cell], u1 = W[(1 + t1) * g.ncell + cell1];
    if (qw) qw[t] = -lam_w * ((54.0 * T0 - 2.0 * T1 - 52.0 * Tw) * m);
    if (tw) tw[t] = mu_w * ((54.0 * u0 - 2.0 * u1) * m);
  }
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

// dJ/dU of the two wall-adjacent cells of every wall column (other interior cells stay zero)
__global__ void k_wall_loss_grad(const double* __restrict__ U, const double* __restrict__ gT2,
                                 double* __restrict__ dJdU, Geo g, Phys ph, int A, int side) {
  const int t1 = A == 0 ? 1 : 0, t2 = 3 - A - t1;
  const int n1 = g.n[t1], n2 = g.n[t2];
  const int total = n1 * n2;
  const int s = stride_of(g, A);
  const int a0 = side == 0 ? g.h[A] : g.h[A] + g.n[A] - 1;
  const int a1 = side == 0 ? a0 + 1 : a0 - 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int c[3];
    c[t1] = g.h[t1] + t % n1;
    c[t2] = g.h[t2] + t / n1;
    c[A] = a0;
    const int cell0 = c[0] + c[1] * g.sy + c[2] * g.sz;
    for (int k = 0; k < 2; ++k) {
      const int cell = cell0 + (k == 0 ? 0 : (a1 - a0) * s);
      double u[5], gw[6] = {0, 0, 0, 0, 0, gT2[2 * t + k]}, gu[5];
      for (int v = 0; v < 5; ++v) u[v] = U[v * g.ncell + cell];
      prim_vjp(u, ph, gw, gu);
      for (int v = 0; v < 5; ++v) dJdU[v * g.ncell + cell] += gu[v];
    }
  }
}

// out = c0 x0 + c1 x1 + c2 x2 + c3 x3 on interior cells (x_k may be null when c_k == 0)
__global__ void k_lincomb(double* out, double c0, const double* x0, double c1, const double* x1,
                          double c2, const double* x2, double c3, const double* x3, Geo g) {
  const int total = g.n[0] * g.n[1] * g.n[2];
  const int nc = g.ncell;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int i = t % g.n[0];
    const int r = t / g.n[0];
    const int c = (i + g.h[0]) + (r % g.n[1] + g.h[1]) * g.sy + (r / g.n[1] + g.h[2]) * g.sz;
    for (int v = 0; v < 5; ++v) {
      const int o = v * nc + c;
      double s = c0 * x0[o];
      if (x1) s += c1 * x1[o];
      if (x2) s += c2 * x2[o];
      if (x3) s += c3 * x3[o];
      out[o] = s;
    }
  }
}

// Segment length of k_adj_face for lines of nf faces: the one that minimises the modelled time,
// (waves of resident threads) x (faces per thread) x (FP64 work per face).  A segment of L faces
// forms 2 + 2 (L - 1) reconstructions' worth of WENO5 work as L + 1 cells (its two ends one value
// each, the cells between two values from one indicator set, about 1.65 times one value), against
// 2 L for faces taken one by one; the rest of a face (reverse HLLC, dissipative flux, slots) is
// about 0.64 of two values.  Resident threads: 8 warps per SM (the kernel's registers).
int adj_segment(long long lines, int nf) {
  const long long resident = 152LL * kAdjWarpsPerSM * 32;
  int best = 1;
  double best_t = 0.0;
  for (int L = 1; L <= 16; L *= 2) {
    const long long threads = lines * ((nf + L - 1) / L);
    const long long waves = (threads + resident - 1) / resident;
    const double per_face = 1.28 + (2.0 + 1.65 * (L - 1)) / L;
    const double t = (double)waves * L * per_face;
    if (L == 1 || t < best_t) {
      best = L;
      best_t = t;
    }
  }
  return best;
}

template <int D, int SCHEME, bool VISC>
cudaError_t adj_face_t(const double* W, const double* G, const double* mu, double* CW, double* CG,
                       const Geo& g, const Phys& ph, cudaStream_t st) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const long long lines = (long long)g.n[A1] * g.n[A2];
  const int nf = g.n[D] + 1;
  const int seg = adj_segment(lines, nf);
  const long long total = lines * ((nf + seg - 1) / seg);
  (k_adj_face<D, SCHEME, VISC><<<grid_for(total, kAdjBlock), kAdjBlock, 0, st>>>(W, G, mu, CW, CG, g, ph, seg), ++t_launches);
  return cudaGetLastError();
}

template <int SCHEME, bool VISC>
cudaError_t adj_dir(int D, const double* W, const double* G, const double* mu, double* CW,
                    double* CG, double* gW, double* gG, const Geo& g, const Phys& ph,
                    cudaStream_t st) {
  cudaError_t e;
  const long long ncol = (D == 0 ? (long long)g.n[1] * g.n[2]
                                 : (D == 1 ? (long long)g.n[0] * g.n[2] : (long long)g.n[0] * g.n[1]));
  const long long tg = ncol * g.p[D];
  if (D == 0) {
    if ((e = adj_face_t<0, SCHEME, VISC>(W, G, mu, CW, CG, g, ph, st)) != cudaSuccess) return e;
    (k_adj_gather<0, VISC><<<grid_for(tg, 256), 256, 0, st>>>(CW, CG, gW, gG, g), ++t_launches);
  } else if (D == 1) {
    if ((e = adj_face_t<1, SCHEME, VISC>(W, G, mu, CW, CG, g, ph, st)) != cudaSuccess) return e;
    (k_adj_gather<1, VISC><<<grid_for(tg, 256), 256, 0, st>>>(CW, CG, gW, gG, g), ++t_launches);
  } else {
    if ((e = adj_face_t<2, SCHEME, VISC>(W, G, mu, CW, CG, g, ph, st)) != cudaSuccess) return e;
    (k_adj_gather<2, VISC><<<grid_for(tg, 256), 256, 0, st>>>(CW, CG, gW, gG, g), ++t_launches);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adj_faces(const double* W, const double* G, const double* mu, double* CW,
                             double* CG, double* gW, double* gG, const Geo& g, const Phys& ph,
                             cudaStream_t st) {
  const bool visc = ph.visc != FLUID_VISC_NONE;
  for (int D = 0; D < g.ndim; ++D) {
    cudaError_t e;
    if (ph.weno == FLUID_WENO_JS)
      e = visc ? adj_dir<FLUID_WENO_JS, true>(D, W, G, mu, CW, CG, gW, gG, g, ph, st)
               : adj_dir<FLUID_WENO_JS, false>(D, W, G, mu, CW, CG, gW, gG, g, ph, st);
    else
      e = visc ? adj_dir<FLUID_WENO_Z, true>(D, W, G, mu, CW, CG, gW, gG, g, ph, st)
               : adj_dir<FLUID_WENO_Z, false>(D, W, G, mu, CW, CG, gW, gG, g, ph, st);
    if (e != cudaSuccess) return e;
  }
  if (visc) {
    (k_adj_grad<<<grid_for(g.ncell, 256), 256, 0, st>>>(gG, gW, g), ++t_launches);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_adj_source(const double* mu, double* gW, const Geo& g, const Phys& ph, cudaStream_t st) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  (k_adj_source<<<grid_for(total, 256), 256, 0, st>>>(mu, gW, g, ph), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_adj_bc(const double* W, double* gW, double* gvw_col, const Geo& g,
                          const Phys& ph, const BC& bc, cudaStream_t st) {
  for (int A = g.ndim - 1; A >= 0; --A) {
    long long cols = 1;
    for (int b = 0; b < 3; ++b)
      if (b != A) cols *= b < A ? g.p[b] : g.n[b];
    const int grid = grid_for(cols, 128);
    if (A == 0) (k_adj_bc<0><<<grid, 128, 0, st>>>(W, gW, gvw_col, g, ph, bc), ++t_launches);
    else if (A == 1) (k_adj_bc<1><<<grid, 128, 0, st>>>(W, gW, gvw_col, g, ph, bc), ++t_launches);
    else (k_adj_bc<2><<<grid, 128, 0, st>>>(W, gW, gvw_col, g, ph, bc), ++t_launches);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_adj_prim(const double* U, const double* gW, double* gU, const Geo& g,
                            const Phys& ph, cudaStream_t st) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  (k_adj_prim<<<grid_for(total, 256), 256, 0, st>>>(U, gW, gU, g, ph), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_adj_phi(const double* gvw_col, const double* xc, double* gphi, int p_t1,
                           int h_t1, int ext_t2, int begin, int count, double amp,
                           double two_pi_kappa, cudaStream_t st) {
  (k_adj_phi<<<grid_for(count, 128), 128, 0, st>>>(gvw_col, xc, gphi, p_t1, h_t1, ext_t2, begin,
                                                   count, amp, two_pi_kappa), ++t_launches);
  return cudaGetLastError();
}

int wall_loss_parts(const Geo& g, int A) {
  const int t1 = A == 0 ? 1 : 0, t2 = 3 - A - t1;
  long long total = (long long)g.n[t1] * g.n[t2];
  long long b = (total + 255) / 256;
  if (b > 1024) b = 1024;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_wall_loss(const double* W, double* part, int nparts, double* J, double* gT2,
                             const Geo& g, const Phys& ph, int A, int side, double Tw,
                             cudaStream_t st) {
  const double lam_w = viscosity(Tw, ph) * ph.lam_fac;
  (k_wall_loss<<<nparts, 256, 0, st>>>(W, part, gT2, g, ph, A, side, Tw, lam_w), ++t_launches);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  (k_sum_parts<<<1, 32, 0, st>>>(part, nparts, J), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_wall_fluxes(const double* W, double* qw, double* tw, const Geo& g, const Phys& ph,
                               int A, int side, double Tw, cudaStream_t st) {
  const int t1 = A == 0 ? 1 : 0, t2 = 3 - A - t1;
  const long long total = (long long)g.n[t1] * g.n[t2];
  const double mu_w = viscosity(Tw, ph);
  (k_wall_fluxes<<<grid_for(total, 128), 128, 0, st>>>(W, qw, tw, g, A, side, Tw, mu_w, mu_w * ph.lam_fac),
   ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_wall_loss_grad(const double* U, const double* gT2, double* dJdU, const Geo& g,
                                  const Phys& ph, int A, int side, cudaStream_t st) {
  const int t1 = A == 0 ? 1 : 0, t2 = 3 - A - t1;
  const long long total = (long long)g.n[t1] * g.n[t2];
  (k_wall_loss_grad<<<grid_for(total, 128), 128, 0, st>>>(U, gT2, dJdU, g, ph, A, side), ++t_launches);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(double* out, double c0, const double* x0, double c1, const double* x1,
                           double c2, const double* x2, double c3, const double* x3, const Geo& g,
                           cudaStream_t st) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  (k_lincomb<<<grid_for(total, 256), 256, 0, st>>>(out, c0, x0, c1, x1, c2, x2, c3, x3, g), ++t_launches);
  return cudaGetLastError();
}

}  // namespace fl
