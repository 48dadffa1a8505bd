// FP64 face kernels with the paper's channel-flow reconstruction (Sec. 3.1): TENO6-A on the
// primitive variables with the interpolation limiter, the HLLC flux, and the dissipative flux by
// central differences of order 4 or 6 (template VORD; 0 = inviscid).
//
// Interpolation limiter (reading of the paper's "interpolation limiter", its solver's
// positivity-preserving limiting of reconstructed states): a face state with rho <= 0 or p <= 0
// falls back, in all five primitives, to the cell on its side of the face.
//
// One thread marches along a segment of a grid line, as the WENO5 kernel does; each face is
// computed once and serves the two cells that share it (across segments through the seam buffer,
// as in k_face).  The cut-off levels of the TENO-A scale
// sensors depend on single cells, so three of the four a face needs carry over from the previous
// face, as do the right state's three-cell measures (the next left state's) and their factors.  A
// segment starts with the terms the march would have carried there, formed by the same
// operations, so the result is the same for every segment length.
#include <cuda_runtime.h>

#include "fluid_internal.cuh"
#include "teno_math.cuh"

namespace fl {

namespace {

// face flux F^c - F^d at face a+1/2 along D; `cell` is the padded index of cell a, s its stride;
// lev[v][0..2] carry the cut-off levels of cells a-1, a, a+1 and b3[v] the three-cell smoothness
// measures of the left state (see teno::face_states); both advance by one cell
template <int D, int VORD>
__device__ __forceinline__ void face_flux_teno(const double* __restrict__ W, const double* __restrict__ G,
                                               int cell, int s, int a, const Geo& g, const Phys& ph,
                                               double F[5], int lev[5][3], double b3[5][3],
                                               double i3[5][3], double kk[5][2],
                                               const double (*omega)[16]) {
  const int nc = g.ncell;
  double q[5][6];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int o = 0; o < 6; ++o) q[v][o] = __ldg(W + v * nc + cell + (o - 2) * s);
  double wl[5], wr[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    // cells a-2 .. a+3 are q[v][0..5] and d their differences (formed again from the loaded
    // values rather than carried: the same subtractions, so the same bits, and 20 doubles fewer
    // live across faces); the sensor level of cell a+2 is the new one
    const double d[5] = {q[v][1] - q[v][0], q[v][2] - q[v][1], q[v][3] - q[v][2], q[v][4] - q[v][3],
                         q[v][5] - q[v][4]};
    const int l3 = teno::sensor_level(d[3], d[4]);
    const double ct = teno::cutoff_of_level(min(min(lev[v][0], lev[v][1]), min(lev[v][2], l3)));
    teno::face_states(q[v], d, ct, b3[v], i3[v], kk[v], omega, wl[v], wr[v]);
    lev[v][0] = lev[v][1];
    lev[v][1] = lev[v][2];
    lev[v][2] = l3;
  }
  // interpolation limiter
  if (wl[0] <= 0.0 || wl[4] <= 0.0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) wl[v] = q[v][2];
  }
  if (wr[0] <= 0.0 || wr[4] <= 0.0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) wr[v] = q[v][3];
  }
  hllc<D>(wl, wr, ph, F);
  if (VORD) add_visc_face<D, VORD ? VORD : 4>(W, G, cell, s, a, g, ph, q, F);
}

template <int D, int VORD>
__global__ void __launch_bounds__(128) k_face_teno(const double* __restrict__ W,
                                                   const double* __restrict__ G, double* __restrict__ R,
                                                   double* __restrict__ FB, Geo g, Phys ph,
                                                   int accumulate, int seg) {
  constexpr int A1 = (D == 0) ? 1 : 0;
  constexpr int A2 = (D == 2) ? 1 : 2;
  const int n1 = g.n[A1], n2 = g.n[A2], nd = g.n[D];
  const int nseg = (nd + seg - 1) / seg;
  const long long lines = (long long)n1 * n2;
  const long long total = lines * nseg;
  const int s = D == 0 ? 1 : (D == 1 ? g.sy : g.sz);
  const int nc = g.ncell;
  // normalised weights per keep mask, k-major: for each k the 16 masks' weights sit in distinct
  // pairs of banks, so lanes reading different masks do not conflict
  __shared__ double omega[4][16];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) teno::weight_entry(i, omega);
  __syncthreads();
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
    // with the seam buffer a segment after the first starts at the face after its first cell
    // (as in k_face)
    const bool seam = FB != nullptr && sg > 0;
    c[D] = seam ? a0 : a0 - 1;
    int cell = c[0] + c[1] * g.sy + c[2] * g.sz;
    double Fp[5], F[5], b3[5][3], i3[5][3], kk[5][2];
    int lev[5][3];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double* f = W + v * nc + cell;                   // cell a = c[D]
      const double qm2 = __ldg(f - 2 * s), qm1 = __ldg(f - s), q0 = __ldg(f), qp1 = __ldg(f + s),
                   qp2 = __ldg(f + 2 * s);
      // the differences of cells a-2 .. a+2 (a = a0 - 1), and the terms the march carries into
      // the first face formed by the march's own operations (teno::face_states at the face
      // before), so that a segment start continues bit for bit: the sensor levels of cells a-1,
      // a, a+1, K of the stencils centred at a-1, a, a+1, then B centred at a, A centred at a+1
      // and C centred at a-1, with their reciprocal factors
      const double D0 = qm1 - qm2, D1 = q0 - qm1, D2 = qp1 - q0, D3 = qp2 - qp1;
      lev[v][0] = teno::sensor_level(D0, D1);
      lev[v][1] = teno::sensor_level(D1, D2);
      lev[v][2] = teno::sensor_level(D2, D3);
      const double tm = D1 - D0, ta = D2 - D1, tb = D3 - D2;
      const double Km = k1312 * tm * tm, Ka = k1312 * ta * ta, Kb = k1312 * tb * tb;
      const double sB = D1 + D2, sA = fma(-3.0, D2, D3), sC = fma(3.0, D1, -D0);
      b3[v][0] = fma(0.25 * sB, sB, Ka);
      b3[v][1] = fma(0.25 * sA, sA, Kb);
      b3[v][2] = fma(0.25 * sC, sC, Km);
      kk[v][0] = Ka;
      kk[v][1] = Kb;
#pragma unroll
      for (int j = 0; j < 3; ++j) i3[v][j] = teno::rcp6(b3[v][j]);
    }
    face_flux_teno<D, VORD>(W, G, cell, s, c[D], g, ph, Fp, lev, b3, i3, kk, omega);
    if (seam) {
#pragma unroll
      for (int v = 0; v < 5; ++v) FB[v * total + t] = Fp[v];
    }
    for (int a = seam ? a0 + 1 : a0; a < a1; ++a) {
      cell += s;
      face_flux_teno<D, VORD>(W, G, cell, s, a, g, ph, F, lev, b3, i3, kk, omega);
      const double id = g.idx[D][a];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double dF = F[v] - Fp[v];
        double* dst = R + v * nc + cell;
        *dst = accumulate ? fma(-id, dF, *dst) : -id * dF;
        Fp[v] = F[v];
      }
    }
    if (FB != nullptr && sg + 1 < nseg) {
#pragma unroll
      for (int v = 0; v < 5; ++v) FB[(5 + v) * total + t + lines] = Fp[v];
    }
  }
}

template <int D, int VORD>
cudaError_t launch_d(const double* W, const double* G, double* R, const Geo& g, const Phys& ph,
                     int accumulate, int block, int seg, SeamBuf fb, cudaStream_t st) {
  int grid;
  face_shape(D, g, block, seg, grid);
  double* FB = seam_buffer(D, g, seg, fb);
  (k_face_teno<D, VORD><<<grid, block, 0, st>>>(W, G, R, FB, g, ph, accumulate, seg), ++t_launches);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !FB) return e;
  return launch_face_seam(D, FB, R, g, accumulate, seg, true, st);
}

template <int VORD>
cudaError_t launch_v(int D, const double* W, const double* G, double* R, const Geo& g,
                     const Phys& ph, int accumulate, int block, int seg, SeamBuf fb, cudaStream_t st) {
  if (D == 0) return launch_d<0, VORD>(W, G, R, g, ph, accumulate, block, seg, fb, st);
  if (D == 1) return launch_d<1, VORD>(W, G, R, g, ph, accumulate, block, seg, fb, st);
  return launch_d<2, VORD>(W, G, R, g, ph, accumulate, block, seg, fb, st);
}

}  // namespace

cudaError_t launch_face_teno(int D, const double* W, const double* G, double* R, const Geo& g,
                             const Phys& ph, int accumulate, int block, int seg, SeamBuf fb,
                             cudaStream_t st) {
  if (ph.visc == FLUID_VISC_NONE) return launch_v<0>(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
  if (ph.visc_order == 6) return launch_v<6>(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
  return launch_v<4>(D, W, G, R, g, ph, accumulate, block, seg, fb, st);
}

}  // namespace fl
