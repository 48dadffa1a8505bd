// Host-compiled check of the hand-written reverse-mode functions in adjoint_math.cuh against
// central finite differences of the forward functions in flux_math.cuh (the same code the kernels
// run).  For random inputs x, cotangents g and directions d it compares <g, J d> (finite
// difference) with <J^T g, d> and prints the worst relative difference per function.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_2406_19494_gb300/csrc/adjoint_math.cuh"

using namespace fl;

static std::mt19937_64 rng(12345);
static double U(double a, double b) { return std::uniform_real_distribution<double>(a, b)(rng); }

static Phys make_phys(int visc) {
  Phys ph{};
  ph.gamma = 1.4; ph.gm1 = 0.4; ph.igm1 = 1.0 / 0.4; ph.R = 1.3; ph.iR = 1.0 / 1.3;
  ph.cp = 1.4 * 1.3 / 0.4; ph.Pr = 0.72; ph.lam_fac = ph.cp / ph.Pr;
  ph.mu_ref = 0.03; ph.T_ref = 1.1; ph.iT_ref = 1.0 / 1.1; ph.visc_exp = 0.7; ph.suth_S = 0.4;
  ph.visc = visc;
  return ph;
}

static double relerr(double fd, double ad) { return std::fabs(fd - ad) / (std::fabs(fd) + std::fabs(ad) + 1e-300); }

template <int S>
static double check_weno(double eps) {
  double worst = 0.0;
  for (int t = 0; t < 400; ++t) {
    double q[5], d[5], gq[5];
    const double sc = std::pow(10.0, U(-3, 1));
    for (int k = 0; k < 5; ++k) { q[k] = U(-1, 1) * sc + (t % 3 == 0 ? 5.0 : 0.0); d[k] = U(-1, 1); }
    const double g = U(-1, 1);
    weno5_vjp<S>(q, eps, g, gq);
    // fourth-order central difference: the weights are steep at small scales
    auto f = [&](double hh) {
      double x[5];
      for (int k = 0; k < 5; ++k) x[k] = q[k] + hh * d[k];
      return weno5<S>(x[0], x[1], x[2], x[3], x[4], eps);
    };
    const double h = 1e-4 * sc;
    const double fd = g * (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h);
    double ad = 0.0;
    for (int k = 0; k < 5; ++k) ad += gq[k] * d[k];
    worst = std::fmax(worst, relerr(fd, ad));
  }
  return worst;
}

// Both values of a cell from weno5_vjp_cell: each value against the forward weno5 (the
// right-biased one is the forward on the mirrored stencil) and each gradient against finite
// differences of that value.
template <int S>
static double check_weno_cell(double eps) {
  double worst = 0.0;
  for (int t = 0; t < 400; ++t) {
    double q[5], d[5], Ju[5], Jd[5], vu = 0.0, vd = 0.0;
    const double sc = std::pow(10.0, U(-3, 1));
    for (int k = 0; k < 5; ++k) { q[k] = U(-1, 1) * sc + (t % 3 == 0 ? 5.0 : 0.0); d[k] = U(-1, 1); }
    weno5_vjp_cell<S>(q, 4.0 * eps, true, true, vu, Ju, vd, Jd);
    auto fu = [&](double hh) {
      double x[5];
      for (int k = 0; k < 5; ++k) x[k] = q[k] + hh * d[k];
      return weno5<S>(x[0], x[1], x[2], x[3], x[4], eps);
    };
    auto fd = [&](double hh) {
      double x[5];
      for (int k = 0; k < 5; ++k) x[k] = q[k] + hh * d[k];
      return weno5<S>(x[4], x[3], x[2], x[1], x[0], eps);
    };
    const double scale = std::fabs(q[2]) + sc;
    worst = std::fmax(worst, std::fabs(vu - fu(0.0)) / scale);
    worst = std::fmax(worst, std::fabs(vd - fd(0.0)) / scale);
    const double h = 1e-4 * sc;
    const double du = (-fu(2 * h) + 8 * fu(h) - 8 * fu(-h) + fu(-2 * h)) / (12 * h);
    const double dd = (-fd(2 * h) + 8 * fd(h) - 8 * fd(-h) + fd(-2 * h)) / (12 * h);
    double au = 0.0, ad = 0.0, su = 0.0, sd = 0.0;
    for (int k = 0; k < 5; ++k) { au += Ju[k] * d[k]; ad += Jd[k] * d[k]; su += Ju[k]; sd += Jd[k]; }
    worst = std::fmax(worst, relerr(du, au));
    worst = std::fmax(worst, relerr(dd, ad));
    worst = std::fmax(worst, std::fmax(std::fabs(su - 1.0), std::fabs(sd - 1.0)));
  }
  return worst;
}

template <int D>
static double check_hllc(int regime) {
  const Phys ph = make_phys(FLUID_VISC_NONE);
  double worst = 0.0;
  for (int t = 0; t < 400; ++t) {
    double wl[5], wr[5];
    const double base = regime == 0 ? 0.0 : (regime == 1 ? 2.5 : -2.5);   // subsonic / supersonic
    wl[0] = U(0.5, 2); wr[0] = U(0.5, 2); wl[4] = U(0.5, 2); wr[4] = U(0.5, 2);
    for (int c = 1; c < 4; ++c) { wl[c] = U(-0.8, 0.8); wr[c] = U(-0.8, 0.8); }
    wl[1 + D] += base; wr[1 + D] += base;
    double dl[5], dr[5], g[5], gwl[5], gwr[5];
    for (int v = 0; v < 5; ++v) { dl[v] = U(-1, 1); dr[v] = U(-1, 1); g[v] = U(-1, 1); }
    hllc_vjp<D>(wl, wr, ph, g, gwl, gwr);
    const double h = 1e-6;
    double lp[5], lm[5], rp[5], rm[5], Fp[5], Fm[5];
    for (int v = 0; v < 5; ++v) { lp[v] = wl[v] + h * dl[v]; lm[v] = wl[v] - h * dl[v]; rp[v] = wr[v] + h * dr[v]; rm[v] = wr[v] - h * dr[v]; }
    hllc<D>(lp, rp, ph, Fp);
    hllc<D>(lm, rm, ph, Fm);
    double fd = 0.0, ad = 0.0;
    for (int v = 0; v < 5; ++v) {
      fd += g[v] * (Fp[v] - Fm[v]) / (2 * h);
      ad += gwl[v] * dl[v] + gwr[v] * dr[v];
    }
    worst = std::fmax(worst, relerr(fd, ad));
  }
  return worst;
}

template <int D>
static double check_visc(int visc, int ndim) {
  const Phys ph = make_phys(visc);
  double worst = 0.0;
  for (int t = 0; t < 300; ++t) {
    double vel[3][4], T[4], gd[3][4], gb[3][4], dv[3][4], dT[4], dgd[3][4], dgb[3][4];
    for (int k = 0; k < 4; ++k) {
      T[k] = U(0.8, 1.6); dT[k] = U(-1, 1);
      for (int c = 0; c < 3; ++c) {
        vel[c][k] = U(-1, 1); dv[c][k] = U(-1, 1);
        gd[c][k] = U(-2, 2); gb[c][k] = U(-2, 2); dgd[c][k] = U(-1, 1); dgb[c][k] = U(-1, 1);
      }
    }
    const double mfa = U(5, 20);
    double g[4], gvel[3][4], gT[4], gGD[3], gGB[3], ggd[3][4], ggb[3][4];
    for (int k = 0; k < 4; ++k) g[k] = U(-1, 1);
    visc_face_vjp<D>(vel, T, gd, gb, ndim, mfa, ph, g, gvel, gT, gGD, gGB);
    // the stencil cells' share: the interpolation weights (-1, 9, 9, -1) / 16
    const double wi[4] = {-1.0 / 16.0, 9.0 / 16.0, 9.0 / 16.0, -1.0 / 16.0};
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) {
        ggd[c][k] = gGD[c] * wi[k];
        ggb[c][k] = gGB[c] * wi[k];
      }
    const double h = 1e-6;
    double vp[3][4], vm[3][4], Tp[4], Tm[4], gdp[3][4], gdm[3][4], gbp[3][4], gbm[3][4];
    for (int k = 0; k < 4; ++k) {
      Tp[k] = T[k] + h * dT[k]; Tm[k] = T[k] - h * dT[k];
      for (int c = 0; c < 3; ++c) {
        vp[c][k] = vel[c][k] + h * dv[c][k]; vm[c][k] = vel[c][k] - h * dv[c][k];
        gdp[c][k] = gd[c][k] + h * dgd[c][k]; gdm[c][k] = gd[c][k] - h * dgd[c][k];
        gbp[c][k] = gb[c][k] + h * dgb[c][k]; gbm[c][k] = gb[c][k] - h * dgb[c][k];
      }
    }
    double Fp[4], Fm[4];
    visc_face<D>(vp, Tp, gdp, gbp, ndim, mfa, ph, Fp);
    visc_face<D>(vm, Tm, gdm, gbm, ndim, mfa, ph, Fm);
    double fd = 0.0, ad = 0.0;
    for (int v = 0; v < 4; ++v) fd += g[v] * (Fp[v] - Fm[v]) / (2 * h);
    for (int k = 0; k < 4; ++k) {
      ad += gT[k] * dT[k];
      for (int c = 0; c < 3; ++c) ad += gvel[c][k] * dv[c][k] + ggd[c][k] * dgd[c][k] + ggb[c][k] * dgb[c][k];
    }
    worst = std::fmax(worst, relerr(fd, ad));
  }
  return worst;
}

static double check_prim() {
  const Phys ph = make_phys(FLUID_VISC_NONE);
  double worst = 0.0;
  for (int t = 0; t < 300; ++t) {
    double u[5], d[5], g[6], gu[5];
    u[0] = U(0.5, 2); u[1] = U(-1, 1); u[2] = U(-1, 1); u[3] = U(-1, 1); u[4] = U(3, 6);
    for (int v = 0; v < 5; ++v) d[v] = U(-1, 1);
    for (int v = 0; v < 6; ++v) g[v] = U(-1, 1);
    prim_vjp(u, ph, g, gu);
    const double h = 1e-6;
    double up[5], um[5], wp[6], wm[6];
    for (int v = 0; v < 5; ++v) { up[v] = u[v] + h * d[v]; um[v] = u[v] - h * d[v]; }
    prim_from_cons(up, ph, wp);
    prim_from_cons(um, ph, wm);
    double fd = 0.0, ad = 0.0;
    for (int v = 0; v < 6; ++v) fd += g[v] * (wp[v] - wm[v]) / (2 * h);
    for (int v = 0; v < 5; ++v) ad += gu[v] * d[v];
    worst = std::fmax(worst, relerr(fd, ad));
  }
  return worst;
}

static double check_wall(int kind) {
  const Phys ph = make_phys(FLUID_VISC_NONE);
  double worst = 0.0;
  for (int t = 0; t < 300; ++t) {
    double w[6], d[6], g[6], gw[6], gvw;
    w[0] = U(0.5, 2); w[1] = U(-1, 1); w[2] = U(-1, 1); w[3] = U(-1, 1); w[4] = U(0.5, 2); w[5] = U(0.5, 1.5);
    for (int v = 0; v < 6; ++v) { d[v] = U(-1, 1); g[v] = U(-1, 1); }
    const double vw = U(-0.1, 0.1), dvw = U(-1, 1), Tw = 2.0;
    const int a = t % 3;
    wall_map_vjp(w, kind, Tw, a, ph, g, gw, &gvw);
    const double h = 1e-6;
    double wp[6], wm[6];
    for (int v = 0; v < 6; ++v) { wp[v] = w[v] + h * d[v]; wm[v] = w[v] - h * d[v]; }
    wall_map_prim(wp, kind, Tw, vw + h * dvw, a, ph);
    wall_map_prim(wm, kind, Tw, vw - h * dvw, a, ph);
    double fd = 0.0, ad = gvw * dvw;
    for (int v = 0; v < 6; ++v) { fd += g[v] * (wp[v] - wm[v]) / (2 * h); ad += gw[v] * d[v]; }
    worst = std::fmax(worst, relerr(fd, ad));
  }
  return worst;
}

int main() {
  std::printf("weno5_js %.3e\n", check_weno<FLUID_WENO_JS>(1e-6));
  std::printf("weno5_z %.3e\n", check_weno<FLUID_WENO_Z>(1e-40));
  std::printf("weno5_cell_js %.3e\n", check_weno_cell<FLUID_WENO_JS>(1e-6));
  std::printf("weno5_cell_z %.3e\n", check_weno_cell<FLUID_WENO_Z>(1e-40));
  for (int r = 0; r < 3; ++r) {
    std::printf("hllc_x_regime%d %.3e\n", r, check_hllc<0>(r));
    std::printf("hllc_y_regime%d %.3e\n", r, check_hllc<1>(r));
    std::printf("hllc_z_regime%d %.3e\n", r, check_hllc<2>(r));
  }
  std::printf("visc_x_power_3d %.3e\n", check_visc<0>(FLUID_VISC_POWER, 3));
  std::printf("visc_y_sutherland_3d %.3e\n", check_visc<1>(FLUID_VISC_SUTHERLAND, 3));
  std::printf("visc_z_constant_3d %.3e\n", check_visc<2>(FLUID_VISC_CONSTANT, 3));
  std::printf("visc_y_sutherland_2d %.3e\n", check_visc<1>(FLUID_VISC_SUTHERLAND, 2));
  std::printf("prim %.3e\n", check_prim());
  std::printf("wall_isothermal %.3e\n", check_wall(FLUID_BC_WALL));
  std::printf("wall_porous %.3e\n", check_wall(FLUID_BC_POROUS));
  std::printf("wall_adiabatic %.3e\n", check_wall(FLUID_BC_ADIABATIC));
  return 0;
}
