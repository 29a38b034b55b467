// Strict arithmetic policy: every formula evaluated as the paper prints it, left to right,
// one IEEE binary64 operation per +, -, *, / and sqrt.  The translation unit that
// instantiates it is compiled with -fmad=false, so nothing is contracted into an FMA and
// the results are those of a literal evaluation, bit for bit.
#pragma once

#include "wt_device.cuh"

namespace wt {

struct StrictMath {
  static constexpr bool kStrict = true;
  static constexpr bool kRoeRows = false;  // the whole Roe matrix per interface (roe)
  // projection v = kProj (L f +- alpha L u) with the stored L = kLScale * L_true
  static constexpr double kProj = 0.5, kLScale = 1.0;
  // the reconstruction is evaluated in one piece (weno_flags)
  static constexpr bool kSplitWeno = false;
  // the projections are taken cell by cell, in the order of Eq. (flux_split_lf)
  static constexpr bool kDiffProj = false;
  struct WenoPart {
    double e[4], tau, fh[4];
    bool theta1;
  };
  __device__ __forceinline__ static bool weno_begin(const double*, double, double, double&, WenoPart&) { return true; }
  __device__ __forceinline__ static double weno_finish(const WenoPart&) { return 0.0; }

  // ---- scalar fluxes (Eq. (lin_eq), Eq. (bur_eq))
  __device__ __forceinline__ static double flux_advection(double a, double u) { return a * u; }
  __device__ __forceinline__ static double flux_burgers(double u) { return 0.5 * u * u; }

  // ---- Euler 1D cell (Sec. 4.2): u = m / rho, p = (gamma - 1)(E - rho u^2 / 2),
  //      f = (m, p + m u, (E + p) u), H = (E + p) / rho, sqrt(rho) for Roe's average
  __device__ __forceinline__ static void euler_cell(const double* U, double gamma, double* f, double& u, double& H,
                                                    double& sr, double& p) {
    u = U[1] / U[0];
    p = (gamma - 1.0) * (U[2] - 0.5 * U[0] * u * u);
    f[0] = U[1];
    f[1] = p + U[1] * u;
    f[2] = (U[2] + p) * u;
    H = (U[2] + p) / U[0];
    sr = sqrt(U[0]);
  }

  // euler_cell and the wave speeds of euler_speeds from the same u and p
  __device__ __forceinline__ static void euler_cell_speeds(const double* U, double gamma, double* f, double& u,
                                                           double& H, double& sr, double* lam) {
    double p;
    euler_cell(U, gamma, f, u, H, sr, p);
    const double c = sqrt(gamma * p / U[0]);
    lam[0] = fabs(u - c);
    lam[1] = fabs(u);
    lam[2] = fabs(u + c);
  }

  // |lambda_s| at a cell: (|u - c|, |u|, |u + c|), c = sqrt(gamma p / rho); returns p
  __device__ __forceinline__ static double euler_speeds(const double* U, double gamma, double* lam) {
    double u = U[1] / U[0];
    double p = (gamma - 1.0) * (U[2] - 0.5 * U[0] * u * u);
    double c = sqrt(gamma * p / U[0]);
    lam[0] = fabs(u - c);
    lam[1] = fabs(u);
    lam[2] = fabs(u + c);
    return p;
  }

  // euler_speeds in two parts, with its operations: |u| (keeping u), then |u - c| and |u + c|
  __device__ __forceinline__ static double speed_u(const double* U, double& u, double& ir) {
    u = U[1] / U[0];
    ir = 0.0;
    return fabs(u);
  }
  __device__ __forceinline__ static void speed_c(const double* U, double gamma, double u, double, double& l0,
                                                 double& l2) {
    double p = (gamma - 1.0) * (U[2] - 0.5 * U[0] * u * u);
    double c = sqrt(gamma * p / U[0]);
    l0 = fabs(u - c);
    l2 = fabs(u + c);
  }

  // ---- Roe's mean state between two cells and the left eigenvectors L (row-major 3x3)
  //      of Roe's matrix; rs = (u~, H~, c~) for the right eigenvectors.
  __device__ __forceinline__ static void roe(double sa, double ua, double Ha, double sb, double ub, double Hb,
                                             double gamma, double* L, double* rs) {
    double u = (sa * ua + sb * ub) / (sa + sb);
    double H = (sa * Ha + sb * Hb) / (sa + sb);
    roe_mean(u, H, gamma, L, rs);
  }
  // the eigenvectors from Roe's mean velocity and enthalpy, exactly as roe() forms them
  __device__ __forceinline__ static void roe_mean(double u, double H, double gamma, double* L, double* rs) {
    double c = sqrt((gamma - 1.0) * (H - 0.5 * u * u));
    double b1 = (gamma - 1.0) / (c * c);
    double b2 = 0.5 * u * u * b1;
    L[0] = 0.5 * (b2 + u / c);
    L[1] = -0.5 * (b1 * u + 1.0 / c);
    L[2] = 0.5 * b1;
    L[3] = 1.0 - b2;
    L[4] = b1 * u;
    L[5] = -b1;
    L[6] = 0.5 * (b2 - u / c);
    L[7] = -0.5 * (b1 * u - 1.0 / c);
    L[8] = 0.5 * b1;
    rs[0] = u;
    rs[1] = H;
    rs[2] = c;
  }

  __device__ __forceinline__ static void roe_row(double, double, double, double, double, double, double, int,
                                                 double*, double*) {}

  // ---- Global Lax-Friedrichs splitting of one projected cell (Eq. (flux_split_lf))
  __device__ __forceinline__ static void project3(const double* l, const double* f, const double* U, double alpha,
                                                  double& vp, double& vm) {
    double a = l[0] * f[0];
    double b = l[0] * U[0];
    a = a + l[1] * f[1];
    b = b + l[1] * U[1];
    a = a + l[2] * f[2];
    b = b + l[2] * U[2];
    vp = 0.5 * (a + alpha * b);
    vm = 0.5 * (a - alpha * b);
  }
  __device__ __forceinline__ static void project1(double f, double u, double alpha, double& vp, double& vm) {
    vp = 0.5 * (f + alpha * u);
    vm = 0.5 * (f - alpha * u);
  }
  // the same projections in two parts: (a, b) = (l.f, l.u) before alpha is known, then v+-
  __device__ __forceinline__ static void project3_ab(const double* l, const double* f, const double* U, double& a,
                                                     double& b) {
    a = l[0] * f[0];
    b = l[0] * U[0];
    a = a + l[1] * f[1];
    b = b + l[1] * U[1];
    a = a + l[2] * f[2];
    b = b + l[2] * U[2];
  }
  // the l.u half of project3_ab alone, with the same operations
  __device__ __forceinline__ static double project3_b(const double* l, const double* U) {
    double b = l[0] * U[0];
    b = b + l[1] * U[1];
    b = b + l[2] * U[2];
    return b;
  }
  __device__ __forceinline__ static void project1_ab(double f, double u, double& a, double& b) {
    a = f;
    b = u;
  }
  __device__ __forceinline__ static void project_v(double a, double b, double alpha, double& vp, double& vm) {
    vp = 0.5 * (a + alpha * b);
    vm = 0.5 * (a - alpha * b);
  }
  // one side of project_v: v+ (minus false) or v- (minus true), the same value
  __device__ __forceinline__ static double project_side(double a, double b, double alpha, bool minus) {
    return minus ? 0.5 * (a - alpha * b) : 0.5 * (a + alpha * b);
  }

  // ---- WENO-theta interface value, Eqs. (fh0)-(fh3), (be0_cen)-(be3_cen), (be_res),
  //      (tau_5), (tau_6), (tau_we6), (gam_we6), (om), (fh_nonlinear); q[i] at x_{j-2+i}
  __device__ __forceinline__ static double weno_flags(const double* q, double eps, double alpha_R, bool& restricted,
                                                    bool& theta1) {
    double fh0 = (2.0 * q[0] - 7.0 * q[1] + 11.0 * q[2]) / 6.0;
    double fh1 = (-q[1] + 5.0 * q[2] + 2.0 * q[3]) / 6.0;
    double fh2 = (2.0 * q[2] + 5.0 * q[3] - q[4]) / 6.0;
    double fh3 = (11.0 * q[3] - 7.0 * q[4] + 2.0 * q[5]) / 6.0;
    double x, y;
    x = q[0] - 2.0 * q[1] + q[2];
    y = q[0] - 3.0 * q[1] + 2.0 * q[2];
    double b0 = (13.0 / 12.0) * (x * x) + y * y;
    x = q[1] - 2.0 * q[2] + q[3];
    y = q[3] - q[2];
    double b1 = (13.0 / 12.0) * (x * x) + y * y;
    x = q[2] - 2.0 * q[3] + q[4];
    y = q[2] - q[3];
    double b2 = (13.0 / 12.0) * (x * x) + y * y;
    x = 3.0 * q[2] - 7.0 * q[3] + 5.0 * q[4] - q[5];
    y = 2.0 * q[3] - 3.0 * q[4] + q[5];
    double b3 = (13.0 / 48.0) * (x * x) + y * y;
    x = q[0] - 4.0 * q[1] + 6.0 * q[2] - 4.0 * q[3] + q[4];
    y = -q[1] + 3.0 * q[2] - 3.0 * q[3] + q[4];
    double tau5 = (13.0 / 12.0) * (x * x) + y * y;
    x = -q[0] + 5.0 * q[1] - 10.0 * q[2] + 10.0 * q[3] - 5.0 * q[4] + q[5];
    y = q[0] - 3.0 * q[1] + 2.0 * q[2] + 2.0 * q[3] - 3.0 * q[4] + q[5];
    double tau6 = (13.0 / 12.0) * (x * x) + 0.25 * (y * y);

    double bmax = b0, bmin = b0;
    bmax = (bmax < b1) ? b1 : bmax;
    bmax = (bmax < b2) ? b2 : bmax;
    bmax = (bmax < b3) ? b3 : bmax;
    bmin = (b1 < bmin) ? b1 : bmin;
    bmin = (b2 < bmin) ? b2 : bmin;
    bmin = (b3 < bmin) ? b3 : bmin;
    double ratio = bmax / (eps + bmin);
    restricted = ratio <= alpha_R;
    theta1 = !(tau6 < tau5);
    if (ratio <= alpha_R) {
      b0 = 0.0;
      b1 = 0.0;
      b2 = 0.0;
      b3 = 0.0;
    }
    double tau, g0, g1, g2, g3;
    if (tau6 < tau5) {  // theta = 0
      tau = tau6;
      g0 = (1.0 + 0.0) / 20.0;
      g1 = (3.0 * (3.0 + 0.0)) / 20.0;
      g2 = (3.0 * (3.0 - 0.0)) / 20.0;
      g3 = (1.0 - 0.0) / 20.0;
    } else {  // theta = 1
      tau = tau5;
      g0 = (1.0 + 1.0) / 20.0;
      g1 = (3.0 * (3.0 + 1.0)) / 20.0;
      g2 = (3.0 * (3.0 - 1.0)) / 20.0;
      g3 = (1.0 - 1.0) / 20.0;
    }
    double a0 = g0 * (1.0 + tau / (eps + b0));
    double a1 = g1 * (1.0 + tau / (eps + b1));
    double a2 = g2 * (1.0 + tau / (eps + b2));
    double a3 = g3 * (1.0 + tau / (eps + b3));
    double asum = a0 + a1 + a2 + a3;
    double w0 = a0 / asum, w1 = a1 / asum, w2 = a2 / asum, w3 = a3 / asum;
    return w0 * fh0 + w1 * fh1 + w2 * fh2 + w3 * fh3;
  }

  __device__ __forceinline__ static double weno(const double* q, double eps, double alpha_R) {
    bool r, t;
    return weno_flags(q, eps, alpha_R, r, t);
  }

  // ---- back-projection h = R (F+ + F-) with R = [r_1 r_2 r_3] of Roe's matrix
  __device__ __forceinline__ static void backproject(const double* rs, const double* F, double* h) {
    const double u = rs[0], H = rs[1], c = rs[2];
    // the acoustic pair (fields 0 and 2) first, so that mirrored data give mirrored fluxes
    h[0] = (1.0 * F[0] + 1.0 * F[2]) + 1.0 * F[1];
    h[1] = ((u - c) * F[0] + (u + c) * F[2]) + u * F[1];
    h[2] = ((H - u * c) * F[0] + (H + u * c) * F[2]) + 0.5 * u * u * F[1];
  }

  // ---- Eq. (mod_semi)
  __device__ __forceinline__ static double flux_diff(double hp, double hm, double dx, double) {
    return -(hp - hm) / dx;
  }

  // ---- Eq. (3rd_RK), stage s of uout from u^n, the stage input us and L(us)
  template <int S>
  __device__ __forceinline__ static double rk(double un, double us, double dt, double L) {
    if (S == 0) return un + dt * L;
    if (S == 1) return 0.75 * un + 0.25 * us + 0.25 * dt * L;
    return (1.0 / 3.0) * un + (2.0 / 3.0) * us + (2.0 / 3.0) * dt * L;
  }

  __device__ __forceinline__ static double cfl_dt(double cfl, double dx, double smax) { return cfl * dx / smax; }

  // ================================ 2D Euler (Sec. 4.3) ================================
  // cell: u, v, p, H, sqrt(rho) and both physical fluxes f (x) and g (y)
  __device__ __forceinline__ static void euler2d_cell(const double* U, double gamma, double* f, double* g, double& u,
                                                      double& v, double& H, double& sr) {
    u = U[1] / U[0];
    v = U[2] / U[0];
    const double p = (gamma - 1.0) * (U[3] - 0.5 * U[0] * (u * u + v * v));
    f[0] = U[1];
    f[1] = p + U[1] * u;
    f[2] = U[1] * v;
    f[3] = (U[3] + p) * u;
    g[0] = U[2];
    g[1] = U[2] * u;
    g[2] = p + U[2] * v;
    g[3] = (U[3] + p) * v;
    H = (U[3] + p) / U[0];
    sr = sqrt(U[0]);
  }
  // g of euler2d_cell alone, from the u and v it returned (the same operations)
  __device__ __forceinline__ static void euler2d_gflux(const double* U, double u, double v, double gamma, double* g) {
    const double p = (gamma - 1.0) * (U[3] - 0.5 * U[0] * (u * u + v * v));
    g[0] = U[2];
    g[1] = U[2] * u;
    g[2] = p + U[2] * v;
    g[3] = (U[3] + p) * v;
  }

  // |lambda| in x (u-c, u, u, u+c) and y (v-c, v, v, v+c) and the CFL quantity
  // (|u| + c)/dx + (|v| + c)/dy
  __device__ __forceinline__ static void euler2d_speeds(const double* U, double gamma, double dx, double dy,
                                                        double* lx, double* ly, double& q) {
    const double u = U[1] / U[0];
    const double v = U[2] / U[0];
    const double p = (gamma - 1.0) * (U[3] - 0.5 * U[0] * (u * u + v * v));
    const double c = sqrt(gamma * p / U[0]);
    lx[0] = fabs(u - c);
    lx[1] = fabs(u);
    lx[2] = fabs(u);
    lx[3] = fabs(u + c);
    ly[0] = fabs(v - c);
    ly[1] = fabs(v);
    ly[2] = fabs(v);
    ly[3] = fabs(v + c);
    q = (fabs(u) + c) / dx + (fabs(v) + c) / dy;
  }

  // Roe state (u, v, H, c) and left eigenvectors L (row-major 4x4) of the Roe matrix of f
  // (dir 0) or g (dir 1); fields ordered (w - c, w, shear, w + c), w the normal velocity.
  __device__ __forceinline__ static void roe2d(int dir, double sa, double ua, double va, double Ha, double sb,
                                               double ub, double vb, double Hb, double gamma, double* L, double* rs) {
    const double u = (sa * ua + sb * ub) / (sa + sb);
    const double v = (sa * va + sb * vb) / (sa + sb);
    const double H = (sa * Ha + sb * Hb) / (sa + sb);
    const double q2 = u * u + v * v;
    const double c = sqrt((gamma - 1.0) * (H - 0.5 * q2));
    const double b1 = (gamma - 1.0) / (c * c);
    const double b2 = 0.5 * q2 * b1;
    if (dir == 0) {
      L[0] = 0.5 * (b2 + u / c); L[1] = -0.5 * (b1 * u + 1.0 / c); L[2] = -0.5 * (b1 * v); L[3] = 0.5 * b1;
      L[4] = 1.0 - b2;           L[5] = b1 * u;                    L[6] = b1 * v;           L[7] = -b1;
      L[8] = -v;                 L[9] = 0.0;                       L[10] = 1.0;             L[11] = 0.0;
      L[12] = 0.5 * (b2 - u / c); L[13] = -0.5 * (b1 * u - 1.0 / c); L[14] = -0.5 * (b1 * v); L[15] = 0.5 * b1;
    } else {
      L[0] = 0.5 * (b2 + v / c); L[1] = -0.5 * (b1 * u); L[2] = -0.5 * (b1 * v + 1.0 / c); L[3] = 0.5 * b1;
      L[4] = 1.0 - b2;           L[5] = b1 * u;          L[6] = b1 * v;                    L[7] = -b1;
      L[8] = -u;                 L[9] = 1.0;             L[10] = 0.0;                      L[11] = 0.0;
      L[12] = 0.5 * (b2 - v / c); L[13] = -0.5 * (b1 * u); L[14] = -0.5 * (b1 * v - 1.0 / c); L[15] = 0.5 * b1;
    }
    rs[0] = u;
    rs[1] = v;
    rs[2] = H;
    rs[3] = c;
  }

  // summed density, normal momentum, tangential momentum, energy: the same order in both
  // sweep directions, so that transposed data give transposed fluxes
  __device__ __forceinline__ static void project4(int dir, const double* l, const double* f, const double* U,
                                                  double alpha, double& vp, double& vm) {
    const int n = 1 + dir, t = 2 - dir;
    double a = l[0] * f[0];
    double b = l[0] * U[0];
    a = a + l[n] * f[n];
    b = b + l[n] * U[n];
    a = a + l[t] * f[t];
    b = b + l[t] * U[t];
    a = a + l[3] * f[3];
    b = b + l[3] * U[3];
    vp = 0.5 * (a + alpha * b);
    vm = 0.5 * (a - alpha * b);
  }

  // h = R F with R the right eigenvectors (columns) of Roe's matrix in direction dir
  __device__ __forceinline__ static void backproject2d(int dir, const double* rs, const double* F, double* h) {
    const double u = rs[0], v = rs[1], H = rs[2], c = rs[3];
    const double q2 = u * u + v * v;
    double R[16];
    if (dir == 0) {
      R[0] = 1.0;       R[1] = 1.0;        R[2] = 0.0;  R[3] = 1.0;
      R[4] = u - c;     R[5] = u;          R[6] = 0.0;  R[7] = u + c;
      R[8] = v;         R[9] = v;          R[10] = 1.0; R[11] = v;
      R[12] = H - u * c; R[13] = 0.5 * q2; R[14] = v;   R[15] = H + u * c;
    } else {
      R[0] = 1.0;       R[1] = 1.0;        R[2] = 0.0;  R[3] = 1.0;
      R[4] = u;         R[5] = u;          R[6] = 1.0;  R[7] = u;
      R[8] = v - c;     R[9] = v;          R[10] = 0.0; R[11] = v + c;
      R[12] = H - v * c; R[13] = 0.5 * q2; R[14] = u;   R[15] = H + v * c;
    }
    // the acoustic pair (fields 0 and 3) first, then entropy + shear: mirror-symmetric sums
    for (int r = 0; r < 4; ++r) {
      double x = R[4 * r] * F[0] + R[4 * r + 3] * F[3];
      x = x + (R[4 * r + 1] * F[1] + R[4 * r + 2] * F[2]);
      h[r] = x;
    }
  }

  __device__ __forceinline__ static double add_sweeps(double Lx, double Ly) { return Lx + Ly; }
  // L + (-g q): a source term -g q added to the flux divergence
  __device__ __forceinline__ static double add_source(double L, double g, double q) { return L + (-(g * q)); }
  __device__ __forceinline__ static double cfl_dt_2d(double cfl, double smax) { return cfl / smax; }
};

}  // namespace wt
