/*
 * Plain serial reference ("oracle") for the adaptive WENO-theta scheme of
 * Jung & Nguyen, arXiv 1504.00731.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this file.  The CUDA library never links it, and the two
 * share no source: this file has no header and includes nothing from the package.
 *
 * It is slow and literal on purpose:
 *   - every formula is written as the paper prints it, in the paper's order;
 *   - it is built with -O2 -ffp-contract=off, so each +, -, *, / below is exactly
 *     one IEEE-754 binary64 operation, evaluated left to right as C++ groups it;
 *   - it is templated on the scalar type R.  R = double gives the values.  R = Dual
 *     gives forward-mode derivatives of exactly the same map, with every branch
 *     frozen where the value goes (used to check the discrete adjoint).  R = Cnt
 *     counts the arithmetic operations.
 *
 * Readings of passages where the paper is silent or ambiguous are marked "Reading".  One
 * of them fixes the order of two sums the paper does not order: the back-projection adds
 * the acoustic pair of characteristic fields first, and the 2D projection adds the normal
 * momentum before the tangential one in both sweeps, so that mirrored or transposed data
 * give mirrored or transposed results in binary64 too (the symmetry the paper reports for
 * its Rayleigh-Taylor and implosion tests).
 *
 * Pins (tests/test_oracle_pins.py): the printed errors of Table 1, the closed-form
 * solution of the linear limit, the linear identities of Eqs. (fh_5) and (fh_6), the
 * Taylor expansions printed with Eqs. (be0_cen)-(be3_cen), (tau_5) and (tau_6),
 * exactness on quadratics, conservation, mirror and transpose symmetry, Roe's defining
 * property f(b) - f(a) = A(b - a), the gravity source (a uniform state, hydrostatic
 * balance), exact translation (resolution test, composite wave), the characteristic
 * solution of Burgers' equation away from its shock, and the exact Riemann solution
 * (itself pinned by its pressure-function residual, the Rankine-Hugoniot relations and
 * the Riemann invariants) for Sod, Lax, 123 and the early blast waves.  Reflective walls
 * (tests/test_oracle_walls.py): a uniform flow between two walls against the exact Riemann
 * solutions of the mirrored states, conservation of mass and energy on data mirrored about
 * the middle, 2D lines across a wall equal to the 1D run; a build with the normal momentum's
 * sign planted wrong fails all three.  The Lax-Friedrichs constants and the CFL step against
 * the eigenvalues of complex-step flux Jacobians, and advection with a = -2 against the
 * closed form of the linear limit.  The sampled RHS equals the whole RHS cell by cell.
 * Parity unpinned:
 * the solution near discontinuities beyond those monotonicity and convergence bounds
 * (Shu-Osher only by self-convergence), and the value alpha_R = 10 on the seeded Euler
 * workloads (a convention; the paper sets alpha_R per test).
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace wto {

/* ------------------------------------------------------------------------- */
/* Scalar types                                                              */
/* ------------------------------------------------------------------------- */

inline double val(double x) { return x; }

/* Forward-mode dual number: v + d*eps, eps^2 = 0. */
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline double val(const Dual& x) { return x.v; }
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
/* the branch taken by the value decides the derivative (frozen branch) */
inline Dual fabs(Dual a) { return a.v < 0 ? -a : a; }

/* Operation counter: same values as double, counts each arithmetic operation. */
struct OpCount {
  long long add, mul, div, sqrt, cmp;
};
static OpCount g_ops;
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline double val(const Cnt& x) { return x.v; }
inline Cnt operator+(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_ops.mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_ops.div++; return Cnt(a.v / b.v); }
inline Cnt sqrt(Cnt a) { g_ops.sqrt++; return Cnt(std::sqrt(a.v)); }
inline Cnt fabs(Cnt a) { return Cnt(std::fabs(a.v)); }

inline double fabs(double x) { return std::fabs(x); }
inline double sqrt(double x) { return std::sqrt(x); }

inline void count_cmp(double) {}
inline void count_cmp(const Dual&) {}
inline void count_cmp(const Cnt&) { g_ops.cmp++; }

/* a < b and a <= b decided on the values; max / min keep the selected operand
 * (and its derivative).  On exact ties the first operand is kept. */
template <class R> inline bool lt(const R& a, const R& b) { count_cmp(a); return val(a) < val(b); }
template <class R> inline bool le(const R& a, const R& b) { count_cmp(a); return val(a) <= val(b); }
template <class R> inline R rmax(const R& a, const R& b) { return lt(a, b) ? b : a; }
template <class R> inline R rmin(const R& a, const R& b) { return lt(b, a) ? b : a; }
template <class R> inline R sq(const R& a) { return a * a; }

/* ------------------------------------------------------------------------- */
/* Problem description (the oracle's own; mirrored in oracle/__init__.py)    */
/* ------------------------------------------------------------------------- */

enum { FLUX_ADVECTION = 0, FLUX_BURGERS = 1, FLUX_EULER1D = 2, FLUX_EULER2D = 3 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECTIVE = 2 };

struct Problem {
  int32_t flux;      /* FLUX_* */
  int32_t m;         /* components: 1, 1, 3, 4 */
  double gamma;      /* ratio of specific heats (Euler) */
  double adv_speed;  /* a in f = a*u (advection) */
  double eps;        /* epsilon of Eq. (om) and of R(beta) in Eq. (be_res) */
  double alpha_R;    /* threshold of Eq. (be_res) */
  int32_t bc_lo[2], bc_hi[2]; /* per direction x, y */
  double gravity;    /* 2D Euler: g of the source terms -g rho (y momentum) and -g rho v (energy), TEST 6 of Sec. 4.3 */
};

const int G = 3; /* ghost cells per side: the six-point stencil S^6 = {j-2..j+3} (Sec. 2, Remark on flux splitting) */

/* ------------------------------------------------------------------------- */
/* WENO-theta reconstruction at one interface x_{j+1/2}  (Sec. 3)            */
/* ------------------------------------------------------------------------- */

struct RecInfo {
  int theta;       /* 0 or 1, Eq. (tau_we6) */
  int restricted;  /* 1 when Eq. (be_res) set every beta to zero */
};

/* Smoothness indicators of one stencil q[0..5] = values at x_{j-2..j+3}.
 * Eqs. (be0_cen)-(be3_cen): central sub-stencil indicators; beta_3 uses the modified
 * second term, not the hat-beta_3 that the paper sets aside.
 * Eqs. (tau_5), (tau_6): large-stencil indicators of S^5 and S^6. */
template <class R>
void smoothness(const R q[6], R b[4], R* tau5, R* tau6) {
  b[0] = (13.0 / 12.0) * sq(q[0] - 2.0 * q[1] + q[2]) + sq(q[0] - 3.0 * q[1] + 2.0 * q[2]);
  b[1] = (13.0 / 12.0) * sq(q[1] - 2.0 * q[2] + q[3]) + sq(q[3] - q[2]);
  b[2] = (13.0 / 12.0) * sq(q[2] - 2.0 * q[3] + q[4]) + sq(q[2] - q[3]);
  b[3] = (13.0 / 48.0) * sq(3.0 * q[2] - 7.0 * q[3] + 5.0 * q[4] - q[5]) + sq(2.0 * q[3] - 3.0 * q[4] + q[5]);
  *tau5 = (13.0 / 12.0) * sq(q[0] - 4.0 * q[1] + 6.0 * q[2] - 4.0 * q[3] + q[4]) +
          sq(-q[1] + 3.0 * q[2] - 3.0 * q[3] + q[4]);
  *tau6 = (13.0 / 12.0) * sq(-q[0] + 5.0 * q[1] - 10.0 * q[2] + 10.0 * q[3] - 5.0 * q[4] + q[5]) +
          0.25 * sq(q[0] - 3.0 * q[1] + 2.0 * q[2] + 2.0 * q[3] - 3.0 * q[4] + q[5]);
}

/* q[i] is the split flux value at x_{j-2+i}, i = 0..5 (the stencil S^6), biased so that
 * S^5 = {j-2..j+2} is the upwind stencil.  Returns the interface value of Eq. (fh_nonlinear). */
template <class R>
R weno_theta(const R q[6], double eps, double alpha_R, RecInfo* info) {
  /* Eqs. (fh0)-(fh2) and (fh3): third-order values at x_{j+1/2} on S_0..S_3 */
  R fh0 = (2.0 * q[0] - 7.0 * q[1] + 11.0 * q[2]) / 6.0;
  R fh1 = (-q[1] + 5.0 * q[2] + 2.0 * q[3]) / 6.0;
  R fh2 = (2.0 * q[2] + 5.0 * q[3] - q[4]) / 6.0;
  R fh3 = (11.0 * q[3] - 7.0 * q[4] + 2.0 * q[5]) / 6.0;

  /* Eqs. (be0_cen)-(be3_cen), (tau_5), (tau_6) */
  R b0, b1, b2, b3, tau5, tau6;
  {
    R b[4];
    smoothness(q, b, &tau5, &tau6);
    b0 = b[0];
    b1 = b[1];
    b2 = b[2];
    b3 = b[3];
  }

  /* Eq. (be_res): R(beta) = max beta / (eps + min beta); all beta := 0 when R <= alpha_R.
   * Reading: the same eps as in Eq. (om); "<=" as printed. */
  R bmax = rmax(rmax(rmax(b0, b1), b2), b3);
  R bmin = rmin(rmin(rmin(b0, b1), b2), b3);
  R ratio = bmax / (eps + bmin);
  int restricted = le(ratio, R(alpha_R)) ? 1 : 0;
  if (restricted) {
    b0 = R(0.0);
    b1 = R(0.0);
    b2 = R(0.0);
    b3 = R(0.0);
  }

  /* Eq. (tau_we6): (tau, theta) = (tau6, 0) if tau6 < tau5, else (tau5, 1) */
  int theta;
  R tau;
  if (lt(tau6, tau5)) {
    tau = tau6;
    theta = 0;
  } else {
    tau = tau5;
    theta = 1;
  }

  /* Eq. (gam_we6): each gamma is an exact integer over 20, so one rounding */
  const double th = (double)theta;
  const double g0 = (1.0 + th) / 20.0;
  const double g1 = (3.0 * (3.0 + th)) / 20.0;
  const double g2 = (3.0 * (3.0 - th)) / 20.0;
  const double g3 = (1.0 - th) / 20.0;

  /* Eq. (om) */
  R a0 = g0 * (1.0 + tau / (eps + b0));
  R a1 = g1 * (1.0 + tau / (eps + b1));
  R a2 = g2 * (1.0 + tau / (eps + b2));
  R a3 = g3 * (1.0 + tau / (eps + b3));
  R asum = a0 + a1 + a2 + a3;
  R w0 = a0 / asum, w1 = a1 / asum, w2 = a2 / asum, w3 = a3 / asum;

  if (info) {
    info->theta = theta;
    info->restricted = restricted;
  }
  /* Eq. (fh_nonlinear) */
  return w0 * fh0 + w1 * fh1 + w2 * fh2 + w3 * fh3;
}

/* ------------------------------------------------------------------------- */
/* Physical fluxes and eigen-structure                                       */
/* ------------------------------------------------------------------------- */

/* Euler 1D (Sec. 4.2, Eq. (eu_eq)): u = (rho, rho u, E),
 * f = (rho u, p + rho u^2, (E + p) u), p = (gamma - 1)(E - rho u^2 / 2). */
template <class R>
void euler1d_flux(const R U[3], double gamma, R f[3], R* vel, R* pres) {
  R u = U[1] / U[0];
  R p = (gamma - 1.0) * (U[2] - 0.5 * U[0] * u * u);
  f[0] = U[1];
  f[1] = p + U[1] * u;
  f[2] = (U[2] + p) * u;
  if (vel) *vel = u;
  if (pres) *pres = p;
}

/* Euler 2D (Sec. 4.3, Eq. (eu2D)): u = (rho, rho u, rho v, E).
 * Reading: the printed equation of state drops rho; p = (gamma - 1)(E - rho (u^2 + v^2) / 2). */
template <class R>
void euler2d_prim(const R U[4], double gamma, R* u, R* v, R* p) {
  *u = U[1] / U[0];
  *v = U[2] / U[0];
  *p = (gamma - 1.0) * (U[3] - 0.5 * U[0] * (*u * *u + *v * *v));
}
template <class R>
void euler2d_flux(const R U[4], double gamma, int dir, R f[4]) {
  R u, v, p;
  euler2d_prim(U, gamma, &u, &v, &p);
  if (dir == 0) { /* f(u) */
    f[0] = U[1];
    f[1] = p + U[1] * u;
    f[2] = U[1] * v;
    f[3] = (U[3] + p) * u;
  } else { /* g(u) */
    f[0] = U[2];
    f[1] = U[2] * u;
    f[2] = p + U[2] * v;
    f[3] = (U[3] + p) * v;
  }
}

/* Eigenvalues lambda_s at one cell, for the global Lax-Friedrichs alpha_s (Eq. (flux_split_lf)). */
template <class R>
void cell_eigenvalues(const Problem& P, const R* U, int dir, R lam[4]) {
  if (P.flux == FLUX_ADVECTION) {
    lam[0] = R(P.adv_speed);
  } else if (P.flux == FLUX_BURGERS) {
    lam[0] = U[0]; /* f'(u) = u for f = u^2/2 */
  } else if (P.flux == FLUX_EULER1D) {
    R f[3], u, p;
    euler1d_flux(U, P.gamma, f, &u, &p);
    R c = sqrt(P.gamma * p / U[0]);
    lam[0] = u - c;
    lam[1] = u;
    lam[2] = u + c;
  } else {
    R u, v, p;
    euler2d_prim(U, P.gamma, &u, &v, &p);
    R c = sqrt(P.gamma * p / U[0]);
    R w = dir == 0 ? u : v;
    lam[0] = w - c;
    lam[1] = w;
    lam[2] = w;
    lam[3] = w + c;
  }
}

/* Roe's mean state between cells a and b (Sec. 4.2: "Roe's mean matrix") and the
 * right (Rm[c][s] = component c of r_s) and left (Lm[s][c] = component c of l_s)
 * eigenvectors of the Roe matrix.  Reading: the standard sqrt(rho)-weighted average
 * of velocity and total enthalpy H = (E + p)/rho; eigenvectors in the usual
 * normalisation with r_s having first component 1 (0 for the shear wave), L = R^{-1}. */
template <class R>
void roe_eigen_1d(const R Ua[3], const R Ub[3], double gamma, R Rm[3][3], R Lm[3][3]) {
  R fa[3], fb[3], ua, pa, ub, pb;
  euler1d_flux(Ua, gamma, fa, &ua, &pa);
  euler1d_flux(Ub, gamma, fb, &ub, &pb);
  R sa = sqrt(Ua[0]), sb = sqrt(Ub[0]);
  R Ha = (Ua[2] + pa) / Ua[0], Hb = (Ub[2] + pb) / Ub[0];
  R u = (sa * ua + sb * ub) / (sa + sb);
  R H = (sa * Ha + sb * Hb) / (sa + sb);
  R c = sqrt((gamma - 1.0) * (H - 0.5 * u * u));

  Rm[0][0] = R(1.0);  Rm[0][1] = R(1.0);      Rm[0][2] = R(1.0);
  Rm[1][0] = u - c;   Rm[1][1] = u;           Rm[1][2] = u + c;
  Rm[2][0] = H - u * c; Rm[2][1] = 0.5 * u * u; Rm[2][2] = H + u * c;

  R b1 = (gamma - 1.0) / (c * c);
  R b2 = 0.5 * u * u * b1;
  Lm[0][0] = 0.5 * (b2 + u / c);  Lm[0][1] = -0.5 * (b1 * u + 1.0 / c); Lm[0][2] = 0.5 * b1;
  Lm[1][0] = 1.0 - b2;            Lm[1][1] = b1 * u;                    Lm[1][2] = -b1;
  Lm[2][0] = 0.5 * (b2 - u / c);  Lm[2][1] = -0.5 * (b1 * u - 1.0 / c); Lm[2][2] = 0.5 * b1;
}

/* 2D: eigenvectors of the Roe matrix of f (dir 0) or g (dir 1).  Fields are ordered
 * (w - c, w, shear, w + c) with w the normal velocity. */
template <class R>
void roe_eigen_2d(const R Ua[4], const R Ub[4], double gamma, int dir, R Rm[4][4], R Lm[4][4]) {
  R ua, va, pa, ub, vb, pb;
  euler2d_prim(Ua, gamma, &ua, &va, &pa);
  euler2d_prim(Ub, gamma, &ub, &vb, &pb);
  R sa = sqrt(Ua[0]), sb = sqrt(Ub[0]);
  R Ha = (Ua[3] + pa) / Ua[0], Hb = (Ub[3] + pb) / Ub[0];
  R u = (sa * ua + sb * ub) / (sa + sb);
  R v = (sa * va + sb * vb) / (sa + sb);
  R H = (sa * Ha + sb * Hb) / (sa + sb);
  R q2 = u * u + v * v;
  R c = sqrt((gamma - 1.0) * (H - 0.5 * q2));
  R b1 = (gamma - 1.0) / (c * c);
  R b2 = 0.5 * q2 * b1;
  if (dir == 0) {
    Rm[0][0] = R(1.0);    Rm[0][1] = R(1.0);     Rm[0][2] = R(0.0); Rm[0][3] = R(1.0);
    Rm[1][0] = u - c;     Rm[1][1] = u;          Rm[1][2] = R(0.0); Rm[1][3] = u + c;
    Rm[2][0] = v;         Rm[2][1] = v;          Rm[2][2] = R(1.0); Rm[2][3] = v;
    Rm[3][0] = H - u * c; Rm[3][1] = 0.5 * q2;   Rm[3][2] = v;      Rm[3][3] = H + u * c;
    Lm[0][0] = 0.5 * (b2 + u / c); Lm[0][1] = -0.5 * (b1 * u + 1.0 / c); Lm[0][2] = -0.5 * (b1 * v); Lm[0][3] = 0.5 * b1;
    Lm[1][0] = 1.0 - b2;           Lm[1][1] = b1 * u;                    Lm[1][2] = b1 * v;           Lm[1][3] = -b1;
    Lm[2][0] = -v;                 Lm[2][1] = R(0.0);                    Lm[2][2] = R(1.0);           Lm[2][3] = R(0.0);
    Lm[3][0] = 0.5 * (b2 - u / c); Lm[3][1] = -0.5 * (b1 * u - 1.0 / c); Lm[3][2] = -0.5 * (b1 * v); Lm[3][3] = 0.5 * b1;
  } else {
    Rm[0][0] = R(1.0);    Rm[0][1] = R(1.0);     Rm[0][2] = R(0.0); Rm[0][3] = R(1.0);
    Rm[1][0] = u;         Rm[1][1] = u;          Rm[1][2] = R(1.0); Rm[1][3] = u;
    Rm[2][0] = v - c;     Rm[2][1] = v;          Rm[2][2] = R(0.0); Rm[2][3] = v + c;
    Rm[3][0] = H - v * c; Rm[3][1] = 0.5 * q2;   Rm[3][2] = u;      Rm[3][3] = H + v * c;
    Lm[0][0] = 0.5 * (b2 + v / c); Lm[0][1] = -0.5 * (b1 * u); Lm[0][2] = -0.5 * (b1 * v + 1.0 / c); Lm[0][3] = 0.5 * b1;
    Lm[1][0] = 1.0 - b2;           Lm[1][1] = b1 * u;          Lm[1][2] = b1 * v;                    Lm[1][3] = -b1;
    Lm[2][0] = -u;                 Lm[2][1] = R(1.0);          Lm[2][2] = R(0.0);                    Lm[2][3] = R(0.0);
    Lm[3][0] = 0.5 * (b2 - v / c); Lm[3][1] = -0.5 * (b1 * u); Lm[3][2] = -0.5 * (b1 * v - 1.0 / c); Lm[3][3] = 0.5 * b1;
  }
}

/* ------------------------------------------------------------------------- */
/* One line of cells: ghost fill, interface fluxes                           */
/* ------------------------------------------------------------------------- */

/* A line holds m components of n interior cells plus G ghosts on each side:
 * W[c][k + G] for k = -G .. n + G - 1. */
template <class R>
struct Line {
  int m, n;
  std::vector<R> w; /* [m][n + 2G] */
  Line(int m_, int n_) : m(m_), n(n_), w((size_t)m_ * (n_ + 2 * G)) {}
  R& at(int c, int k) { return w[(size_t)c * (n + 2 * G) + (k + G)]; }
};

/* Boundary conditions (ghost cells).  Periodic: u_{-k} = u_{n-k}.  Outflow
 * ("transmissive", "zero-gradient" in Sec. 4.2): ghost = nearest interior cell.
 * Reflective: mirror image with the normal momentum negated. */
template <class R>
void fill_ghosts(Line<R>& L, int bc_lo, int bc_hi, int normal_comp) {
#ifdef WTO_PLANT_REFLECT_SIGN
  /* A deliberately wrong variant, built only by a test that must see its pins fail: the
   * reflective ghost keeps the sign of the normal momentum. */
  normal_comp = -1;
#endif
  for (int c = 0; c < L.m; ++c) {
    for (int k = 1; k <= G; ++k) {
      R lo, hi;
      if (bc_lo == BC_PERIODIC) lo = L.at(c, L.n - k);
      else if (bc_lo == BC_OUTFLOW) lo = L.at(c, 0);
      else lo = (c == normal_comp) ? -L.at(c, k - 1) : L.at(c, k - 1);
      if (bc_hi == BC_PERIODIC) hi = L.at(c, k - 1);
      else if (bc_hi == BC_OUTFLOW) hi = L.at(c, L.n - 1);
      else hi = (c == normal_comp) ? -L.at(c, L.n - k) : L.at(c, L.n - k);
      L.at(c, -k) = lo;
      L.at(c, L.n - 1 + k) = hi;
    }
  }
}

/* Flux splitting constants alpha_s = max over the interior cells of |lambda_s(u_j)|
 * (Eq. (flux_split_lf): "max |f'(u)| over the whole computational domain").
 * Reading: one alpha per characteristic field, re-evaluated from each stage's input. */

/* Interface fluxes hF[c][i + 1] at x_{i+1/2}, i = -1 .. n-1, for one line whose ghosts
 * are filled.  Systems: characteristic-wise WENO (Sec. 4.2): project the six cells onto
 * the left eigenvectors of the Roe matrix at x_{i+1/2}, split each field with its
 * alpha_s, reconstruct both sides, project back with the right eigenvectors. */
template <class R>
void line_fluxes(const Problem& P, Line<R>& L, int dir, const R* alpha, std::vector<R>& hF, long long* theta1_count,
                 long long* restricted_count) {
  const int m = L.m, n = L.n;
  hF.assign((size_t)m * (n + 1), R(0.0));
  /* cell fluxes f(u_k), k = -G .. n+G-1 */
  Line<R> F(m, n);
  for (int k = -G; k < n + G; ++k) {
    R U[4], f[4];
    for (int c = 0; c < m; ++c) U[c] = L.at(c, k);
    if (P.flux == FLUX_ADVECTION) f[0] = P.adv_speed * U[0];
    else if (P.flux == FLUX_BURGERS) f[0] = 0.5 * U[0] * U[0]; /* Eq. (bur_eq) */
    else if (P.flux == FLUX_EULER1D) euler1d_flux(U, P.gamma, f, (R*)0, (R*)0);
    else euler2d_flux(U, P.gamma, dir, f);
    for (int c = 0; c < m; ++c) F.at(c, k) = f[c];
  }
  for (int i = -1; i < n; ++i) {
    if (m == 1) {
      /* scalar: Eq. (flux_split_lf), f^- mirrored about x_{i+1/2} */
      R vp[6], vm[6], qp[6], qm[6];
      for (int k = 0; k < 6; ++k) {
        R f = F.at(0, i - 2 + k), u = L.at(0, i - 2 + k);
        vp[k] = 0.5 * (f + alpha[0] * u);
        vm[k] = 0.5 * (f - alpha[0] * u);
      }
      for (int k = 0; k < 6; ++k) {
        qp[k] = vp[k];
        qm[k] = vm[5 - k];
      }
      RecInfo ip, im;
      R Fp = weno_theta(qp, P.eps, P.alpha_R, &ip);
      R Fm = weno_theta(qm, P.eps, P.alpha_R, &im);
      hF[(size_t)(i + 1)] = Fp + Fm;
      if (theta1_count) *theta1_count += ip.theta + im.theta;
      if (restricted_count) *restricted_count += ip.restricted + im.restricted;
      continue;
    }
    R Rm[4][4], Lm[4][4];
    R Ua[4], Ub[4];
    for (int c = 0; c < m; ++c) {
      Ua[c] = L.at(c, i);
      Ub[c] = L.at(c, i + 1);
    }
    if (m == 3) {
      R R3[3][3], L3[3][3];
      roe_eigen_1d(Ua, Ub, P.gamma, R3, L3);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          Rm[a][b] = R3[a][b];
          Lm[a][b] = L3[a][b];
        }
    } else {
      roe_eigen_2d(Ua, Ub, P.gamma, dir, Rm, Lm);
    }
    R Fs[4];
    for (int s = 0; s < m; ++s) {
      R vp[6], vm[6], qp[6], qm[6];
      for (int k = 0; k < 6; ++k) {
        int cell = i - 2 + k;
        /* l_s . f and l_s . u, summed density, normal momentum, tangential momentum (2D),
         * energy: the same order in both sweep directions */
        R a = Lm[s][0] * F.at(0, cell);
        R b = Lm[s][0] * L.at(0, cell);
        const int nc = (m == 4) ? 1 + dir : 1, tc = 2 - dir;
        a = a + Lm[s][nc] * F.at(nc, cell);
        b = b + Lm[s][nc] * L.at(nc, cell);
        if (m == 4) {
          a = a + Lm[s][tc] * F.at(tc, cell);
          b = b + Lm[s][tc] * L.at(tc, cell);
        }
        a = a + Lm[s][m - 1] * F.at(m - 1, cell);
        b = b + Lm[s][m - 1] * L.at(m - 1, cell);
        vp[k] = 0.5 * (a + alpha[s] * b);
        vm[k] = 0.5 * (a - alpha[s] * b);
      }
      for (int k = 0; k < 6; ++k) {
        qp[k] = vp[k];
        qm[k] = vm[5 - k];
      }
      RecInfo ip, im;
      R Fp = weno_theta(qp, P.eps, P.alpha_R, &ip);
      R Fm = weno_theta(qm, P.eps, P.alpha_R, &im);
      Fs[s] = Fp + Fm;
      if (theta1_count) *theta1_count += ip.theta + im.theta;
      if (restricted_count) *restricted_count += ip.restricted + im.restricted;
    }
    /* h = R (F+ + F-): the two acoustic fields (u - c, u + c) summed first, then the others,
     * so that a mirrored state gives the mirrored flux in floating point too */
    for (int c = 0; c < m; ++c) {
      R h = Rm[c][0] * Fs[0] + Rm[c][m - 1] * Fs[m - 1];
      if (m == 3) h = h + Rm[c][1] * Fs[1];
      else h = h + (Rm[c][1] * Fs[1] + Rm[c][2] * Fs[2]);
      hF[(size_t)c * (n + 1) + (i + 1)] = h;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Right-hand side L(u) (Eq. (mod_semi)), alpha_s and the CFL time step      */
/* ------------------------------------------------------------------------- */

struct Grid {
  int64_t nx, ny; /* ny = 1 for 1D */
  double dx, dy;
};

inline int ndim_of(const Problem& P) { return P.flux == FLUX_EULER2D ? 2 : 1; }

/* alpha_s per direction: alpha[dir * 4 + s] */
template <class R>
void compute_alpha(const Problem& P, const Grid& g, const R* u, R* alpha) {
  const int m = P.m;
  const int64_t cells = g.nx * g.ny;
  for (int d = 0; d < ndim_of(P); ++d) {
    for (int s = 0; s < m; ++s) alpha[d * 4 + s] = R(0.0);
    for (int64_t j = 0; j < cells; ++j) {
      R U[4], lam[4];
      for (int c = 0; c < m; ++c) U[c] = u[(size_t)c * cells + j];
      cell_eigenvalues(P, U, d, lam);
      for (int s = 0; s < m; ++s) alpha[d * 4 + s] = rmax(alpha[d * 4 + s], fabs(lam[s]));
    }
  }
}

/* Reading of "a proper CFL condition" (Sec. 2.1):
 *   1D: dt = CFL dx / max_j (|u_j| + c_j)   (advection: |a|, Burgers: |u_j|)
 *   2D: dt = CFL / max_j ((|u_j| + c_j)/dx + (|v_j| + c_j)/dy) */
template <class R>
R cfl_dt(const Problem& P, const Grid& g, const R* u, double cfl) {
  const int m = P.m;
  const int64_t cells = g.nx * g.ny;
  R smax = R(0.0);
  for (int64_t j = 0; j < cells; ++j) {
    R U[4];
    for (int c = 0; c < m; ++c) U[c] = u[(size_t)c * cells + j];
    R s;
    if (P.flux == FLUX_ADVECTION) s = R(std::fabs(P.adv_speed));
    else if (P.flux == FLUX_BURGERS) s = fabs(U[0]);
    else if (P.flux == FLUX_EULER1D) {
      R f[3], uu, p;
      euler1d_flux(U, P.gamma, f, &uu, &p);
      R c = sqrt(P.gamma * p / U[0]);
      s = fabs(uu) + c;
    } else {
      R uu, vv, p;
      euler2d_prim(U, P.gamma, &uu, &vv, &p);
      R c = sqrt(P.gamma * p / U[0]);
      s = (fabs(uu) + c) / g.dx + (fabs(vv) + c) / g.dy;
    }
    smax = rmax(smax, s);
  }
  if (ndim_of(P) == 2) return cfl / smax;
  return cfl * g.dx / smax;
}

/* L(u), Eq. (mod_semi): L_j = -(h_{j+1/2} - h_{j-1/2}) / dx, summed over the two
 * directions for 2D (dimension by dimension, Sec. 4.3). */
template <class R>
void rhs(const Problem& P, const Grid& g, const R* u, R* Lout, long long* theta1, long long* restricted) {
  const int m = P.m;
  const int64_t nx = g.nx, ny = g.ny, cells = nx * ny;
  R alpha[8];
  compute_alpha(P, g, u, alpha);
  for (int64_t j = 0; j < cells * m; ++j) Lout[j] = R(0.0);
  /* Rows (and columns) are independent and write disjoint entries of Lout, so with OpenMP they
   * may run on several threads (values only: the counters and the Dual / Cnt types stay serial);
   * every entry is computed by the same operations either way. */
  const bool par = std::is_same<R, double>::value && !theta1 && !restricted;
  (void)par;
  /* x sweep: every row */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (par && ny > 1)
#endif
  for (int64_t r = 0; r < ny; ++r) {
    std::vector<R> hF;
    Line<R> L(m, (int)nx);
    for (int c = 0; c < m; ++c)
      for (int64_t i = 0; i < nx; ++i) L.at(c, (int)i) = u[(size_t)c * cells + r * nx + i];
    fill_ghosts(L, P.bc_lo[0], P.bc_hi[0], 1);
    line_fluxes(P, L, 0, alpha, hF, theta1, restricted);
    for (int c = 0; c < m; ++c)
      for (int64_t i = 0; i < nx; ++i) {
        R hp = hF[(size_t)c * (nx + 1) + (i + 1)], hm = hF[(size_t)c * (nx + 1) + i];
        Lout[(size_t)c * cells + r * nx + i] = -(hp - hm) / g.dx;
      }
  }
  if (ndim_of(P) == 1) return;
  /* y sweep: every column; L = Lx + Ly */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (par)
#endif
  for (int64_t col = 0; col < nx; ++col) {
    std::vector<R> hF;
    Line<R> L(m, (int)ny);
    for (int c = 0; c < m; ++c)
      for (int64_t j = 0; j < ny; ++j) L.at(c, (int)j) = u[(size_t)c * cells + j * nx + col];
    fill_ghosts(L, P.bc_lo[1], P.bc_hi[1], 2);
    line_fluxes(P, L, 1, alpha + 4, hF, theta1, restricted);
    for (int c = 0; c < m; ++c)
      for (int64_t j = 0; j < ny; ++j) {
        R hp = hF[(size_t)c * (ny + 1) + (j + 1)], hm = hF[(size_t)c * (ny + 1) + j];
        size_t idx = (size_t)c * cells + j * nx + col;
        Lout[idx] = Lout[idx] + (-(hp - hm) / g.dy);
      }
  }
  /* gravity in -y (TEST 6, Sec. 4.3): -g rho added to the y-momentum and -g rho v to the energy
   * equation, rho v being the conserved y momentum */
  if (P.gravity != 0.0) {
    for (int64_t j = 0; j < cells; ++j) {
      Lout[2 * cells + j] = Lout[2 * cells + j] + (-(P.gravity * u[j]));
      Lout[3 * cells + j] = Lout[3 * cells + j] + (-(P.gravity * u[2 * cells + j]));
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Time integration: 3rd-order TVD Runge-Kutta, Eq. (3rd_RK)                 */
/* ------------------------------------------------------------------------- */

/* Advances u in place.  dt = CFL step from u^n (or dt_fixed > 0), clipped to
 * t_final - t.  Stops after n_steps steps or when t reaches t_final. */
template <class R>
void run(const Problem& P, const Grid& g, R* u, double cfl, double dt_fixed, double t_final, int64_t n_steps,
         double* t_out, int64_t* steps_out) {
  const size_t len = (size_t)P.m * g.nx * g.ny;
  std::vector<R> un(u, u + len), u1(len), u2(len), L(len);
  double t = 0.0;
  int64_t steps = 0;
  const double c13 = 1.0 / 3.0, c23 = 2.0 / 3.0;
  while (steps < n_steps && t < t_final) {
    R dt = dt_fixed > 0.0 ? R(dt_fixed) : cfl_dt(P, g, un.data(), cfl);
    if (t_final - t < val(dt)) dt = R(t_final - t);
    rhs(P, g, un.data(), L.data(), (long long*)0, (long long*)0);
    for (size_t j = 0; j < len; ++j) u1[j] = un[j] + dt * L[j];
    rhs(P, g, u1.data(), L.data(), (long long*)0, (long long*)0);
    for (size_t j = 0; j < len; ++j) u2[j] = 0.75 * un[j] + 0.25 * u1[j] + 0.25 * dt * L[j];
    rhs(P, g, u2.data(), L.data(), (long long*)0, (long long*)0);
    for (size_t j = 0; j < len; ++j) un[j] = c13 * un[j] + c23 * u2[j] + c23 * dt * L[j];
    t = t + val(dt);
    steps = steps + 1;
  }
  for (size_t j = 0; j < len; ++j) u[j] = un[j];
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = steps;
}

/* ------------------------------------------------------------------------- */
/* Exact Riemann solver for the 1D Euler equations (reference solution of the */
/* shock-tube tests, Sec. 4.2 TEST 3).  Written from the standard pressure-    */
/* function formulation: f_L(p) + f_R(p) + (u_R - u_L) = 0, each f_K being the */
/* shock (Rankine-Hugoniot) or rarefaction (isentropic Riemann invariant) branch. */
/* ------------------------------------------------------------------------- */

struct RState {
  double rho, u, p;
};

static double pfun(double p, const RState& K, double g, double* dfdp) {
  double c = std::sqrt(g * K.p / K.rho);
  if (p > K.p) { /* shock */
    double A = 2.0 / ((g + 1.0) * K.rho), B = (g - 1.0) / (g + 1.0) * K.p;
    double q = std::sqrt(A / (p + B));
    *dfdp = q * (1.0 - 0.5 * (p - K.p) / (p + B));
    return (p - K.p) * q;
  }
  /* rarefaction */
  double e = (g - 1.0) / (2.0 * g);
  *dfdp = 1.0 / (K.rho * c) * std::pow(p / K.p, -(g + 1.0) / (2.0 * g));
  return 2.0 * c / (g - 1.0) * (std::pow(p / K.p, e) - 1.0);
}

/* star-region pressure and velocity by Newton's method on the pressure function */
static void riemann_star(const RState& Lf, const RState& Rt, double g, double* pstar, double* ustar, int* iters) {
  double cL = std::sqrt(g * Lf.p / Lf.rho), cR = std::sqrt(g * Rt.p / Rt.rho);
  /* two-rarefaction estimate as the starting point */
  double e = (g - 1.0) / (2.0 * g);
  double p = std::pow((cL + cR - 0.5 * (g - 1.0) * (Rt.u - Lf.u)) / (cL / std::pow(Lf.p, e) + cR / std::pow(Rt.p, e)),
                      1.0 / e);
  if (!(p > 1e-14)) p = 1e-14;
  int it = 0;
  for (; it < 200; ++it) {
    double dL, dR;
    double f = pfun(p, Lf, g, &dL) + pfun(p, Rt, g, &dR) + (Rt.u - Lf.u);
    double pn = p - f / (dL + dR);
    if (pn < 1e-14) pn = 1e-14;
    double change = std::fabs(pn - p) / (0.5 * (pn + p));
    p = pn;
    if (change < 1e-15) break;
  }
  double dL, dR;
  *pstar = p;
  *ustar = 0.5 * (Lf.u + Rt.u) + 0.5 * (pfun(p, Rt, g, &dR) - pfun(p, Lf, g, &dL));
  if (iters) *iters = it;
}

/* Sample the self-similar solution at s = (x - x0)/t. */
static RState riemann_sample(const RState& Lf, const RState& Rt, double g, double pstar, double ustar, double s) {
  double cL = std::sqrt(g * Lf.p / Lf.rho), cR = std::sqrt(g * Rt.p / Rt.rho);
  double gm = (g - 1.0) / (g + 1.0);
  if (s <= ustar) { /* left of the contact */
    if (pstar > Lf.p) {
      double rs = Lf.rho * (pstar / Lf.p + gm) / (gm * pstar / Lf.p + 1.0);
      double S = Lf.u - cL * std::sqrt((g + 1.0) / (2.0 * g) * pstar / Lf.p + (g - 1.0) / (2.0 * g));
      if (s <= S) return Lf;
      return RState{rs, ustar, pstar};
    }
    double rs = Lf.rho * std::pow(pstar / Lf.p, 1.0 / g);
    double cs = cL * std::pow(pstar / Lf.p, (g - 1.0) / (2.0 * g));
    double head = Lf.u - cL, tail = ustar - cs;
    if (s <= head) return Lf;
    if (s >= tail) return RState{rs, ustar, pstar};
    double u = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * Lf.u + s);
    double c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (Lf.u - s));
    double rho = Lf.rho * std::pow(c / cL, 2.0 / (g - 1.0));
    double p = Lf.p * std::pow(c / cL, 2.0 * g / (g - 1.0));
    return RState{rho, u, p};
  }
  if (pstar > Rt.p) {
    double rs = Rt.rho * (pstar / Rt.p + gm) / (gm * pstar / Rt.p + 1.0);
    double S = Rt.u + cR * std::sqrt((g + 1.0) / (2.0 * g) * pstar / Rt.p + (g - 1.0) / (2.0 * g));
    if (s >= S) return Rt;
    return RState{rs, ustar, pstar};
  }
  double rs = Rt.rho * std::pow(pstar / Rt.p, 1.0 / g);
  double cs = cR * std::pow(pstar / Rt.p, (g - 1.0) / (2.0 * g));
  double head = Rt.u + cR, tail = ustar + cs;
  if (s >= head) return Rt;
  if (s <= tail) return RState{rs, ustar, pstar};
  double u = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * Rt.u + s);
  double c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (Rt.u - s));
  double rho = Rt.rho * std::pow(c / cR, 2.0 / (g - 1.0));
  double p = Rt.p * std::pow(c / cR, 2.0 * g / (g - 1.0));
  return RState{rho, u, p};
}

} /* namespace wto */

/* ------------------------------------------------------------------------- */
/* C entry points for the Python test harness (ctypes)                        */
/* ------------------------------------------------------------------------- */

using namespace wto;

extern "C" {

/* One reconstruction: q[6] -> value; theta and restriction flags out. */
double wto_weno_theta(const double* q, double eps, double alpha_R, int32_t* theta, int32_t* restricted) {
  RecInfo info;
  double r = weno_theta(q, eps, alpha_R, &info);
  if (theta) *theta = info.theta;
  if (restricted) *restricted = info.restricted;
  return r;
}

/* Smoothness indicators: out = {beta0, beta1, beta2, beta3, tau5, tau6} (before Eq. (be_res)). */
void wto_indicators(const double* q, double* out) {
  double b[4], t5, t6;
  smoothness(q, b, &t5, &t6);
  for (int k = 0; k < 4; ++k) out[k] = b[k];
  out[4] = t5;
  out[5] = t6;
}

/* Roe eigenvectors: Rm, Lm row-major m x m (m = 3 for 1D, 4 for 2D). */
void wto_roe_eigen(int32_t m, const double* Ua, const double* Ub, double gamma, int32_t dir, double* Rm, double* Lm) {
  if (m == 3) {
    double R3[3][3], L3[3][3];
    roe_eigen_1d(Ua, Ub, gamma, R3, L3);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        Rm[a * 3 + b] = R3[a][b];
        Lm[a * 3 + b] = L3[a][b];
      }
  } else {
    double R4[4][4], L4[4][4];
    roe_eigen_2d(Ua, Ub, gamma, dir, R4, L4);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        Rm[a * 4 + b] = R4[a][b];
        Lm[a * 4 + b] = L4[a][b];
      }
  }
}

/* alpha[dir*4 + s] and the CFL step of state u ([m][ny][nx], x fastest). */
void wto_alpha(const Problem* P, int64_t nx, int64_t ny, double dx, double dy, const double* u, double cfl,
               double* alpha8, double* dt) {
  Grid g{nx, ny, dx, dy};
  compute_alpha(*P, g, u, alpha8);
  if (dt) *dt = cfl_dt(*P, g, u, cfl);
}

/* L(u); theta1 / restricted count the reconstructions with theta = 1 / beta restricted. */
void wto_rhs(const Problem* P, int64_t nx, int64_t ny, double dx, double dy, const double* u, double* L,
             int64_t* theta1, int64_t* restricted) {
  Grid g{nx, ny, dx, dy};
  long long t1 = 0, rs = 0;
  rhs(*P, g, u, L, &t1, &rs);
  if (theta1) *theta1 = t1;
  if (restricted) *restricted = rs;
}

/* L(u) at selected cells only (cells[k] = y * nx + x), with the Lax-Friedrichs constants
 * alpha8[dir * 4 + s] of the whole state given (wto_alpha computes them).  Each sampled cell
 * takes the interface fluxes of its own row and column, computed exactly as in rhs(). */
void wto_rhs_at(const Problem* P, int64_t nx, int64_t ny, double dx, double dy, const double* u, const double* alpha8,
                const int64_t* cells, int64_t ncells, double* out) {
  const int m = P->m;
  const int64_t all = nx * ny;
  std::vector<double> hF;
  for (int64_t q = 0; q < ncells; ++q) {
    const int64_t y = cells[q] / nx, x = cells[q] - y * nx;
    Line<double> row(m, (int)nx);
    for (int c = 0; c < m; ++c)
      for (int64_t i = 0; i < nx; ++i) row.at(c, (int)i) = u[(size_t)c * all + y * nx + i];
    fill_ghosts(row, P->bc_lo[0], P->bc_hi[0], 1);
    line_fluxes(*P, row, 0, alpha8, hF, (long long*)0, (long long*)0);
    for (int c = 0; c < m; ++c) {
      double hp = hF[(size_t)c * (nx + 1) + (x + 1)], hm = hF[(size_t)c * (nx + 1) + x];
      out[q * m + c] = -(hp - hm) / dx;
    }
    if (ndim_of(*P) == 1) continue;
    Line<double> col(m, (int)ny);
    for (int c = 0; c < m; ++c)
      for (int64_t j = 0; j < ny; ++j) col.at(c, (int)j) = u[(size_t)c * all + j * nx + x];
    fill_ghosts(col, P->bc_lo[1], P->bc_hi[1], 2);
    line_fluxes(*P, col, 1, alpha8 + 4, hF, (long long*)0, (long long*)0);
    for (int c = 0; c < m; ++c) {
      double hp = hF[(size_t)c * (ny + 1) + (y + 1)], hm = hF[(size_t)c * (ny + 1) + y];
      out[q * m + c] = out[q * m + c] + (-(hp - hm) / dy);
    }
    if (P->gravity != 0.0) {
      out[q * m + 2] = out[q * m + 2] + (-(P->gravity * u[cells[q]]));
      out[q * m + 3] = out[q * m + 3] + (-(P->gravity * u[2 * all + cells[q]]));
    }
  }
}

/* Forward-mode derivative of L at u in direction du. */
void wto_rhs_jvp(const Problem* P, int64_t nx, int64_t ny, double dx, double dy, const double* u, const double* du,
                 double* L, double* dL) {
  Grid g{nx, ny, dx, dy};
  size_t len = (size_t)P->m * nx * ny;
  std::vector<Dual> U(len), LL(len);
  for (size_t j = 0; j < len; ++j) U[j] = Dual(u[j], du[j]);
  rhs(*P, g, U.data(), LL.data(), (long long*)0, (long long*)0);
  for (size_t j = 0; j < len; ++j) {
    L[j] = LL[j].v;
    dL[j] = LL[j].d;
  }
}

/* Time integration in place. */
void wto_run(const Problem* P, int64_t nx, int64_t ny, double dx, double dy, double* u, double cfl, double dt_fixed,
             double t_final, int64_t n_steps, double* t_out, int64_t* steps_out) {
  Grid g{nx, ny, dx, dy};
  run(*P, g, u, cfl, dt_fixed, t_final, n_steps, t_out, steps_out);
}

/* Forward-mode derivative of the whole run: u -> u(T), direction du -> du(T). */
void wto_run_jvp(const Problem* P, int64_t nx, int64_t ny, double dx, double dy, double* u, double* du, double cfl,
                 double dt_fixed, double t_final, int64_t n_steps, double* t_out, int64_t* steps_out) {
  Grid g{nx, ny, dx, dy};
  size_t len = (size_t)P->m * nx * ny;
  std::vector<Dual> U(len);
  for (size_t j = 0; j < len; ++j) U[j] = Dual(u[j], du[j]);
  run(*P, g, U.data(), cfl, dt_fixed, t_final, n_steps, t_out, steps_out);
  for (size_t j = 0; j < len; ++j) {
    u[j] = U[j].v;
    du[j] = U[j].d;
  }
}

/* Arithmetic operations of one L(u) evaluation: out = {add/sub, mul, div, sqrt, compare}. */
void wto_count_rhs_ops(const Problem* P, int64_t nx, int64_t ny, double dx, double dy, const double* u, int64_t* out) {
  Grid g{nx, ny, dx, dy};
  size_t len = (size_t)P->m * nx * ny;
  std::vector<Cnt> U(len), LL(len);
  for (size_t j = 0; j < len; ++j) U[j] = Cnt(u[j]);
  g_ops = OpCount{0, 0, 0, 0, 0};
  rhs(*P, g, U.data(), LL.data(), (long long*)0, (long long*)0);
  out[0] = g_ops.add;
  out[1] = g_ops.mul;
  out[2] = g_ops.div;
  out[3] = g_ops.sqrt;
  out[4] = g_ops.cmp;
}

/* Arithmetic operations of n_steps RK3 steps (CFL step from u^n included). */
void wto_count_run_ops(const Problem* P, int64_t nx, int64_t ny, double dx, double dy, const double* u, double cfl,
                       int64_t n_steps, int64_t* out) {
  Grid g{nx, ny, dx, dy};
  size_t len = (size_t)P->m * nx * ny;
  std::vector<Cnt> U(len);
  for (size_t j = 0; j < len; ++j) U[j] = Cnt(u[j]);
  g_ops = OpCount{0, 0, 0, 0, 0};
  run(*P, g, U.data(), cfl, 0.0, INFINITY, n_steps, (double*)0, (int64_t*)0);
  out[0] = g_ops.add;
  out[1] = g_ops.mul;
  out[2] = g_ops.div;
  out[3] = g_ops.sqrt;
  out[4] = g_ops.cmp;
}

/* Time integration of nprob independent 1D problems stored in packed planes
 * u[c * total + offsets[p] + j] (j < lengths[p]), each on its own grid [lo[p], hi[p]] with
 * boundary condition bc[p] at both ends, n_steps steps each with its own CFL step (t_final =
 * +inf).  Every problem is the serial run() above on its own copy of the data, so the result
 * does not depend on how many threads share the problems (OpenMP over problems, largest
 * first, when the library is built with -fopenmp).  steps_out[p] (may be NULL): steps taken. */
void wto_run_batch(const Problem* P, int32_t nprob, const int64_t* offsets, const int64_t* lengths, const double* lo,
                   const double* hi, const int32_t* bc, double* u, int64_t total, double cfl, int64_t n_steps,
                   int32_t nthreads, int64_t* steps_out) {
  std::vector<int32_t> order((size_t)nprob);
  for (int32_t p = 0; p < nprob; ++p) order[(size_t)p] = p;
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return lengths[a] > lengths[b]; });
#ifdef _OPENMP
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int32_t k = 0; k < nprob; ++k) {
    const int32_t p = order[(size_t)k];
    const int64_t n = lengths[p];
    Problem Q = *P;
    Q.bc_lo[0] = Q.bc_hi[0] = bc[p];
    Grid g{n, 1, (hi[p] - lo[p]) / (double)n, 1.0};
    std::vector<double> w((size_t)Q.m * n);
    for (int c = 0; c < Q.m; ++c)
      for (int64_t j = 0; j < n; ++j) w[(size_t)c * n + j] = u[(size_t)c * total + offsets[p] + j];
    int64_t steps = 0;
    run(Q, g, w.data(), cfl, 0.0, INFINITY, n_steps, (double*)0, &steps);
    for (int c = 0; c < Q.m; ++c)
      for (int64_t j = 0; j < n; ++j) u[(size_t)c * total + offsets[p] + j] = w[(size_t)c * n + j];
    if (steps_out) steps_out[p] = steps;
  }
}

/* The forward-mode derivative of wto_run_batch: du (same packing as u) is the direction and
 * returns the derivative of u(T) along it, problem by problem (each one run_jvp's map). */
void wto_run_jvp_batch(const Problem* P, int32_t nprob, const int64_t* offsets, const int64_t* lengths,
                       const double* lo, const double* hi, const int32_t* bc, double* u, double* du, int64_t total,
                       double cfl, int64_t n_steps, int32_t nthreads) {
  std::vector<int32_t> order((size_t)nprob);
  for (int32_t p = 0; p < nprob; ++p) order[(size_t)p] = p;
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return lengths[a] > lengths[b]; });
#ifdef _OPENMP
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int32_t k = 0; k < nprob; ++k) {
    const int32_t p = order[(size_t)k];
    const int64_t n = lengths[p];
    Problem Q = *P;
    Q.bc_lo[0] = Q.bc_hi[0] = bc[p];
    Grid g{n, 1, (hi[p] - lo[p]) / (double)n, 1.0};
    std::vector<Dual> w((size_t)Q.m * n);
    for (int c = 0; c < Q.m; ++c)
      for (int64_t j = 0; j < n; ++j) {
        const size_t at = (size_t)c * total + offsets[p] + j;
        w[(size_t)c * n + j] = Dual(u[at], du[at]);
      }
    run(Q, g, w.data(), cfl, 0.0, INFINITY, n_steps, (double*)0, (int64_t*)0);
    for (int c = 0; c < Q.m; ++c)
      for (int64_t j = 0; j < n; ++j) {
        const size_t at = (size_t)c * total + offsets[p] + j;
        u[at] = w[(size_t)c * n + j].v;
        du[at] = w[(size_t)c * n + j].d;
      }
  }
}

/* Threads wto_run_batch and the 2D sweeps use when nthreads = 0 (1 without OpenMP). */
int32_t wto_max_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sets that thread count (ignored without OpenMP); returns 1 if the library has OpenMP. */
int32_t wto_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return 1;
#else
  (void)n;
  return 0;
#endif
}

/* Exact Riemann problem: star state and the solution sampled at xs (jump at x0, time t). */
void wto_riemann_star(double rL, double uL, double pL, double rR, double uR, double pR, double gamma, double* pstar,
                      double* ustar, int32_t* iters) {
  int it = 0;
  riemann_star(RState{rL, uL, pL}, RState{rR, uR, pR}, gamma, pstar, ustar, &it);
  if (iters) *iters = it;
}

void wto_riemann_sample(double rL, double uL, double pL, double rR, double uR, double pR, double gamma, double x0,
                        double t, const double* xs, int64_t n, double* rho, double* u, double* p) {
  RState Lf{rL, uL, pL}, Rt{rR, uR, pR};
  double ps, us;
  riemann_star(Lf, Rt, gamma, &ps, &us, (int*)0);
  for (int64_t i = 0; i < n; ++i) {
    RState s = riemann_sample(Lf, Rt, gamma, ps, us, (xs[i] - x0) / t);
    rho[i] = s.rho;
    u[i] = s.u;
    p[i] = s.p;
  }
}

} /* extern "C" */
