// Fast arithmetic policy.  Same mathematics as the strict policy, rearranged for a GPU
// whose FP64 pipe is its scarce resource (about 2 FMA per clock per SM on GB300, with
// integer and FP32 pipes 30-60x wider):
//   - fused multiply-adds throughout;
//   - the indicators of Eqs. (be0_cen)-(be3_cen), (tau_5), (tau_6) from first and second
//     differences of the stencil, which share most of their terms;
//   - comparisons of non-negative doubles on their bit patterns (integer pipe);
//   - the weights of Eq. (om) over a common denominator prod_l (eps + beta_l), so one
//     division per reconstruction; a restricted stencil (all beta = 0, Eq. (be_res)) has
//     weights equal to gamma^theta and takes the equivalent linear scheme in closed form;
//   - the restriction test R(beta) <= alpha_R as max beta <= alpha_R (eps + min beta);
//   - the 1/2 of the flux splitting folded into the left eigenvectors.
// Results agree with the strict policy to rounding.
#pragma once

#include "wt_device.cuh"

namespace wt {

struct FastMath {
  static constexpr bool kStrict = false;
  static constexpr bool kRoeRows = false;  // Roe matrix one row per thread (roe_row)
  // projection v = kProj (L f +- alpha L u) with the stored L = kLScale * L_true
  static constexpr double kProj = 1.0, kLScale = 0.5;

  __device__ __forceinline__ static long long bits(double x) { return __double_as_longlong(x); }
  // a b + c d with both products rounded and no contraction into an FMA: the same value when
  // the two terms trade places (mirrored or transposed data give mirrored or transposed fluxes)
  __device__ __forceinline__ static double dot2(double a, double b, double c, double d) {
    return __dadd_rn(__dmul_rn(a, b), __dmul_rn(c, d));
  }
  // max / min / less-than of non-negative doubles through their bit patterns
  __device__ __forceinline__ static double nmax(double a, double b) { return bits(a) < bits(b) ? b : a; }
  __device__ __forceinline__ static double nmin(double a, double b) { return bits(b) < bits(a) ? b : a; }

  __device__ __forceinline__ static double flux_advection(double a, double u) { return a * u; }
  __device__ __forceinline__ static double flux_burgers(double u) { return 0.5 * u * u; }

  // 1 / rho and sqrt(rho) from one reciprocal square root
  __device__ __forceinline__ static void euler_cell_ir(const double* U, double gamma, double* f, double& u, double& H,
                                                       double& sr, double& p, double& ir) {
    const double r = rsqrt(U[0]);
    ir = r * r;
    sr = U[0] * r;
    u = U[1] * ir;
    p = (gamma - 1.0) * fma(-0.5 * U[1], u, U[2]);
    const double e = U[2] + p;
    f[0] = U[1];
    f[1] = fma(U[1], u, p);
    f[2] = e * u;
    H = e * ir;
  }
  __device__ __forceinline__ static void euler_cell(const double* U, double gamma, double* f, double& u, double& H,
                                                    double& sr, double& p) {
    double ir;
    euler_cell_ir(U, gamma, f, u, H, sr, p, ir);
  }
  // sound speed c = sqrt(c2) as c2 rsqrt(c2), a shorter dependent chain than the IEEE square
  // root (the wave speeds open the alpha exchange of every stage); c2 <= 0, huge or NaN keeps
  // the square root
  __device__ __forceinline__ static double sound_speed(double c2) {
    return (c2 > 0.0 && c2 < 1e300) ? c2 * rsqrt(c2) : sqrt(c2);
  }
  __device__ __forceinline__ static void euler_cell_speeds(const double* U, double gamma, double* f, double& u,
                                                           double& H, double& sr, double* lam) {
    double p, ir;
    euler_cell_ir(U, gamma, f, u, H, sr, p, ir);
    const double c = sound_speed(gamma * p * ir);
    lam[0] = fabs(u - c);
    lam[1] = fabs(u);
    lam[2] = fabs(u + c);
  }

  // the wave speeds exactly as euler_cell_speeds computes them
  __device__ __forceinline__ static double euler_speeds(const double* U, double gamma, double* lam) {
    double f[3], u, H, sr, p, ir;
    euler_cell_ir(U, gamma, f, u, H, sr, p, ir);
    const double c = sound_speed(gamma * p * ir);
    lam[0] = fabs(u - c);
    lam[1] = fabs(u);
    lam[2] = fabs(u + c);
    return p;
  }

  // euler_speeds in two parts, with its operations: |u| (keeping u and 1 / rho), then
  // |u - c| and |u + c|
  __device__ __forceinline__ static double speed_u(const double* U, double& u, double& ir) {
    const double r = rsqrt(U[0]);
    ir = r * r;
    u = U[1] * ir;
    return fabs(u);
  }
  __device__ __forceinline__ static void speed_c(const double* U, double gamma, double u, double ir, double& l0,
                                                 double& l2) {
    const double p = (gamma - 1.0) * fma(-0.5 * U[1], u, U[2]);
    const double c = sound_speed(gamma * p * ir);
    l0 = fabs(u - c);
    l2 = fabs(u + c);
  }

  // L is stored pre-scaled by 1/2 (the factor of Eq. (flux_split_lf))
  __device__ __forceinline__ static void roe(double sa, double ua, double Ha, double sb, double ub, double Hb,
                                             double gamma, double* L, double* rs) {
    const double is = 1.0 / (sa + sb);
    const double wa = sa * is, wb = sb * is;
    const double u = dot2(wa, ua, wb, ub);
    const double H = dot2(wa, Ha, wb, Hb);
    roe_mean(u, H, gamma, L, rs);
  }
  // the (1/2-scaled) left eigenvectors and (u, H, c) from Roe's mean velocity and enthalpy,
  // exactly as roe() forms them
  __device__ __forceinline__ static void roe_mean(double u, double H, double gamma, double* L, double* rs) {
    const double gm1 = gamma - 1.0;
    const double c2 = gm1 * fma(-0.5 * u, u, H);
    const double ic = rsqrt(c2);
    const double c = c2 * ic;
    const double hb1 = 0.5 * gm1 * ic * ic;  // b1 / 2
    const double hb2 = 0.5 * u * u * hb1;    // b2 / 2
    const double uic = 0.5 * u * ic;
    const double hb1u = hb1 * u;
    L[0] = 0.5 * (hb2 + uic);
    L[1] = -0.5 * (hb1u + 0.5 * ic);
    L[2] = 0.5 * hb1;
    L[3] = 0.5 - hb2;
    L[4] = hb1u;
    L[5] = -hb1;
    L[6] = 0.5 * (hb2 - uic);
    L[7] = -0.5 * (hb1u - 0.5 * ic);
    L[8] = 0.5 * hb1;
    rs[0] = u;
    rs[1] = H;
    rs[2] = c;
  }

  // Roe's mean state and row `row` of the (1/2-scaled) left eigenvectors, the rows written as
  // one formula with row-dependent coefficients (no divergence between rows); rs as in roe
  __device__ __forceinline__ static void roe_row(double sa, double ua, double Ha, double sb, double ub, double Hb,
                                                 double gamma, int row, double* l, double* rs) {
    const double is = 1.0 / (sa + sb);
    const double wa = sa * is, wb = sb * is;
    const double u = dot2(wa, ua, wb, ub);
    const double H = dot2(wa, Ha, wb, Hb);
    const double gm1 = gamma - 1.0;
    const double c2 = gm1 * fma(-0.5 * u, u, H);
    const double ic = rsqrt(c2);
    const double hb1 = 0.5 * gm1 * ic * ic;
    const double hb2 = 0.5 * u * u * hb1;
    const double uic = 0.5 * u * ic;
    const double hb1u = hb1 * u;
    // rows: (0.5 (hb2 + uic), -0.5 hb1u - 0.25 ic, 0.5 hb1), (0.5 - hb2, hb1u, -hb1),
    //       (0.5 (hb2 - uic), -0.5 hb1u + 0.25 ic, 0.5 hb1)
    const double A = row == 1 ? -1.0 : 0.5, B = row == 0 ? 0.5 : (row == 1 ? 0.0 : -0.5);
    const double C = row == 1 ? 0.5 : 0.0, D = row == 1 ? 1.0 : -0.5;
    const double E = row == 0 ? -0.25 : (row == 1 ? 0.0 : 0.25), F = row == 1 ? -1.0 : 0.5;
    l[0] = fma(A, hb2, fma(B, uic, C));
    l[1] = fma(D, hb1u, E * ic);
    l[2] = F * hb1;
    rs[0] = u;
    rs[1] = H;
    rs[2] = c2 * ic;
  }

  __device__ __forceinline__ static void project3(const double* l, const double* f, const double* U, double alpha,
                                                  double& vp, double& vm) {
    const double a = fma(l[2], f[2], fma(l[1], f[1], l[0] * f[0]));
    const double b = fma(l[2], U[2], fma(l[1], U[1], l[0] * U[0]));
    vp = fma(alpha, b, a);
    vm = fma(-alpha, b, a);
  }
  __device__ __forceinline__ static void project1(double f, double u, double alpha, double& vp, double& vm) {
    const double hu = 0.5 * u;
    vp = fma(alpha, hu, 0.5 * f);
    vm = fma(-alpha, hu, 0.5 * f);
  }
  // the same projections in two parts: (a, b) = (l.f, l.u) before alpha is known, then v+-
  __device__ __forceinline__ static void project3_ab(const double* l, const double* f, const double* U, double& a,
                                                     double& b) {
    a = fma(l[2], f[2], fma(l[1], f[1], l[0] * f[0]));
    b = fma(l[2], U[2], fma(l[1], U[1], l[0] * U[0]));
  }
  // the l.u half of project3_ab alone, with the same operations
  __device__ __forceinline__ static double project3_b(const double* l, const double* U) {
    return fma(l[2], U[2], fma(l[1], U[1], l[0] * U[0]));
  }
  __device__ __forceinline__ static void project1_ab(double f, double u, double& a, double& b) {
    a = 0.5 * f;
    b = 0.5 * u;
  }
  __device__ __forceinline__ static void project_v(double a, double b, double alpha, double& vp, double& vm) {
    vp = fma(alpha, b, a);
    vm = fma(-alpha, b, a);
  }
  // Differences first (kDiffProj): with the products (da_k, db_k) = (l.(f_{k+1} - f_k),
  // l.(u_{k+1} - u_k)) of the cell differences of an interface's stencil cells 0..5 (the middle
  // one, k = 2, taken as the difference of the two centre cells' products (a2, b2), (a3, b3)),
  // the + side's stencil differences are d_k = da_k + alpha db_k and its q_2 = a2 + alpha b2;
  // the - side reads v- = a - alpha b mirrored, so d_k = alpha db_{4-k} - da_{4-k} and
  // q_2 = a3 - alpha b3.  (The thread pairs of the step-blocked tiles form the - side negated
  // instead, from products they already hold in that side's order.)
  static constexpr bool kDiffProj = true;
  __device__ __forceinline__ static void side_diffs(const double* da, const double* db, double a2, double b2,
                                                    double a3, double b3, double alpha, bool minus, double* d,
                                                    double& q2) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const double x = minus ? da[4 - k] : da[k];
      const double y = minus ? db[4 - k] : db[k];
      d[k] = fma(alpha, y, minus ? -x : x);
    }
    q2 = fma(minus ? -alpha : alpha, minus ? b3 : b2, minus ? a3 : a2);
  }
  // one side of project_v: v+ (minus false) or v- (minus true), the same value
  __device__ __forceinline__ static double project_side(double a, double b, double alpha, bool minus) {
    return fma(minus ? -alpha : alpha, b, a);
  }

  // The reconstruction in two parts.  weno_begin evaluates the sub-stencil values, the
  // indicators, tau and the theta switch; a restricted stencil (Eq. (be_res)) finishes there
  // with the linear combination (returns true, value in out).  Otherwise the nonlinear
  // weights of Eq. (om) are left to weno_finish, which needs only the record w.
  static constexpr bool kSplitWeno = true;
  struct WenoPart {
    double e[4];   // eps + beta_k
    double tau;    // tau^theta
    double fh[4];  // sub-stencil values
    bool theta1;
  };

  __device__ __forceinline__ static void gammas(bool theta1, double& g0, double& g1, double& g2, double& g3) {
    g0 = theta1 ? 2.0 / 20.0 : 1.0 / 20.0;
    g1 = theta1 ? 12.0 / 20.0 : 9.0 / 20.0;
    g2 = theta1 ? 6.0 / 20.0 : 9.0 / 20.0;
    g3 = theta1 ? 0.0 : 1.0 / 20.0;
  }

  // restricted stencil: the weights are gamma^theta (Eq. (gam_we6)) and sum_k gamma_k fh_k is
  // the linear scheme q2 + sum_j c_j (q_{j+1} - q_j) / 60; theta = 1: (-2, 11, 24, -3, 0),
  // theta = 0: (-1, 7, 30, -7, 1)
  __device__ __forceinline__ static double linear_theta(double d0, double d1, double d2, double d3, double d4,
                                                        double q2, bool theta1) {
    const double c0 = theta1 ? -2.0 / 60.0 : -1.0 / 60.0;
    const double c1 = theta1 ? 11.0 / 60.0 : 7.0 / 60.0;
    const double c2 = theta1 ? 24.0 / 60.0 : 30.0 / 60.0;
    const double c3 = theta1 ? -3.0 / 60.0 : -7.0 / 60.0;
    const double c4 = theta1 ? 0.0 : 1.0 / 60.0;
    return fma(c4, d4, fma(c3, d3, fma(c2, d2, fma(c1, d1, c0 * d0)))) + q2;
  }

  // |x| as the high word of its bit pattern (orders like |x| for finite x; inf and NaN top it)
  __device__ __forceinline__ static int hw(double x) { return __double2hiint(x) & 0x7fffffff; }
  // The high 32 bits of a double as a float: its sign, its exponent rebiased and the top 20
  // bits of its mantissa, so |hi32(x) - x| < 2^-20 |x|; 0 below 2^-126.  Integer pipe only;
  // the caller keeps |x| < 2^60.
  __device__ __forceinline__ static float hi32(double x) {
    const int hi = __double2hiint(x);
    const int mag = hi & 0x7fffffff;
    return mag < 0x38100000 ? 0.0f : __int_as_float(((mag - 0x38000000) << 3) | (hi & 0x80000000));
  }

  // FP32 screen of the two decisions of a stencil: the restriction test of Eq. (be_res) and
  // theta of Eq. (tau_we6), from the FP64 differences s0..s3, d1..d3 and the large-stencil
  // terms t5a, t5b, t6a, t6b.  Returns 1 (restricted, theta = 1) or 2 (restricted, theta = 0)
  // only where an error bound proves that the FP64 evaluation decides the same, else 0.
  // Bound: each FP32 input is within 2^-20 of its FP64 value, so each indicator computed in
  // FP32 is within 2^-15 S^2 of its value from the FP64 inputs (S the largest input; at
  // most 21 * 2^-20 S^2 for beta_3), and tau5, tau6 (sums of squares) within 2.3 * 2^-20 of
  // theirs; the FP64 evaluation is within a few 2^-53 of the same values.  The restriction
  // is taken as proven with the indicators moved by 2^-14 S^2 against it and a further
  // 2^-18 of slack for the FP32 rounding of the test; theta with a gap above 2^-16 of the
  // larger tau, which must exceed 2^-120 so that subnormal rounding (2^-149 per operation)
  // stays far below the gap.
  __device__ __forceinline__ static int screen(double s0, double s1, double s2, double s3, double d1, double d2,
                                               double d3, double t5a, double t5b, double t6a, double t6b, double eps,
                                               double alpha_R) {
    int hm = max(max(max(hw(s0), hw(s1)), max(hw(s2), hw(s3))), max(max(hw(d1), hw(d2)), hw(d3)));
    hm = max(hm, max(max(hw(t5a), hw(t5b)), max(hw(t6a), hw(t6b))));
    hm = max(hm, hw(alpha_R));
    if (hm >= 0x43b00000) return 0;  // some input at or beyond 2^60, or not finite
    constexpr float F1312 = 13.0f / 12.0f, F1348 = 13.0f / 48.0f;
    const float a0 = hi32(s0), a1 = hi32(s1), a2 = hi32(s2), a3 = hi32(s3);
    const float x1 = hi32(d1), x2 = hi32(d2), x3 = hi32(d3);
    const float e0 = a0 + x1, g3 = fmaf(3.0f, a2, -a3), e3 = a3 - x3, dd = x2 * x2;
    const float b0 = fmaf(F1312 * a0, a0, e0 * e0);
    const float b1 = fmaf(F1312 * a1, a1, dd);
    const float b2 = fmaf(F1312 * a2, a2, dd);
    const float b3 = fmaf(F1348 * g3, g3, e3 * e3);
    const float sg = fmaxf(fmaxf(fmaxf(fabsf(a0), fabsf(a1)), fmaxf(fabsf(a2), fabsf(a3))),
                           fmaxf(fmaxf(fabsf(x1), fabsf(x2)), fabsf(x3)));
    const float del = 0x1p-14f * (sg * sg);
    const float bmax = fmaxf(fmaxf(b0, b1), fmaxf(b2, b3)), bmin = fminf(fminf(b0, b1), fminf(b2, b3));
    const float aR = hi32(alpha_R), ef = hi32(eps);
    if (!(aR * ef > 1e-30f)) return 0;
    if (!((bmax + del) < aR * (ef + (bmin - del)) * (1.0f - 0x1p-18f))) return 0;
    const float u5a = hi32(t5a), u5b = hi32(t5b), u6a = hi32(t6a), u6b = hi32(t6b);
    const float tau5 = fmaf(F1312 * u5a, u5a, u5b * u5b);
    const float tau6 = fmaf(F1312 * u6a, u6a, 0.25f * (u6b * u6b));
    const float tm = fmaxf(tau5, tau6);
    if (tm > 0x1p-120f && fabsf(tau6 - tau5) > 0x1p-16f * tm) return (tau6 < tau5) ? 2 : 1;
    // every large-stencil term zero: tau5 = tau6 = 0 in FP64 too, a tie, theta = 1
    if (((bits(t5a) | bits(t5b) | bits(t6a) | bits(t6b)) << 1) == 0) return 1;
    return 0;
  }

  __device__ __forceinline__ static bool weno_begin(const double* q, double eps, double alpha_R, double& out,
                                                    WenoPart& w) {
    const double d0 = q[1] - q[0], d1 = q[2] - q[1], d2 = q[3] - q[2], d3 = q[4] - q[3], d4 = q[5] - q[4];
    return weno_core<false>(d0, d1, d2, d3, d4, q[2], q[3], eps, alpha_R, out, w);
  }
  // the same from the stencil's differences d_k = q_{k+1} - q_k and q_2 (q_3 taken as q_2 + d_2)
  __device__ __forceinline__ static bool weno_begin_d(const double* d, double q2, double eps, double alpha_R,
                                                      double& out, WenoPart& w) {
    return weno_core<true>(d[0], d[1], d[2], d[3], d[4], q2, 0.0, eps, alpha_R, out, w);
  }
  template <bool Q3D>
  __device__ __forceinline__ static bool weno_core(double d0, double d1, double d2, double d3, double d4, double q2,
                                                   double q3, double eps, double alpha_R, double& out, WenoPart& w) {
    constexpr double C1312 = 13.0 / 12.0, C1348 = 13.0 / 48.0;
    const double s0 = d1 - d0, s1 = d2 - d1, s2 = d3 - d2, s3 = d4 - d3;
    // the large-stencil terms of Eqs. (tau_5), (tau_6)
    const double t5b = s2 - s1;                // -q1 + 3 q2 - 3 q3 + q4
    const double t5a = fma(-2.0, s1, s0) + s2; // q0 - 4 q1 + 6 q2 - 4 q3 + q4
    const double t6a = fma(-3.0, t5b, s3 - s0);      // fifth difference
    const double t6b = (s0 + s3) - (s1 + s2);        // q0 - 3 q1 + 2 q2 + 2 q3 - 3 q4 + q5
    // the decisions, where FP32 proves them: no FP64 indicator is needed
    const int scr = screen(s0, s1, s2, s3, d1, d2, d3, t5a, t5b, t6a, t6b, eps, alpha_R);
    if (scr != 0) {
      w.theta1 = scr == 1;
      out = linear_theta(d0, d1, d2, d3, d4, q2, w.theta1);
      return true;
    }
    // Eqs. (be0_cen)-(be3_cen)
    const double e0 = s0 + d1;                 // q0 - 3 q1 + 2 q2
    const double dd = d2 * d2;                 // (q3 - q2)^2, shared by beta_1 and beta_2
    const double g3 = fma(3.0, s2, -s3);       // 3 q2 - 7 q3 + 5 q4 - q5
    const double e3 = s3 - d3;                 // 2 q3 - 3 q4 + q5
    const double b0 = fma(C1312 * s0, s0, e0 * e0);
    const double b1 = fma(C1312 * s1, s1, dd);
    const double b2 = fma(C1312 * s2, s2, dd);
    const double b3 = fma(C1348 * g3, g3, e3 * e3);
    // Eqs. (tau_5), (tau_6)
    const double tau5 = fma(C1312 * t5a, t5a, t5b * t5b);
    const double tau6 = fma(C1312 * t6a, t6a, 0.25 * (t6b * t6b));
    // Eq. (tau_we6)
    w.theta1 = !(bits(tau6) < bits(tau5));
    w.tau = w.theta1 ? tau5 : tau6;
    // Eq. (be_res)
    const double bmax = nmax(nmax(b0, b1), nmax(b2, b3));
    const double bmin = nmin(nmin(b0, b1), nmin(b2, b3));
    if (!(bits(fma(alpha_R, bmin, alpha_R * eps)) < bits(bmax))) {
      out = linear_theta(d0, d1, d2, d3, d4, q2, w.theta1);
      return true;
    }
    // Eqs. (fh0)-(fh3) in difference form
    w.fh[0] = fma(5.0 / 6.0, d1, fma(-1.0 / 3.0, d0, q2));
    w.fh[1] = fma(1.0 / 6.0, d1, fma(1.0 / 3.0, d2, q2));
    w.fh[2] = fma(2.0 / 3.0, d2, fma(-1.0 / 6.0, d3, q2));
    w.fh[3] = fma(1.0 / 3.0, d4, fma(-5.0 / 6.0, d3, Q3D ? q2 + d2 : q3));
    w.e[0] = eps + b0;
    w.e[1] = eps + b1;
    w.e[2] = eps + b2;
    w.e[3] = eps + b3;
    return false;
  }

  // ---- The reconstruction in a front and a back half, for the step-blocked kernel.
  // weno_front takes the differences, the large-stencil terms and the FP32 screen; a screened
  // stencil finishes there (linear scheme, returns true).  Any other stencil leaves a record of
  // kDeferRec doubles (d0..d4, s0..s3, t5a, t5b, t6a, t6b, q2, q3) that a quad of lanes
  // completes in weno_back_quad with the operations of weno_begin's FP64 path and of
  // weno_finish, so the value is the same as theirs.
  static constexpr int kDeferRec = 15;
  __device__ __forceinline__ static bool weno_front(const double* q, double eps, double alpha_R, double& out,
                                                    double* rec) {
    const double d0 = q[1] - q[0], d1 = q[2] - q[1], d2 = q[3] - q[2], d3 = q[4] - q[3], d4 = q[5] - q[4];
    return weno_front_core<false>(d0, d1, d2, d3, d4, q[2], q[3], eps, alpha_R, out, rec);
  }
  // the same from the stencil's differences and q_2 (q_3 taken as q_2 + d_2)
  __device__ __forceinline__ static bool weno_front_d(const double* d, double q2, double eps, double alpha_R,
                                                      double& out, double* rec) {
    return weno_front_core<true>(d[0], d[1], d[2], d[3], d[4], q2, 0.0, eps, alpha_R, out, rec);
  }
  template <bool Q3D>
  __device__ __forceinline__ static bool weno_front_core(double d0, double d1, double d2, double d3, double d4,
                                                         double q2, double q3, double eps, double alpha_R,
                                                         double& out, double* rec) {
    const double s0 = d1 - d0, s1 = d2 - d1, s2 = d3 - d2, s3 = d4 - d3;
    const double t5b = s2 - s1;
    const double t5a = fma(-2.0, s1, s0) + s2;
    const double t6a = fma(-3.0, t5b, s3 - s0);
    const double t6b = (s0 + s3) - (s1 + s2);
    const int scr = screen(s0, s1, s2, s3, d1, d2, d3, t5a, t5b, t6a, t6b, eps, alpha_R);
    if (scr != 0) {
      out = linear_theta(d0, d1, d2, d3, d4, q2, scr == 1);
      return true;
    }
    rec[0] = d0; rec[1] = d1; rec[2] = d2; rec[3] = d3; rec[4] = d4;
    rec[5] = s0; rec[6] = s1; rec[7] = s2; rec[8] = s3;
    rec[9] = t5a; rec[10] = t5b; rec[11] = t6a; rec[12] = t6b;
    rec[13] = q2; rec[14] = Q3D ? q2 + d2 : q3;
    return false;
  }

  // Lane k (0..3) of the quad of lanes `qmask` completes a deferred stencil: indicator k
  // (Eqs. (be0_cen)-(be3_cen)), the four shared by shuffles, tau5, tau6 and theta, the
  // restriction test, then either the linear scheme or weight k and the quad's sums.  The
  // result is valid in lane 0 of the quad.  Every lane of the quad must call it.
  __device__ __forceinline__ static double weno_back_quad(int k, const double* r, double eps, double alpha_R,
                                                          unsigned qmask) {
    constexpr double C1312 = 13.0 / 12.0, C1348 = 13.0 / 48.0;
    const double d0 = r[0], d1 = r[1], d2 = r[2], d3 = r[3], d4 = r[4];
    const double s0 = r[5], s1 = r[6], s2 = r[7], s3 = r[8];
    const double t5a = r[9], t5b = r[10], t6a = r[11], t6b = r[12], q2 = r[13], q3 = r[14];
    const double e0 = s0 + d1;
    const double g3 = fma(3.0, s2, -s3);
    const double e3 = s3 - d3;
    // indicator k as fma(C x, x, y y): (s0, e0), (s1, d2), (s2, d2), (g3, e3) with 13/48 for k = 3
    const double x = k == 0 ? s0 : (k == 1 ? s1 : (k == 2 ? s2 : g3));
    const double y = k == 0 ? e0 : (k == 3 ? e3 : d2);
    const double bk = fma((k == 3 ? C1348 : C1312) * x, x, y * y);
    const double x1 = __shfl_xor_sync(qmask, bk, 1), x2 = __shfl_xor_sync(qmask, bk, 2),
                 x3 = __shfl_xor_sync(qmask, bk, 3);
    // indicator j comes from the lane at xor distance j ^ k
    const double b0 = k == 0 ? bk : (k == 1 ? x1 : (k == 2 ? x2 : x3));
    const double b1 = k == 1 ? bk : (k == 0 ? x1 : (k == 3 ? x2 : x3));
    const double b2 = k == 2 ? bk : (k == 3 ? x1 : (k == 0 ? x2 : x3));
    const double b3 = k == 3 ? bk : (k == 2 ? x1 : (k == 1 ? x2 : x3));
    const double tau5 = fma(C1312 * t5a, t5a, t5b * t5b);
    const double tau6 = fma(C1312 * t6a, t6a, 0.25 * (t6b * t6b));
    const bool theta1 = !(bits(tau6) < bits(tau5));
    const double tau = theta1 ? tau5 : tau6;
    const double bmax = nmax(nmax(b0, b1), nmax(b2, b3));
    const double bmin = nmin(nmin(b0, b1), nmin(b2, b3));
    if (!(bits(fma(alpha_R, bmin, alpha_R * eps)) < bits(bmax))) return linear_theta(d0, d1, d2, d3, d4, q2, theta1);
    // Eqs. (fh0)-(fh3): fh_k = fma(A, X, fma(B, Y, Z))
    const double A = k == 0 ? 5.0 / 6.0 : (k == 1 ? 1.0 / 6.0 : (k == 2 ? 2.0 / 3.0 : 1.0 / 3.0));
    const double X = k == 0 ? d1 : (k == 1 ? d1 : (k == 2 ? d2 : d4));
    const double B = k == 0 ? -1.0 / 3.0 : (k == 1 ? 1.0 / 3.0 : (k == 2 ? -1.0 / 6.0 : -5.0 / 6.0));
    const double Y = k == 0 ? d0 : (k == 1 ? d2 : d3);
    const double Z = k == 3 ? q3 : q2;
    const double fhk = fma(A, X, fma(B, Y, Z));
    const double e[4] = {eps + b0, eps + b1, eps + b2, eps + b3};
    double wk, nk;
    weno_weight(k, e, tau, theta1, fhk, wk, nk);
    wk += __shfl_xor_sync(qmask, wk, 1);
    nk += __shfl_xor_sync(qmask, nk, 1);
    wk += __shfl_xor_sync(qmask, wk, 2);
    nk += __shfl_xor_sync(qmask, nk, 2);
    return nk / wk;
  }

  // Eq. (om) over the common denominator prod_l (eps + beta_l)
  __device__ __forceinline__ static double weno_finish(const WenoPart& w) {
    double g0, g1, g2, g3;
    gammas(w.theta1, g0, g1, g2, g3);
    const double p01 = w.e[0] * w.e[1], p23 = w.e[2] * w.e[3];
    const double w0 = g0 * (w.e[0] + w.tau) * (w.e[1] * p23);
    const double w1 = g1 * (w.e[1] + w.tau) * (w.e[0] * p23);
    const double w2 = g2 * (w.e[2] + w.tau) * (p01 * w.e[3]);
    const double w3 = g3 * (w.e[3] + w.tau) * (p01 * w.e[2]);
    // numerator and denominator summed in pairs, products rounded on their own: the order
    // in which a quad of lanes sums them (weno_weight), so every kernel gets the same value
    const double num = __dadd_rn(__dadd_rn(__dmul_rn(w0, w.fh[0]), __dmul_rn(w1, w.fh[1])),
                                 __dadd_rn(__dmul_rn(w2, w.fh[2]), __dmul_rn(w3, w.fh[3])));
    return num / ((w0 + w1) + (w2 + w3));
  }

  // Weight k of Eq. (om) over the common denominator, exactly as weno_finish forms it, and its
  // term of the numerator; a quad of lanes forms the four and sums them (see stage1d_compute)
  __device__ __forceinline__ static void weno_weight(int k, const double* e, double tau, bool theta1, double fhk,
                                                     double& wk, double& nk) {
    double g0, g1, g2, g3;
    gammas(theta1, g0, g1, g2, g3);
    const double gk = k == 0 ? g0 : (k == 1 ? g1 : (k == 2 ? g2 : g3));
    const double ek = k == 0 ? e[0] : (k == 1 ? e[1] : (k == 2 ? e[2] : e[3]));
    // the product of the other three: e1 p23, e0 p23, p01 e3, p01 e2
    const double pa = (k == 0) ? e[1] : ((k == 1) ? e[0] : e[0] * e[1]);
    const double pb = (k < 2) ? e[2] * e[3] : ((k == 2) ? e[3] : e[2]);
    wk = gk * (ek + tau) * (pa * pb);
    nk = __dmul_rn(wk, fhk);
  }

  __device__ __forceinline__ static double weno_flags(const double* q, double eps, double alpha_R, bool& restricted_out,
                                                    bool& theta1_out) {
    WenoPart w;
    double out;
    restricted_out = weno_begin(q, eps, alpha_R, out, w);
    theta1_out = w.theta1;
    return restricted_out ? out : weno_finish(w);
  }

  __device__ __forceinline__ static double weno(const double* q, double eps, double alpha_R) {
    bool r, t;
    return weno_flags(q, eps, alpha_R, r, t);
  }
  __device__ __forceinline__ static double weno_d(const double* d, double q2, double eps, double alpha_R) {
    WenoPart w;
    double out;
    return weno_begin_d(d, q2, eps, alpha_R, out, w) ? out : weno_finish(w);
  }

  __device__ __forceinline__ static void backproject(const double* rs, const double* F, double* h) {
    const double u = rs[0], H = rs[1], c = rs[2];
    const double s02 = F[0] + F[2], d20 = F[2] - F[0];
    h[0] = s02 + F[1];
    h[1] = fma(u, h[0], c * d20);
    h[2] = fma(H, s02, fma(u * c, d20, 0.5 * u * u * F[1]));
  }

  // rounded on its own (never contracted into the sum of the two sweeps), so that
  // Lx + Ly is the same value for transposed data
  __device__ __forceinline__ static double flux_diff(double hp, double hm, double, double inv_dx) {
    return __dmul_rn(hm - hp, inv_dx);
  }

  template <int S>
  __device__ __forceinline__ static double rk(double un, double us, double dt, double L) {
    if (S == 0) return fma(dt, L, un);
    if (S == 1) return fma(0.25, fma(dt, L, us), 0.75 * un);
    return fma(2.0 / 3.0, fma(dt, L, us), (1.0 / 3.0) * un);
  }

  __device__ __forceinline__ static double cfl_dt(double cfl, double dx, double smax) { return cfl * dx / smax; }

  // ================================ 2D Euler (Sec. 4.3) ================================
  __device__ __forceinline__ static void euler2d_cell(const double* U, double gamma, double* f, double* g, double& u,
                                                      double& v, double& H, double& sr) {
    const double ir = 1.0 / U[0];
    u = U[1] * ir;
    v = U[2] * ir;
    const double p = __dmul_rn(gamma - 1.0, fma(-0.5, dot2(U[1], u, U[2], v), U[3]));
    const double e = __dadd_rn(U[3], p);
    f[0] = U[1];
    f[1] = fma(U[1], u, p);
    f[2] = U[1] * v;
    f[3] = e * u;
    g[0] = U[2];
    g[1] = U[2] * u;  // rho v u, computed as the transpose of f[2]
    g[2] = fma(U[2], v, p);
    g[3] = e * v;
    H = e * ir;
    sr = sqrt(U[0]);
  }
  // g of euler2d_cell alone, from the u and v it returned (the same operations; p and e are
  // rounded explicitly in both, so that neither is contracted differently at either site)
  __device__ __forceinline__ static void euler2d_gflux(const double* U, double u, double v, double gamma, double* g) {
    const double p = __dmul_rn(gamma - 1.0, fma(-0.5, dot2(U[1], u, U[2], v), U[3]));
    const double e = __dadd_rn(U[3], p);
    g[0] = U[2];
    g[1] = U[2] * u;  // rho v u, computed as the transpose of f[2]
    g[2] = fma(U[2], v, p);
    g[3] = e * v;
  }

  __device__ __forceinline__ static void euler2d_speeds(const double* U, double gamma, double dx, double dy,
                                                        double* lx, double* ly, double& q) {
    const double ir = 1.0 / U[0];
    const double u = U[1] * ir, v = U[2] * ir;
    const double p = (gamma - 1.0) * fma(-0.5, dot2(U[1], u, U[2], v), U[3]);
    const double c = sqrt(gamma * p * ir);
    const double au = fabs(u), av = fabs(v);
    lx[0] = fabs(u - c);
    lx[1] = au;
    lx[2] = au;
    lx[3] = fabs(u + c);
    ly[0] = fabs(v - c);
    ly[1] = av;
    ly[2] = av;
    ly[3] = fabs(v + c);
    q = (au + c) / dx + (av + c) / dy;
  }

  // L pre-scaled by 1/2 (the factor of Eq. (flux_split_lf))
  __device__ __forceinline__ static void roe2d(int dir, double sa, double ua, double va, double Ha, double sb,
                                               double ub, double vb, double Hb, double gamma, double* L, double* rs) {
    const double is = 1.0 / (sa + sb);
    const double wa = sa * is, wb = sb * is;
    const double u = dot2(wa, ua, wb, ub);
    const double v = dot2(wa, va, wb, vb);
    const double H = dot2(wa, Ha, wb, Hb);
    const double q2 = dot2(u, u, v, v);
    const double gm1 = gamma - 1.0;
    const double c2 = gm1 * fma(-0.5, q2, H);
    const double ic = rsqrt(c2);
    const double c = c2 * ic;
    const double hb1 = 0.5 * gm1 * ic * ic;
    const double hb2 = 0.5 * q2 * hb1;
    const double w = dir == 0 ? u : v;
    const double wic = 0.5 * w * ic;
    const double hb1u = hb1 * u, hb1v = hb1 * v;
    if (dir == 0) {
      L[0] = 0.5 * (hb2 + wic); L[1] = -0.5 * (hb1u + 0.5 * ic); L[2] = -0.5 * hb1v; L[3] = 0.5 * hb1;
      L[12] = 0.5 * (hb2 - wic); L[13] = -0.5 * (hb1u - 0.5 * ic); L[14] = -0.5 * hb1v; L[15] = 0.5 * hb1;
      L[8] = -0.5 * v; L[9] = 0.0; L[10] = 0.5; L[11] = 0.0;
    } else {
      L[0] = 0.5 * (hb2 + wic); L[1] = -0.5 * hb1u; L[2] = -0.5 * (hb1v + 0.5 * ic); L[3] = 0.5 * hb1;
      L[12] = 0.5 * (hb2 - wic); L[13] = -0.5 * hb1u; L[14] = -0.5 * (hb1v - 0.5 * ic); L[15] = 0.5 * hb1;
      L[8] = -0.5 * u; L[9] = 0.5; L[10] = 0.0; L[11] = 0.0;
    }
    L[4] = 0.5 - hb2;
    L[5] = hb1u;
    L[6] = hb1v;
    L[7] = -hb1;
    rs[0] = u;
    rs[1] = v;
    rs[2] = H;
    rs[3] = c;
  }

  // density, normal momentum, tangential momentum, energy: the same order in both directions
  __device__ __forceinline__ static void project4(int dir, const double* l, const double* f, const double* U,
                                                  double alpha, double& vp, double& vm) {
    const int n = 1 + dir, t = 2 - dir;
    const double a = fma(l[3], f[3], fma(l[t], f[t], fma(l[n], f[n], l[0] * f[0])));
    const double b = fma(l[3], U[3], fma(l[t], U[t], fma(l[n], U[n], l[0] * U[0])));
    vp = fma(alpha, b, a);
    vm = fma(-alpha, b, a);
  }

  __device__ __forceinline__ static void backproject2d(int dir, const double* rs, const double* F, double* h) {
    const double u = rs[0], v = rs[1], H = rs[2], c = rs[3];
    const double s03 = F[0] + F[3], d30 = F[3] - F[0];
    const double a = s03 + F[1];
    h[0] = a;
    const double hq2 = 0.5 * dot2(u, u, v, v);
    if (dir == 0) {
      h[1] = fma(u, a, c * d30);
      h[2] = fma(v, a, F[2]);
      h[3] = fma(H, s03, fma(u * c, d30, fma(hq2, F[1], v * F[2])));
    } else {
      h[1] = fma(u, a, F[2]);
      h[2] = fma(v, a, c * d30);
      h[3] = fma(H, s03, fma(v * c, d30, fma(hq2, F[1], u * F[2])));
    }
  }

  __device__ __forceinline__ static double add_sweeps(double Lx, double Ly) { return Lx + Ly; }
  // L + (-g q): a source term -g q added to the flux divergence
  __device__ __forceinline__ static double add_source(double L, double g, double q) { return fma(-g, q, L); }
  __device__ __forceinline__ static double cfl_dt_2d(double cfl, double smax) { return cfl / smax; }
};

}  // namespace wt
