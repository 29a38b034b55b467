// Discrete adjoint of the 1D Euler hot path (reverse mode of the exact map the forward pass
// computes).  Every branch is frozen where the forward pass took it: theta and the
// restriction of each reconstruction are re-decided by the same arithmetic policy as the
// forward, and the derivative of each maximum (the Lax-Friedrichs alphas, the CFL step)
// goes to the first cell that attains it.
//
//   adj_stage_kernel   one RK stage in reverse over a tile: recomputes the stage's interface
//                      fluxes, then reverses back-projection, both WENO-theta
//                      reconstructions, the Lax-Friedrichs split and projection and Roe's
//                      average per interface; writes 36 contributions per interface (to the
//                      physical fluxes and to the states of its six cells) and per-tile
//                      partial sums of d/d alpha and d/d dt
//   adj_gather_kernel  per cell, in a fixed order: sums the contributions of the interfaces
//                      whose stencils (ghost cells mapped through the boundary conditions)
//                      contain it, applies the flux Jacobian, and combines the RK weights
//   adj_argmax_kernel, adj_reduce_apply_kernel
//                      first-index argmax cells of the alphas and of max(|u| + c), and the
//                      rank-one updates that carry d/d alpha and d/d dt back to them
#pragma once

#include "wt_kernels.cuh"

namespace wt {

// ---------------------------------------------------------------------------------------
// Derivative building blocks
// ---------------------------------------------------------------------------------------

// qbar += Fbar * dF/dq for the WENO-theta value F(q) of Eqs. (fh_nonlinear)-(tau_we6), with the
// restriction of Eq. (be_res) and the theta of Eq. (tau_we6) frozen as given.  A restricted
// stencil has every alpha_k scaled by the same factor 1 + tau/eps, so its weights are the
// linear gamma^theta and dF/dq is the coefficient vector of Eq. (fh_5) (theta = 1) or
// Eq. (fh_6) (theta = 0).
__device__ __forceinline__ void weno_grad(const double* q, double eps, bool restricted, bool theta1, double Fbar,
                                          double* qbar) {
  if (restricted) {
    if (theta1) {
      constexpr double c5[6] = {2.0 / 60, -13.0 / 60, 47.0 / 60, 27.0 / 60, -3.0 / 60, 0.0};
#pragma unroll
      for (int i = 0; i < 5; ++i) qbar[i] = fma(c5[i], Fbar, qbar[i]);
    } else {
      constexpr double c6[6] = {1.0 / 60, -8.0 / 60, 37.0 / 60, 37.0 / 60, -8.0 / 60, 1.0 / 60};
#pragma unroll
      for (int i = 0; i < 6; ++i) qbar[i] = fma(c6[i], Fbar, qbar[i]);
    }
    return;
  }
  constexpr double C12 = 13.0 / 12.0, C48 = 13.0 / 48.0;
  constexpr double cfh[4][6] = {{2.0 / 6, -7.0 / 6, 11.0 / 6, 0, 0, 0},
                                {0, -1.0 / 6, 5.0 / 6, 2.0 / 6, 0, 0},
                                {0, 0, 2.0 / 6, 5.0 / 6, -1.0 / 6, 0},
                                {0, 0, 0, 11.0 / 6, -7.0 / 6, 2.0 / 6}};
  // beta_k = cb_k x_k^2 + y_k^2 with x_k = vx_k . q, y_k = vy_k . q
  constexpr double vx[4][6] = {{1, -2, 1, 0, 0, 0}, {0, 1, -2, 1, 0, 0}, {0, 0, 1, -2, 1, 0}, {0, 0, 3, -7, 5, -1}};
  constexpr double vy[4][6] = {{1, -3, 2, 0, 0, 0}, {0, 0, -1, 1, 0, 0}, {0, 0, 1, -1, 0, 0}, {0, 0, 0, 2, -3, 1}};
  constexpr double cb[4] = {C12, C12, C12, C48};
  constexpr double v5x[6] = {1, -4, 6, -4, 1, 0}, v5y[6] = {0, -1, 3, -3, 1, 0};
  constexpr double v6x[6] = {-1, 5, -10, 10, -5, 1}, v6y[6] = {1, -3, 2, 2, -3, 1};
  double fh[4], xb[4], yb[4], beta[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double f = 0, x = 0, y = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (cfh[k][i] != 0.0) f = fma(cfh[k][i], q[i], f);
      if (vx[k][i] != 0.0) x = fma(vx[k][i], q[i], x);
      if (vy[k][i] != 0.0) y = fma(vy[k][i], q[i], y);
    }
    fh[k] = f;
    xb[k] = x;
    yb[k] = y;
    beta[k] = fma(cb[k] * x, x, y * y);
  }
  double xt = 0, yt = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (theta1) {
      if (v5x[i] != 0.0) xt = fma(v5x[i], q[i], xt);
      if (v5y[i] != 0.0) yt = fma(v5y[i], q[i], yt);
    } else {
      if (v6x[i] != 0.0) xt = fma(v6x[i], q[i], xt);
      if (v6y[i] != 0.0) yt = fma(v6y[i], q[i], yt);
    }
  }
  const double tau = theta1 ? fma(C12 * xt, xt, yt * yt) : fma(C12 * xt, xt, 0.25 * yt * yt);
  const double g[4] = {theta1 ? 2.0 / 20.0 : 1.0 / 20.0, theta1 ? 12.0 / 20.0 : 9.0 / 20.0,
                       theta1 ? 6.0 / 20.0 : 9.0 / 20.0, theta1 ? 0.0 : 1.0 / 20.0};
  // 1 / (eps + beta_k) from one division: the product of the four, times the other three
  double d[4], id[4], a[4], S = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k] = eps + beta[k];
  const double p01 = d[0] * d[1], p23 = d[2] * d[3], ip = 1.0 / (p01 * p23);
  id[0] = d[1] * p23 * ip;
  id[1] = d[0] * p23 * ip;
  id[2] = p01 * d[3] * ip;
  id[3] = p01 * d[2] * ip;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = g[k] * fma(tau, id[k], 1.0);
    S += a[k];
  }
  const double iS = 1.0 / S;
  double F = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) F = fma(a[k] * iS, fh[k], F);
  double taub = 0, fhb[4], xbb[4], ybb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double ab = Fbar * (fh[k] - F) * iS;  // adjoint of a_k
    taub = fma(ab * g[k], id[k], taub);
    const double bbk = -ab * g[k] * tau * id[k] * id[k];  // adjoint of beta_k
    xbb[k] = 2.0 * cb[k] * xb[k] * bbk;
    ybb[k] = 2.0 * yb[k] * bbk;
    fhb[k] = Fbar * a[k] * iS;
  }
  const double xtb = 2.0 * C12 * xt * taub, ytb = (theta1 ? 2.0 : 0.5) * yt * taub;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double s = qbar[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (cfh[k][i] != 0.0) s = fma(cfh[k][i], fhb[k], s);
      if (vx[k][i] != 0.0) s = fma(vx[k][i], xbb[k], s);
      if (vy[k][i] != 0.0) s = fma(vy[k][i], ybb[k], s);
    }
    if (theta1) {
      if (v5x[i] != 0.0) s = fma(v5x[i], xtb, s);
      if (v5y[i] != 0.0) s = fma(v5y[i], ytb, s);
    } else {
      if (v6x[i] != 0.0) s = fma(v6x[i], xtb, s);
      if (v6y[i] != 0.0) s = fma(v6y[i], ytb, s);
    }
    qbar[i] = s;
  }
}

// Ubar += A(U)^T fbar with A the Jacobian of the 1D Euler flux (Sec. 4.2).
__device__ __forceinline__ void euler_flux_jt(const double* U, double gamma, const double* fb, double* Ub) {
  const double ir = 1.0 / U[0], u = U[1] * ir, e = U[2] * ir, gm1 = gamma - 1.0;
  Ub[0] += -0.5 * (3.0 - gamma) * u * u * fb[1] + (-gamma * e * u + gm1 * u * u * u) * fb[2];
  Ub[1] += fb[0] + (3.0 - gamma) * u * fb[1] + (gamma * e - 1.5 * gm1 * u * u) * fb[2];
  Ub[2] += gm1 * fb[1] + gamma * u * fb[2];
}

// gradients of u, c with respect to (rho, m, E) at a cell
__device__ __forceinline__ void euler_uc_grad(const double* U, double gamma, double* du, double* dc) {
  const double rho = U[0], u = U[1] / rho, gm1 = gamma - 1.0;
  const double p = gm1 * (U[2] - 0.5 * U[1] * u);
  const double c = sqrt(gamma * p / rho);
  du[0] = -u / rho;
  du[1] = 1.0 / rho;
  du[2] = 0.0;
  const double k = gamma / (2.0 * c * rho);
  dc[0] = k * (0.5 * gm1 * u * u - p / rho);
  dc[1] = -k * gm1 * u;
  dc[2] = k * gm1;
}

// Reverse of Roe's average and the eigenvectors: true Lbar (3x3) and Rbar (3x3, R[c][s]) of
// the interface between cells a and b -> Ubar_a, Ubar_b.
// ira, irb: 1 / rho of the two cells.
__device__ __forceinline__ void roe_reverse(const double* Ua, const double* Ub, double sa, double ua, double Ha,
                                            double ira, double sb, double ub, double Hb, double irb, const double* rs,
                                            double gamma, const double* Lb, const double* Rb, double* Uab,
                                            double* Ubb) {
  // reciprocals from square roots (an IEEE division costs about nine FMA slots of the narrow
  // FP64 pipe): 1 / c from c^2 = (gamma - 1)(H - u^2 / 2), and the cells' 1 / rho given
  const double u = rs[0], H = rs[1], c = rs[2], gm1 = gamma - 1.0;
  const double ic = rsqrt(gm1 * fma(-0.5 * u, u, H)), ic2 = ic * ic;
  const double b1 = gm1 * ic2;
  double ubar = 0, cbar = 0, Hbar = 0, b1b = 0, b2b = 0, r1b = 0, r2b = 0;
  b2b += 0.5 * Lb[0];
  r1b += 0.5 * Lb[0];
  b1b += -0.5 * u * Lb[1];
  ubar += -0.5 * b1 * Lb[1];
  r2b += -0.5 * Lb[1];
  b1b += 0.5 * Lb[2];
  b2b -= Lb[3];
  b1b += u * Lb[4];
  ubar += b1 * Lb[4];
  b1b -= Lb[5];
  b2b += 0.5 * Lb[6];
  r1b -= 0.5 * Lb[6];
  b1b += -0.5 * u * Lb[7];
  ubar += -0.5 * b1 * Lb[7];
  r2b += 0.5 * Lb[7];
  b1b += 0.5 * Lb[8];
  b1b += 0.5 * u * u * b2b;  // b2 = u^2 b1 / 2
  ubar += u * b1 * b2b;
  ubar += r1b * ic;  // r1 = u / c
  cbar += -r1b * u * ic2;
  cbar += -r2b * ic2;  // r2 = 1 / c
  cbar += b1b * (-2.0 * gm1 * ic2 * ic);
  // R: rows (1,1,1), (u-c, u, u+c), (H-uc, u^2/2, H+uc)
  ubar += Rb[3] + Rb[4] + Rb[5] + u * Rb[7] - c * Rb[6] + c * Rb[8];
  cbar += -Rb[3] + Rb[5] - u * Rb[6] + u * Rb[8];
  Hbar += Rb[6] + Rb[8];
  // c^2 = (gamma - 1)(H - u^2 / 2)
  const double c2b = 0.5 * cbar * ic;
  Hbar += gm1 * c2b;
  ubar += -gm1 * u * c2b;
  // u~ = (sa ua + sb ub) / D, H~ = (sa Ha + sb Hb) / D
  const double iD = 1.0 / (sa + sb);
  const double uab = ubar * sa * iD, ubb = ubar * sb * iD, Hab = Hbar * sa * iD, Hbb = Hbar * sb * iD;
  const double sab = (ubar * (ua - u) + Hbar * (Ha - H)) * iD;
  const double sbb = (ubar * (ub - u) + Hbar * (Hb - H)) * iD;
  // per cell: u = m / rho, H = gamma E / rho - (gamma - 1) u^2 / 2, s = sqrt(rho); 1/s = s / rho
  {
    const double ir = ira, E = Ua[2];
    Uab[0] += uab * (-ua * ir) + Hab * ((-gamma * E * ir + gm1 * ua * ua) * ir) + 0.5 * sab * sa * ir;
    Uab[1] += uab * ir + Hab * (-gm1 * ua * ir);
    Uab[2] += Hab * gamma * ir;
  }
  {
    const double ir = irb, E = Ub[2];
    Ubb[0] += ubb * (-ub * ir) + Hbb * ((-gamma * E * ir + gm1 * ub * ub) * ir) + 0.5 * sbb * sb * ir;
    Ubb[1] += ubb * ir + Hbb * (-gm1 * ub * ir);
    Ubb[2] += Hbb * gamma * ir;
  }
}

// ---------------------------------------------------------------------------------------
// Reverse stage over one tile
// ---------------------------------------------------------------------------------------

// T cells per tile; IPT (interface, field) items per thread in the per-item phase, so the
// tile has about a 1/IPT of the threads (every phase loops over its items)
template <int T, int IPT = 1>
struct AdjTile {
  static constexpr int M = 3;
  static constexpr int W = (T + 9) & ~1;
  static constexpr int NI = T + 1;
  static constexpr int NT = ((M * NI + 32 * IPT - 1) / (32 * IPT)) * 32;
  static constexpr int kBar = 0;
  static constexpr int kUin = 2;
  static constexpr int kF = kUin + M * W;
  static constexpr int kVel = kF + M * W;
  static constexpr int kH = kVel + W;
  static constexpr int kSr = kH + W;
  static constexpr int kIr = kSr + W;        // 1 / rho per cell
  static constexpr int kL = kIr + W;         // [9][NI] stored L
  static constexpr int kRs = kL + 9 * NI;    // [3][NI]
  static constexpr int kFs = kRs + 3 * NI;   // [3][NI] F_s = F+ + F-
  static constexpr int kHf = kFs + 3 * NI;   // [3][NI] h
  static constexpr int kW = kHf + 3 * NI;    // [3][T + 2] w = cL dt ubar_out on cells j0-1 .. j0+T
  static constexpr int kHb = kW + 3 * (T + 2);  // [3][NI] hbar
  static constexpr int kLb = kHb + 3 * NI;   // [3 fields][NI][3] adjoint of the stored L rows
  static constexpr int kG = kLb + 9 * NI;    // [3 fields][NI][12]: per stencil cell, the adjoints
                                             // of its projected flux and state (ab, bb)
  static constexpr int kRed = kG + 3 * NI * 12;  // 4 * 32
  static constexpr int kTotal = kRed + 4 * 32;
  static constexpr size_t bytes = sizeof(double) * kTotal;
};

__device__ __forceinline__ double block_sum_to(double v, double* scratch, int k) {
  // deterministic block sum (fixed shuffle tree, fixed warp order); result valid in thread 0
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) scratch[k * 32 + warp] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) s += scratch[k * 32 + w];
  return s;
}

template <class MATH, int T, int IPT>
__global__ void __launch_bounds__(AdjTile<T, IPT>::NT) adj_stage_kernel(const AdjArgs a) {
  using TL = AdjTile<T, IPT>;
  constexpr int W = TL::W, NI = TL::NI, NT = TL::NT;
  extern __shared__ __align__(16) double sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TL::kBar);
  double* s_uin = sm + TL::kUin;
  double* s_f = sm + TL::kF;
  double* s_vel = sm + TL::kVel;
  double* s_H = sm + TL::kH;
  double* s_sr = sm + TL::kSr;
  double* s_ir = sm + TL::kIr;
  double* s_L = sm + TL::kL;
  double* s_rs = sm + TL::kRs;
  double* s_F = sm + TL::kFs;
  double* s_h = sm + TL::kHf;
  double* s_w = sm + TL::kW;
  double* s_hb = sm + TL::kHb;
  double* s_Lb = sm + TL::kLb;
  double* s_G = sm + TL::kG;
  double* s_red = sm + TL::kRed;
  const int tid = threadIdx.x;
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  uint32_t phase = 0;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int2 item = a.tiles[tile];
    const int p = item.x;
    const BatchSeg sg = a.segs[p];
    const long long n = sg.n;
    const long long j0 = (long long)item.y * T;
    const int Tc = (int)((n - j0 < T) ? (n - j0) : T);
    const int ni = Tc + 1;
    const double* uin = a.uin + sg.poff;
    const double al[3] = {a.alpha[4 * p], a.alpha[4 * p + 1], a.alpha[4 * p + 2]};
    const double dt = a.dt[p];
    const double* ubo = a.ubar_out + sg.uoff;

    // ---- A: stage the input window (cells j0-3 .. j0+Tc+2) and w on cells j0-1 .. j0+Tc
    const long long s0 = j0 & ~1LL;
    const int off = (int)(j0 - s0);
    const int cells = Tc + 2 * G;
    const int len = (off + cells + 1) & ~1;
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)len * 8u;
      mbar_arrive_expect_tx(bar, bytes * 3u);
#pragma unroll
      for (int c = 0; c < 3; ++c) bulk_g2s(s_uin + c * W, uin + c * a.pitch + s0, bytes, bar);
    }
    for (int k = tid; k < 3 * (Tc + 2); k += NT) {
      const int c = k / (Tc + 2), jj = k - c * (Tc + 2);
      const long long j = j0 - 1 + jj;
      s_w[c * (T + 2) + jj] = (j >= 0 && j < n) ? a.cL * dt * ubo[c * a.ustride + j] : 0.0;
    }
    const bool ok = mbar_wait_bounded(bar, phase);
    if (__syncthreads_or(ok ? 0 : 1)) {
      if (tid == 0) a.partial[4 * tile] = __longlong_as_double(0x7ff8000000000000LL);  // NaN marks the timeout
      mbar_wait_bounded(bar, phase);
      return;
    }
    phase ^= 1u;

    // ---- B: per-cell quantities
    for (int k = tid; k < cells; k += NT) {
      double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
      double f[3], u, H, sr, pp;
      MATH::euler_cell(U, a.gamma, f, u, H, sr, pp);
      s_f[k] = f[0];
      s_f[W + k] = f[1];
      s_f[2 * W + k] = f[2];
      s_vel[k] = u;
      s_H[k] = H;
      s_sr[k] = sr;
      const double r = rsqrt(U[0]);
      s_ir[k] = r * r;  // for the reverse Roe average (two per interface), one per cell
    }
    __syncthreads();
    // ---- C0: per interface (local li: cells li+2 | li+3; global interface j0 - 1 + li, record
    //      slot j0 + li), from the forward stage's record: the eigenvectors rebuilt from Roe's
    //      mean state exactly as the forward formed them, F_s = F+_s + F-_s and the branch flags
    const double* recp = a.rec + (size_t)a.goff[p] * kAdjRec;
    unsigned* s_flags = reinterpret_cast<unsigned*>(s_red);  // free until the tile sums of phase E
    static_assert(NI <= 4 * 32 * 2, "one flags word per interface in the reduction buffer");
    for (int i = tid; i < ni; i += NT) {
      const double* r = recp + (size_t)(j0 + i) * kAdjRec;
      double L[9], rs[3];
      MATH::roe_mean(r[0], r[1], a.gamma, L, rs);
#pragma unroll
      for (int e = 0; e < 9; ++e) s_L[e * NI + i] = L[e];
#pragma unroll
      for (int e = 0; e < 3; ++e) s_rs[e * NI + i] = rs[e];
#pragma unroll
      for (int e = 0; e < 3; ++e) s_F[e * NI + i] = r[2 + e];
      s_flags[i] = (unsigned)__double_as_longlong(r[5]);
    }
    __syncthreads();
    // ---- hbar per interface: L_gi and L_gi+1 depend on h of interface gi = j0 - 1 + i
    for (int k = tid; k < 3 * ni; k += NT) {
      const int c = k / ni, i = k - c * ni;
      const long long gi = j0 - 1 + i;
      const double wl = (gi >= 0) ? s_w[c * (T + 2) + i] : 0.0;
      const double wr = (gi + 1 < n) ? s_w[c * (T + 2) + i + 1] : 0.0;
      s_hb[c * NI + i] = (wr - wl) * sg.inv_dx;
    }
    __syncthreads();
    // ---- C1: per (interface, field) of the owned interfaces: the reverse of both
    //      reconstructions with the forward's branches (a restricted stencil's gradient is a
    //      fixed coefficient vector; only the others need the projected stencil values, taken
    //      with the forward's operations), of the Lax-Friedrichs split and of the projection
    double abar0 = 0.0, abar1 = 0.0, abar2 = 0.0;
    for (int item2 = tid; item2 < 3 * ni; item2 += NT) {
      const int s = item2 / ni, i = item2 - s * ni;
      const bool owned = (i >= 1) || (j0 == 0);
      if (!owned) continue;
      const double l[3] = {s_L[(3 * s) * NI + i], s_L[(3 * s + 1) * NI + i], s_L[(3 * s + 2) * NI + i]};
      const unsigned fl = s_flags[i];
      const bool rp = (fl >> (2 * s)) & 1u, tp = (fl >> (2 * s + 1)) & 1u;
      const bool rm = (fl >> (2 * (3 + s))) & 1u, tm = (fl >> (2 * (3 + s) + 1)) & 1u;
      // only a stencil that was not restricted needs its projected values (weno_grad)
      double vp[6] = {0, 0, 0, 0, 0, 0}, qm[6] = {0, 0, 0, 0, 0, 0};
      if (!(rp && rm)) {
        double vm[6];
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) {
          const int k = i + kk;
          const double f[3] = {s_f[k], s_f[W + k], s_f[2 * W + k]};
          const double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
          double pa, pb;
          MATH::project3_ab(l, f, U, pa, pb);  // the same operations as project3
          MATH::project_v(pa, pb, al[s], vp[kk], vm[kk]);
        }
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) qm[kk] = vm[5 - kk];
      }
      double* Gs = s_G + (s * NI + i) * 12;
      double* Lbs = s_Lb + (s * NI + i) * 3;
      const double u = s_rs[i], H = s_rs[NI + i], c = s_rs[2 * NI + i];
      const double hb[3] = {s_hb[i], s_hb[NI + i], s_hb[2 * NI + i]};
      // Fbar_s = sum_c R[c][s] hbar_c, R columns (1, u-c, H-uc), (1, u, u^2/2), (1, u+c, H+uc)
      double Fb;
      if (s == 0) Fb = hb[0] + (u - c) * hb[1] + (H - u * c) * hb[2];
      else if (s == 1) Fb = hb[0] + u * hb[1] + 0.5 * u * u * hb[2];
      else Fb = hb[0] + (u + c) * hb[1] + (H + u * c) * hb[2];
      double vpb[6] = {0, 0, 0, 0, 0, 0}, qmb[6] = {0, 0, 0, 0, 0, 0};
      weno_grad(vp, a.eps, rp, tp, Fb, vpb);
      weno_grad(qm, a.eps, rm, tm, Fb, qmb);
      // With s_k = v+bar_k + v-bar_k and d_k = v+bar_k - v-bar_k (v-bar mirrored), the stored
      // L row's adjoint is kProj (Sf + alpha Su), Sf = sum_k s_k f_k, Su = sum_k d_k u_k, and
      // d/d alpha is kProj l.Su: one pass over the stencil for both
      double Sf[3] = {0, 0, 0}, Su[3] = {0, 0, 0};
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) {
        const int k = i + kk;
        const double f[3] = {s_f[k], s_f[W + k], s_f[2 * W + k]};
        const double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
        const double vmb = qmb[5 - kk];
        const double sk = vpb[kk] + vmb, dk = vpb[kk] - vmb;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          Sf[e] = fma(sk, f[e], Sf[e]);
          Su[e] = fma(dk, U[e], Su[e]);
        }
        // adjoints of the projected flux and state of stencil cell kk; phase D reverse forms
        // their images under the three fields' L rows
        Gs[kk] = MATH::kProj * sk;
        Gs[6 + kk] = MATH::kProj * al[s] * dk;
      }
#pragma unroll
      for (int e = 0; e < 3; ++e) Lbs[e] = MATH::kProj * fma(al[s], Su[e], Sf[e]);
      const double ab_alpha = MATH::kProj * MATH::project3_b(l, Su);
      if (s == 0) abar0 += ab_alpha;
      else if (s == 1) abar1 += ab_alpha;
      else abar2 += ab_alpha;
    }
    __syncthreads();
    // ---- D forward: h per interface, and the d/d dt partial  cL sum_j ubar_out_j . L_j
    for (int i = tid; i < ni; i += NT) {
      const double rs[3] = {s_rs[i], s_rs[NI + i], s_rs[2 * NI + i]};
      const double F[3] = {s_F[i], s_F[NI + i], s_F[2 * NI + i]};
      double h[3];
      MATH::backproject(rs, F, h);
#pragma unroll
      for (int c = 0; c < 3; ++c) s_h[c * NI + i] = h[c];
    }
    __syncthreads();
    double dtb = 0.0;
    for (int t = tid; t < Tc; t += NT) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double L = MATH::flux_diff(s_h[c * NI + t + 1], s_h[c * NI + t], sg.dx, sg.inv_dx);
        dtb += a.cL * ubo[c * a.ustride + j0 + t] * L;
      }
    }
    // ---- D reverse: Roe's average per owned interface, fold the fields, write G
    for (int i = tid; i < ni; i += NT) {
      const bool owned = (i >= 1) || (j0 == 0);
      if (!owned) continue;
      const double rs[3] = {s_rs[i], s_rs[NI + i], s_rs[2 * NI + i]};
      const double hb[3] = {s_hb[i], s_hb[NI + i], s_hb[2 * NI + i]};
      double Lb[9], Rb[9];
#pragma unroll
      for (int s = 0; s < 3; ++s) {
#pragma unroll
        for (int e = 0; e < 3; ++e) Lb[3 * s + e] = MATH::kLScale * s_Lb[(s * NI + i) * 3 + e];
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
#pragma unroll
        for (int s = 0; s < 3; ++s) Rb[3 * cc + s] = hb[cc] * s_F[s * NI + i];
      }
      const int ka = i + 2, kb = i + 3;
      const double Ua[3] = {s_uin[off + ka], s_uin[W + off + ka], s_uin[2 * W + off + ka]};
      const double Ubv[3] = {s_uin[off + kb], s_uin[W + off + kb], s_uin[2 * W + off + kb]};
      double Uab[3] = {0, 0, 0}, Ubb[3] = {0, 0, 0};
      roe_reverse(Ua, Ubv, s_sr[ka], s_vel[ka], s_H[ka], s_ir[ka], s_sr[kb], s_vel[kb], s_H[kb], s_ir[kb], rs, a.gamma,
                  Lb, Rb, Uab, Ubb);
      const long long gi = j0 - 1 + i;
      double* out = a.G + (a.goff[p] + gi + 1) * 36;
      // the stencil cells' flux and state adjoints: sum over the fields s of ab_s l_s, bb_s l_s
      double lr[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) lr[e] = s_L[e * NI + i];
      const double* G0 = s_G + (0 * NI + i) * 12;
      const double* G1 = s_G + (1 * NI + i) * 12;
      const double* G2 = s_G + (2 * NI + i) * 12;
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) {
        const double a0 = G0[kk], a1 = G1[kk], a2 = G2[kk];
        const double c0 = G0[6 + kk], c1 = G1[6 + kk], c2 = G2[6 + kk];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          out[kk * 6 + e] = fma(a2, lr[6 + e], fma(a1, lr[3 + e], a0 * lr[e]));
          double v = fma(c2, lr[6 + e], fma(c1, lr[3 + e], c0 * lr[e]));
          if (kk == 2) v += Uab[e];
          if (kk == 3) v += Ubb[e];
          out[kk * 6 + 3 + e] = v;
        }
      }
    }
    // ---- E: per-tile partial sums (fixed order)
    double r0 = block_sum_to(abar0, s_red, 0);
    double r1 = block_sum_to(abar1, s_red, 1);
    double r2 = block_sum_to(abar2, s_red, 2);
    double r3 = block_sum_to(dtb, s_red, 3);
    if (tid == 0) {
      a.partial[4 * tile + 0] = r0;
      a.partial[4 * tile + 1] = r1;
      a.partial[4 * tile + 2] = r2;
      a.partial[4 * tile + 3] = r3;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Gather per cell.  out = a_self * x + A^T fbar + Ubar (+ out if accumulate); acc += a_acc * x.
// ---------------------------------------------------------------------------------------
#ifdef WT_ADJOINT_COMMON_KERNELS  // defined in exactly one translation unit
__device__ __forceinline__ void gather_add(const double* Gi, int kk, const double* U, double gamma, double* Ub,
                                           bool flip) {
  double fb[3] = {Gi[kk * 6 + 0], Gi[kk * 6 + 1], Gi[kk * 6 + 2]};
  double t[3] = {Gi[kk * 6 + 3], Gi[kk * 6 + 4], Gi[kk * 6 + 5]};
  euler_flux_jt(U, gamma, fb, t);
  Ub[0] += t[0];
  Ub[1] += flip ? -t[1] : t[1];
  Ub[2] += t[2];
}

__global__ void __launch_bounds__(256) adj_gather_kernel(const GatherArgs a) {
  const int p = blockIdx.y;
  const BatchSeg sg = a.segs[p];
  const long long n = sg.n;
  const double* uin = a.uin + sg.poff;
  const double* Gp = a.G + a.goff[p] * 36;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    double Ub[3] = {0, 0, 0};
    const double Uj[3] = {uin[j + G], uin[a.pitch + j + G], uin[2 * a.pitch + j + G]};
    // interfaces whose stencil holds cell j directly: i = j + 2 - kk, i in [-1, n-1]
    double fb[3] = {0, 0, 0}, ub[3] = {0, 0, 0};
    for (int kk = 0; kk < 6; ++kk) {
      const long long i = j + 2 - kk;
      if (i < -1 || i > n - 1) continue;
      const double* Gi = Gp + (i + 1) * 36;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        fb[e] += Gi[kk * 6 + e];
        ub[e] += Gi[kk * 6 + 3 + e];
      }
    }
    euler_flux_jt(Uj, a.gamma, fb, ub);
#pragma unroll
    for (int e = 0; e < 3; ++e) Ub[e] += ub[e];
    // ghost cells whose value is taken from cell j (boundary conditions)
    if (j < G || j >= n - G) {
      const long long lo_end = (n <= 8) ? n - 1 : 1;
      const long long hi_start = (n <= 8) ? n : n - 3;
      for (int pass = 0; pass < 2; ++pass) {
        const long long ib = pass == 0 ? -1 : hi_start, ie = pass == 0 ? lo_end : n - 1;
        for (long long i = ib; i <= ie; ++i) {
          for (int kk = 0; kk < 6; ++kk) {
            const long long g = i - 2 + kk;
            if (g >= 0 && g < n) continue;
            bool flip;
            const long long src = ghost_source(g, n, sg.bc_lo, sg.bc_hi, &flip);
            if (src != j) continue;
            const double Ug[3] = {uin[g + G], uin[a.pitch + g + G], uin[2 * a.pitch + g + G]};
            gather_add(Gp + (i + 1) * 36, kk, Ug, a.gamma, Ub, flip);
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long idx = sg.uoff + c * a.ustride + j;
      const double xv = a.x[idx];
      double v = a.a_self * xv + Ub[c];
      if (a.accumulate) v += a.out[idx];
      a.out[idx] = v;
      if (a.acc) a.acc[idx] += a.a_acc * xv;
    }
  }
}

#endif  // WT_ADJOINT_COMMON_KERNELS

// first index attaining each alpha_s and max(|u| + c) of the stage input; arg[p][0..3] preset to n
template <class MATH>
__global__ void __launch_bounds__(256) adj_argmax_kernel(const double* uin, long long pitch, const BatchSeg* segs,
                                                         const double* alpha, double gamma, int* arg) {
  const int p = blockIdx.y;
  const BatchSeg sg = segs[p];
  const double* u = uin + sg.poff;
  const double a0 = alpha[4 * p], a1 = alpha[4 * p + 1], a2 = alpha[4 * p + 2];
  const double smax = (a0 < a2) ? a2 : a0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < sg.n;
       j += (long long)gridDim.x * blockDim.x) {
    const double U[3] = {u[j + G], u[pitch + j + G], u[2 * pitch + j + G]};
    double lam[3];
    MATH::euler_speeds(U, gamma, lam);
    if (lam[0] == a0) atomicMin(&arg[4 * p + 0], (int)j);
    if (lam[1] == a1) atomicMin(&arg[4 * p + 1], (int)j);
    if (lam[2] == a2) atomicMin(&arg[4 * p + 2], (int)j);
    const double s = (lam[0] < lam[2]) ? lam[2] : lam[0];
    if (s == smax) atomicMin(&arg[4 * p + 3], (int)j);
  }
}

#ifdef WT_ADJOINT_COMMON_KERNELS
// Per problem: sum the tile partials in order; carry d/d alpha_s to the argmax cells of the
// stage input; accumulate d/d dt; after stage 1 (final != 0) carry d/d dt to the argmax of
// max(|u| + c) of u^n through dt = cfl dx / smax.
__global__ void adj_apply_kernel(const double* uin, long long pitch, const BatchSeg* segs, const int* tstart,
                                 const int* tcount, const double* partial, const double* alpha, const double* dt,
                                 const int* arg, double* ubar, long long ustride, double* dtbar, int final_stage,
                                 double gamma, int nprob) {
  // one warp per problem: the lanes sum strided tiles' partials, then a fixed-order shuffle
  // reduction (deterministic); lane 0 applies the derivatives of the maxima
  const int p = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= nprob) return;  // the same for the whole warp
  const BatchSeg sg = segs[p];
  const double* u = uin + sg.poff;
  double ab[4] = {0, 0, 0, 0};
  for (int t = tstart[p] + lane; t < tstart[p] + tcount[p]; t += 32)
    for (int e = 0; e < 4; ++e) ab[e] += partial[4 * t + e];
  for (int o = 16; o > 0; o >>= 1)
    for (int e = 0; e < 4; ++e) ab[e] += __shfl_xor_sync(0xffffffffu, ab[e], o);
  if (lane != 0) return;
  for (int s = 0; s < 3; ++s) {
    const int j = arg[4 * p + s];
    if (j < 0 || j >= sg.n) continue;
    const double U[3] = {u[j + G], u[pitch + j + G], u[2 * pitch + j + G]};
    double du[3], dc[3];
    euler_uc_grad(U, gamma, du, dc);
    const double uu = U[1] / U[0];
    const double pp = (gamma - 1.0) * (U[2] - 0.5 * U[1] * uu);
    const double cc = sqrt(gamma * pp / U[0]);
    const double lam = s == 0 ? uu - cc : (s == 1 ? uu : uu + cc);
    const double sgn = lam < 0 ? -1.0 : 1.0;
    for (int e = 0; e < 3; ++e) {
      const double dl = s == 0 ? du[e] - dc[e] : (s == 1 ? du[e] : du[e] + dc[e]);
      ubar[sg.uoff + e * ustride + j] += ab[s] * sgn * dl;
    }
  }
  double db = dtbar[p] + ab[3];
  if (final_stage) {
    const int j = arg[4 * p + 3];
    if (j >= 0 && j < sg.n) {
      const double U[3] = {u[j + G], u[pitch + j + G], u[2 * pitch + j + G]};
      double du[3], dc[3];
      euler_uc_grad(U, gamma, du, dc);
      const double uu = U[1] / U[0];
      const double sgn = uu < 0 ? -1.0 : 1.0;
      const double a0 = alpha[4 * p], a2 = alpha[4 * p + 2];
      const double smax = (a0 < a2) ? a2 : a0;
      const double k = -db * dt[p] / smax;  // d dt / d smax = -dt / smax
      for (int e = 0; e < 3; ++e) ubar[sg.uoff + e * ustride + j] += k * (sgn * du[e] + dc[e]);
    }
    db = 0.0;
  }
  dtbar[p] = db;
}

// records of the forward recompute: alphas of a slot (and dt) per problem
__global__ void adj_record_kernel(const Ctl* ctl, int slot, double* alpha_out, double* dt_out, int nprob) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  for (int s = 0; s < 3; ++s) alpha_out[4 * p + s] = bits_to_double(ctl[p].amax[slot][s]);
  alpha_out[4 * p + 3] = 0.0;
  if (dt_out) dt_out[p] = ctl[p].dt;
}

#endif  // WT_ADJOINT_COMMON_KERNELS

// grid <= 0: as many CTAs as can be resident (persistent loop over the tile table)
template <class MATH, int T, int IPT>
cudaError_t launch_adj_stage_t(const AdjArgs& a, int grid, cudaStream_t st) {
  using TL = AdjTile<T, IPT>;
  static_assert(TL::bytes <= 48 * 1024, "tile exceeds the default dynamic shared memory limit");
  if (grid <= 0) {
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, adj_stage_kernel<MATH, T, IPT>, TL::NT, TL::bytes);
    long long g = (long long)(nb > 0 ? nb : 1) * (sms > 0 ? sms : 1);
    grid = (int)(g < a.ntiles ? g : a.ntiles);
  }
  adj_stage_kernel<MATH, T, IPT><<<grid, TL::NT, TL::bytes, st>>>(a);
  return cudaGetLastError();
}

// code: cells per reverse tile + 1000 x (items per thread - 1) (adj_tile_code)
template <class MATH>
cudaError_t launch_adj_stage_policy(const AdjArgs& a, int grid, int code, cudaStream_t st) {
  switch (code) {
    case 31: return launch_adj_stage_t<MATH, 31, 1>(a, grid, st);
    case 2031: return launch_adj_stage_t<MATH, 31, 3>(a, grid, st);
    case 63: return launch_adj_stage_t<MATH, 63, 1>(a, grid, st);
    case 1063: return launch_adj_stage_t<MATH, 63, 2>(a, grid, st);
    case 2063: return launch_adj_stage_t<MATH, 63, 3>(a, grid, st);
  }
  return cudaErrorInvalidValue;
}

template <class MATH>
cudaError_t prepare_adj_policy() {
  return cudaSuccess;  // every reverse tile fits the default 48 KB of dynamic shared memory
}

template <class MATH>
cudaError_t launch_adj_argmax_policy(const double* uin, long long pitch, const BatchSeg* segs, int nprob,
                                     long long maxn, const double* alpha, double gamma, int* arg, cudaStream_t st) {
  long long bx = (maxn + 255) / 256;
  if (bx > 64) bx = 64;
  adj_argmax_kernel<MATH><<<dim3((unsigned)(bx < 1 ? 1 : bx), (unsigned)nprob), 256, 0, st>>>(uin, pitch, segs, alpha,
                                                                                            gamma, arg);
  return cudaGetLastError();
}

}  // namespace wt
