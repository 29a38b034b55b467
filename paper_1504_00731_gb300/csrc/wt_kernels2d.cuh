// Kernel templates of the 2D Euler hot path (dimension by dimension, Sec. 4.3), instantiated
// once per arithmetic policy:
//   pack2d / unpack2d   caller's [4][ny][nx] state <-> padded planes with ghost rows/columns
//   alpha2d             alpha_s per direction and the 2D CFL quantity (warp-shuffle maxima)
//   stage2d             fused RHS + RK stage: a TX x TY tile plus its 3-cell halo staged row by
//                       row with bulk copies, the x sweep then the y sweep in shared memory,
//                       one output write per cell; 104 KB of shared memory, so that two
//                       CTAs (16 warps) share an SM
#pragma once

#include "wt_device.cuh"
#include "wt_launch.h"

namespace wt {

template <int TX, int TY>
struct Tile2D {
  static_assert(TX % 2 == 0, "tile width must be even so that staged rows start 16-byte aligned");
  static constexpr int WX = TX + 2 * G;          // staged row length (even)
  static constexpr int RY = TY + 2 * G;          // staged rows
  static constexpr int NCELL = WX * RY;
  static constexpr int NIX = (TX + 1) * TY;      // x-interfaces of the tile
  static constexpr int NIY = TX * (TY + 1);      // y-interfaces
  static constexpr int NI = NIX > NIY ? NIX : NIY;
  static constexpr int NT = 256;
  static_assert(TX * TY <= NT, "one cell per thread in the flux difference and the stage update");
  // Buffers are reused across the sweeps: the physical flux buffer holds f for the x sweep,
  // then g for the y sweep; the reconstruction buffer holds F, then h of the same sweep; the
  // x sweep's flux difference stays in registers until the update; the eigenvector buffer
  // takes the block reductions at the end.
  static constexpr int kBar = 0;
  static constexpr int kUin = 2;                       // [4][RY][WX]
  static constexpr int kU = kUin + 4 * NCELL;          // velocity u per staged cell
  static constexpr int kV = kU + NCELL;
  static constexpr int kH = kV + NCELL;
  static constexpr int kSr = kH + NCELL;
  static constexpr int kFg = kSr + NCELL;              // [4][NCELL] f, then g
  static constexpr int kL = kFg + 4 * NCELL;           // [16][NI]; 8 * 32 + 32 for the reductions
  static constexpr int kRs = kL + 16 * NI;             // [4][NI]
  static constexpr int kF = kRs + 4 * NI;              // [4][NI] F, then h
  static constexpr int kTotal = kF + 4 * NI;
  static_assert(16 * NI >= 9 * 32, "reduction scratch inside the eigenvector buffer");
  static constexpr size_t bytes = sizeof(double) * kTotal;
  // two CTAs per SM: 228 KB of shared memory per SM, 1 KB of it reserved per CTA
  static_assert(2 * (bytes + 1024) <= 228 * 1024, "two tiles must fit on one SM");
};

__global__ void pack2d_kernel(const double* __restrict__ src, double* __restrict__ dst, long long nx, long long ny,
                              long long rowp, long long planep, int bxl, int bxh, int byl, int byh);
__global__ void unpack2d_kernel(const double* __restrict__ src, double* __restrict__ dst, long long nx, long long ny,
                                long long rowp, long long planep);

template <class MATH>
__global__ void __launch_bounds__(256) alpha2d_kernel(const double* __restrict__ u, long long nx, long long ny,
                                                      long long rowp, long long planep, double gamma, double dx,
                                                      double dy, Ctl* ctl, int slot) {
  __shared__ double red[9 * 32];
  unsigned long long v[8], q = 0ull;
#pragma unroll
  for (int s = 0; s < 8; ++s) v[s] = 0ull;
  const long long cells = nx * ny;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < cells;
       k += (long long)gridDim.x * blockDim.x) {
    const long long y = k / nx, x = k - y * nx;
    const long long idx = (y + G) * rowp + x + G;
    double U[4] = {u[idx], u[planep + idx], u[2 * planep + idx], u[3 * planep + idx]};
    double lx[4], ly[4], qq;
    MATH::euler2d_speeds(U, gamma, dx, dy, lx, ly, qq);
    if (!(isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]))) flag_error(ctl, WT_ERR_NONPHYSICAL);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      key_max(v[s], lx[s]);
      key_max(v[4 + s], ly[s]);
    }
    key_max(q, qq);
  }
  block_max_atomic<8>(v, red, ctl->amax[slot]);
  unsigned long long qa[1] = {q};
  block_max_atomic<1>(qa, red + 8 * 32, &ctl->cfl2d[slot]);
}

template <class MATH, int STAGE, int TX, int TY>
__global__ void __launch_bounds__(Tile2D<TX, TY>::NT, 2) stage2d_kernel(const Stage2DArgs a) {
  using TL = Tile2D<TX, TY>;
  constexpr int WX = TL::WX, RY = TL::RY, NCELL = TL::NCELL, NI = TL::NI, NT = TL::NT;
  extern __shared__ __align__(16) double sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TL::kBar);
  double* s_uin = sm + TL::kUin;
  double* s_u = sm + TL::kU;
  double* s_v = sm + TL::kV;
  double* s_H = sm + TL::kH;
  double* s_sr = sm + TL::kSr;
  double* s_fg = sm + TL::kFg;
  double* s_L = sm + TL::kL;
  double* s_rs = sm + TL::kRs;
  double* s_F = sm + TL::kF;
  double* s_h = s_F;
  double* s_red = s_L;

  pdl_launch_dependents();
  pdl_wait();
  const int tid = threadIdx.x;
  Ctl* ctl = a.ctl;
  const long long nx = a.nx, ny = a.ny;
  const long long x0 = (long long)blockIdx.x * TX, y0 = (long long)blockIdx.y * TY;
  if (x0 >= nx || y0 >= ny) return;
  const int tcx = (int)((nx - x0 < TX) ? (nx - x0) : TX);
  const int tcy = (int)((ny - y0 < TY) ? (ny - y0) : TY);
  const bool first_tile = (blockIdx.x == 0 && blockIdx.y == 0);

  double dt = 0.0;
  if (STAGE != STAGE_RHS) {
    if (STAGE == STAGE_RK1) {
      const bool act = (ctl->status == 0) && (ctl->t < ctl->t_final);
      if (!act) {
        if (first_tile && tid == 0) ctl->active = 0;
        return;
      }
    } else if (ctl->active == 0) {
      return;
    }
    if (first_tile && tid < 8) ctl->amax[(STAGE + 2) % 3][tid] = 0ull;
    if (first_tile && tid == 8) ctl->cfl2d[(STAGE + 2) % 3] = 0ull;
  }
  const int slot_in = (STAGE == STAGE_RHS) ? 0 : STAGE;
  double ax[4], ay[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    ax[s] = bits_to_double(ctl->amax[slot_in][s]);
    ay[s] = bits_to_double(ctl->amax[slot_in][4 + s]);
  }
  if (STAGE == STAGE_RK1) {
    dt = ctl->dt_fixed > 0.0 ? ctl->dt_fixed : MATH::cfl_dt_2d(ctl->cfl, bits_to_double(ctl->cfl2d[0]));
    const double rem = ctl->t_final - ctl->t;
    if (rem < dt) dt = rem;
    if (first_tile && tid == 0) {
      ctl->dt = dt;
      ctl->active = 1;
    }
  } else if (STAGE != STAGE_RHS) {
    dt = ctl->dt;
  }

  // ---- A: stage rows y0-3 .. y0+tcy+2, columns x0-3 .. x0+tcx+2 of every plane (u^n of
  //      stages 2 and 3 is read in phase E, one load per cell)
  const int rows = tcy + 2 * G;
  const int len = (tcx + 2 * G + 1) & ~1;
  constexpr bool kNeedUn = (STAGE == STAGE_RK2 || STAGE == STAGE_RK3);
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid < 32) {
    const uint32_t bytes = (uint32_t)len * 8u;
    const int ncopy = 4 * rows;
    if (tid == 0) mbar_arrive_expect_tx(bar, bytes * (uint32_t)ncopy);
    __syncwarp();
    for (int k = tid; k < ncopy; k += 32) {
      const int c = k / rows, r = k - c * rows;
      bulk_g2s(s_uin + (c * RY + r) * WX, a.uin + c * a.planep + (y0 + r) * a.rowp + x0, bytes, bar);
    }
  }
  const bool ok = mbar_wait_bounded(bar, 0);
  if (__syncthreads_or(ok ? 0 : 1)) {
    if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
    mbar_wait_bounded(bar, 0);
    return;
  }

  // ---- B: per staged cell of the cross (interior rows with x-halo, interior columns with
  //      y-halo): velocities, H, sqrt(rho) and f; g follows once the x sweep is done with f
  for (int k = tid; k < NCELL; k += NT) {
    const int r = k / WX, col = k - r * WX;
    if (r >= rows || col >= tcx + 2 * G) continue;
    const bool xin = (col >= G && col < G + tcx), yin = (r >= G && r < G + tcy);
    if (!xin && !yin) continue;  // corner: not on any stencil
    double U[4] = {s_uin[k], s_uin[NCELL + k], s_uin[2 * NCELL + k], s_uin[3 * NCELL + k]};
    if (!(isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]))) flag_error(ctl, WT_ERR_NONPHYSICAL);
    double f[4], g[4], u, v, H, sr;
    MATH::euler2d_cell(U, a.gamma, f, g, u, v, H, sr);
    s_u[k] = u;
    s_v[k] = v;
    s_H[k] = H;
    s_sr[k] = sr;
    if (yin) {
#pragma unroll
      for (int c = 0; c < 4; ++c) s_fg[c * NCELL + k] = f[c];
    }
  }
  __syncthreads();

  // ---- x sweep.  Interface i of row r sits between cells (r+3, i+2) and (r+3, i+3).
  const int nix = (tcx + 1) * tcy;
  for (int it = tid; it < nix; it += NT) {
    const int r = it / (tcx + 1), i = it - r * (tcx + 1);
    const int ka = (r + G) * WX + i + 2, kb = ka + 1;
    double L[16], rs[4];
    MATH::roe2d(0, s_sr[ka], s_u[ka], s_v[ka], s_H[ka], s_sr[kb], s_u[kb], s_v[kb], s_H[kb], a.gamma, L, rs);
#pragma unroll
    for (int e = 0; e < 16; ++e) s_L[e * NI + it] = L[e];
#pragma unroll
    for (int e = 0; e < 4; ++e) s_rs[e * NI + it] = rs[e];
  }
  __syncthreads();
  for (int item = tid; item < 4 * nix; item += NT) {
    const int s = item / nix, it = item - s * nix;
    const int r = it / (tcx + 1), i = it - r * (tcx + 1);
    const double l[4] = {s_L[(4 * s) * NI + it], s_L[(4 * s + 1) * NI + it], s_L[(4 * s + 2) * NI + it],
                         s_L[(4 * s + 3) * NI + it]};
    const double al = s == 0 ? ax[0] : (s == 1 ? ax[1] : (s == 2 ? ax[2] : ax[3]));
    double vp[6], vm[6];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) {
      const int k = (r + G) * WX + i + kk;
      const double f[4] = {s_fg[k], s_fg[NCELL + k], s_fg[2 * NCELL + k], s_fg[3 * NCELL + k]};
      const double U[4] = {s_uin[k], s_uin[NCELL + k], s_uin[2 * NCELL + k], s_uin[3 * NCELL + k]};
      MATH::project4(0, l, f, U, al, vp[kk], vm[kk]);
    }
    double qm[6];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) qm[kk] = vm[5 - kk];
    s_F[s * NI + it] = MATH::weno(vp, a.eps, a.alpha_R) + MATH::weno(qm, a.eps, a.alpha_R);
  }
  __syncthreads();
  // back-projection in place (F -> h of the same interface), and g of the y-sweep cells into
  // the flux buffer, which the x sweep no longer reads
  for (int it = tid; it < nix; it += NT) {
    const double rs[4] = {s_rs[it], s_rs[NI + it], s_rs[2 * NI + it], s_rs[3 * NI + it]};
    const double F[4] = {s_F[it], s_F[NI + it], s_F[2 * NI + it], s_F[3 * NI + it]};
    double h[4];
    MATH::backproject2d(0, rs, F, h);
#pragma unroll
    for (int c = 0; c < 4; ++c) s_h[c * NI + it] = h[c];
  }
  for (int q = tid; q < rows * tcx; q += NT) {
    const int r = q / tcx, k = r * WX + G + (q - r * tcx);
    const double U[4] = {s_uin[k], s_uin[NCELL + k], s_uin[2 * NCELL + k], s_uin[3 * NCELL + k]};
    double g[4];
    MATH::euler2d_gflux(U, s_u[k], s_v[k], a.gamma, g);
#pragma unroll
    for (int c = 0; c < 4; ++c) s_fg[c * NCELL + k] = g[c];
  }
  __syncthreads();
  // the x sweep's flux difference of this thread's cell (the cell of phase E), and the y
  // sweep's Roe averages
  double Lx[4] = {0.0, 0.0, 0.0, 0.0};
  if (tid < tcx * tcy) {
    const int r = tid / tcx, t = tid - r * tcx;
    const int it = r * (tcx + 1) + t;
#pragma unroll
    for (int c = 0; c < 4; ++c) Lx[c] = MATH::flux_diff(s_h[c * NI + it + 1], s_h[c * NI + it], a.dx, a.inv_dx);
  }

  // ---- y sweep.  Interface j of column t sits between cells (j+2, t+3) and (j+3, t+3).
  const int niy = tcx * (tcy + 1);
  for (int it = tid; it < niy; it += NT) {
    const int j = it / tcx, t = it - j * tcx;
    const int ka = (j + 2) * WX + t + G, kb = ka + WX;
    double L[16], rs[4];
    MATH::roe2d(1, s_sr[ka], s_u[ka], s_v[ka], s_H[ka], s_sr[kb], s_u[kb], s_v[kb], s_H[kb], a.gamma, L, rs);
#pragma unroll
    for (int e = 0; e < 16; ++e) s_L[e * NI + it] = L[e];
#pragma unroll
    for (int e = 0; e < 4; ++e) s_rs[e * NI + it] = rs[e];
  }
  __syncthreads();
  for (int item = tid; item < 4 * niy; item += NT) {
    const int s = item / niy, it = item - s * niy;
    const int j = it / tcx, t = it - j * tcx;
    const double l[4] = {s_L[(4 * s) * NI + it], s_L[(4 * s + 1) * NI + it], s_L[(4 * s + 2) * NI + it],
                         s_L[(4 * s + 3) * NI + it]};
    const double al = s == 0 ? ay[0] : (s == 1 ? ay[1] : (s == 2 ? ay[2] : ay[3]));
    double vp[6], vm[6];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) {
      const int k = (j + kk) * WX + t + G;
      const double f[4] = {s_fg[k], s_fg[NCELL + k], s_fg[2 * NCELL + k], s_fg[3 * NCELL + k]};
      const double U[4] = {s_uin[k], s_uin[NCELL + k], s_uin[2 * NCELL + k], s_uin[3 * NCELL + k]};
      MATH::project4(1, l, f, U, al, vp[kk], vm[kk]);
    }
    double qm[6];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) qm[kk] = vm[5 - kk];
    s_F[s * NI + it] = MATH::weno(vp, a.eps, a.alpha_R) + MATH::weno(qm, a.eps, a.alpha_R);
  }
  __syncthreads();
  for (int it = tid; it < niy; it += NT) {
    const double rs[4] = {s_rs[it], s_rs[NI + it], s_rs[2 * NI + it], s_rs[3 * NI + it]};
    const double F[4] = {s_F[it], s_F[NI + it], s_F[2 * NI + it], s_F[3 * NI + it]};
    double h[4];
    MATH::backproject2d(1, rs, F, h);
#pragma unroll
    for (int c = 0; c < 4; ++c) s_h[c * NI + it] = h[c];
  }
  __syncthreads();

  // ---- E: L = Lx + Ly, RK combine, ghost images, wave speeds of the new state
  unsigned long long vmax[8], qmax = 0ull;
#pragma unroll
  for (int s = 0; s < 8; ++s) vmax[s] = 0ull;
  if (tid < tcx * tcy) {
    const int r = tid / tcx, t = tid - r * tcx;
    const long long x = x0 + t, y = y0 + r;
    const int kc = (r + G) * WX + t + G;
    double un4[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) un4[c] = kNeedUn ? a.un[c * a.planep + (y + G) * a.rowp + x + G] : 0.0;
    double uo[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double Ly = MATH::flux_diff(s_h[c * NI + (r + 1) * tcx + t], s_h[c * NI + r * tcx + t], a.dy, a.inv_dy);
      double L = MATH::add_sweeps(Lx[c], Ly);
      // gravity along -y (TEST 6, Sec. 4.3): -g rho on the y momentum, -g rho v on the energy
      if (c >= 2 && a.gravity != 0.0) L = MATH::add_source(L, a.gravity, s_uin[(c == 2 ? 0 : 2) * NCELL + kc]);
      if (STAGE == STAGE_RHS) {
        a.Lout[(c * ny + y) * nx + x] = L;
      } else {
        const double us = s_uin[c * NCELL + kc];
        const double un = kNeedUn ? un4[c] : us;
        uo[c] = MATH::template rk<(STAGE == STAGE_RHS ? 0 : STAGE)>(un, us, dt, L);
      }
    }
    if (STAGE != STAGE_RHS) {
      const long long row = (y + G) * a.rowp;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        double* o = a.uout + c * a.planep;
        const double val = uo[c];
        o[row + x + G] = val;
        // x ghosts of this row (reflective: x-momentum negated)
        const double vx = (c == 1) ? -val : val;
        if (x < G || x >= nx - G) {
          if (a.bcx_hi == WT_BC_PERIODIC && x < G) o[row + nx + x + G] = val;
          if (a.bcx_lo == WT_BC_PERIODIC && x >= nx - G) o[row + x - nx + G] = val;
          if (a.bcx_lo == WT_BC_OUTFLOW && x == 0) o[row] = o[row + 1] = o[row + 2] = val;
          if (a.bcx_hi == WT_BC_OUTFLOW && x == nx - 1) o[row + nx + 3] = o[row + nx + 4] = o[row + nx + 5] = val;
          if (a.bcx_lo == WT_BC_REFLECTIVE && x < G) o[row + 2 - x] = vx;
          if (a.bcx_hi == WT_BC_REFLECTIVE && x >= nx - G) o[row + 2 * nx + 2 - x] = vx;
        }
        // y ghosts of this column (reflective: y-momentum negated)
        const double vy = (c == 2) ? -val : val;
        const long long col = x + G;
        if (y < G || y >= ny - G) {
          if (a.bcy_hi == WT_BC_PERIODIC && y < G) o[(ny + y + G) * a.rowp + col] = val;
          if (a.bcy_lo == WT_BC_PERIODIC && y >= ny - G) o[(y - ny + G) * a.rowp + col] = val;
          if (a.bcy_lo == WT_BC_OUTFLOW && y == 0) o[col] = o[a.rowp + col] = o[2 * a.rowp + col] = val;
          if (a.bcy_hi == WT_BC_OUTFLOW && y == ny - 1)
            o[(ny + 3) * a.rowp + col] = o[(ny + 4) * a.rowp + col] = o[(ny + 5) * a.rowp + col] = val;
          if (a.bcy_lo == WT_BC_REFLECTIVE && y < G) o[(2 - y) * a.rowp + col] = vy;
          if (a.bcy_hi == WT_BC_REFLECTIVE && y >= ny - G) o[(2 * ny + 2 - y) * a.rowp + col] = vy;
        }
      }
      if (!(isfinite(uo[0]) && isfinite(uo[1]) && isfinite(uo[2]) && isfinite(uo[3])))
        flag_error(ctl, WT_ERR_NONPHYSICAL);
      double lx[4], ly[4], q;
      MATH::euler2d_speeds(uo, a.gamma, a.dx, a.dy, lx, ly, q);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        key_max(vmax[s], lx[s]);
        key_max(vmax[4 + s], ly[s]);
      }
      key_max(qmax, q);
    }
  }
  if (STAGE != STAGE_RHS) {
    const int nxt = (STAGE + 1) % 3;
    block_max_atomic<8>(vmax, s_red, ctl->amax[nxt]);
    unsigned long long qa[1] = {qmax};
    block_max_atomic<1>(qa, s_red + 8 * 32, &ctl->cfl2d[nxt]);
    if (STAGE == STAGE_RK3 && first_tile && tid == 0) {
      ctl->t = ctl->t + dt;
      ctl->steps = ctl->steps + 1;
    }
  }
}

template <class MATH, int STAGE>
cudaError_t launch_stage2d_t(const Stage2DArgs& a, cudaStream_t st) {
  constexpr int TX = 32, TY = 8;
  using TL = Tile2D<TX, TY>;
  auto kern = stage2d_kernel<MATH, STAGE, TX, TY>;  // prepare_stage2d_policy() raised its shared-memory limit
  dim3 grid((unsigned)((a.nx + TX - 1) / TX), (unsigned)((a.ny + TY - 1) / TY));
  return launch_pdl(kern, grid, dim3(TL::NT), TL::bytes, st, a);
}

template <class MATH>
cudaError_t prepare_stage2d_policy() {
  constexpr int TX = 32, TY = 8;
  using TL = Tile2D<TX, TY>;
  cudaError_t e = cudaSuccess;
  // the tile's shared memory, and the largest carveout, so that two CTAs fit on an SM
  const void* kerns[4] = {(const void*)stage2d_kernel<MATH, STAGE_RK1, TX, TY>,
                          (const void*)stage2d_kernel<MATH, STAGE_RK2, TX, TY>,
                          (const void*)stage2d_kernel<MATH, STAGE_RK3, TX, TY>,
                          (const void*)stage2d_kernel<MATH, STAGE_RHS, TX, TY>};
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
    e = cudaFuncSetAttribute(kerns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kerns[i], cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  }
  return e;
}

template <class MATH>
cudaError_t launch_stage2d_policy(int stage, const Stage2DArgs& a, cudaStream_t st) {
  switch (stage) {
    case STAGE_RK1: return launch_stage2d_t<MATH, STAGE_RK1>(a, st);
    case STAGE_RK2: return launch_stage2d_t<MATH, STAGE_RK2>(a, st);
    case STAGE_RK3: return launch_stage2d_t<MATH, STAGE_RK3>(a, st);
    case STAGE_RHS: return launch_stage2d_t<MATH, STAGE_RHS>(a, st);
  }
  return cudaErrorInvalidValue;
}

template <class MATH>
cudaError_t launch_alpha2d_policy(const double* u, long long nx, long long ny, long long rowp, long long planep,
                                  double gamma, double dx, double dy, Ctl* ctl, int slot, cudaStream_t st) {
  long long blocks = (nx * ny + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  alpha2d_kernel<MATH><<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(u, nx, ny, rowp, planep, gamma, dx, dy,
                                                                          ctl, slot);
  return cudaGetLastError();
}

}  // namespace wt
