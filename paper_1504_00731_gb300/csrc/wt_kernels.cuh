// Kernel templates of the 1D hot path, instantiated once per arithmetic policy
// (wt_kernels_strict.cu, wt_kernels_fast.cu):
//   pack1d      caller's unpadded state -> padded planes + ghost cells (boundary fill)
//   alpha1d     max-wavespeed reduction: alpha_s = max_j |lambda_s(u_j)| (warp shuffles)
//   stage1d     fused RHS + RK stage over a tile staged in shared memory by bulk copies
#pragma once

#include "wt_device.cuh"
#include "wt_launch.h"

namespace wt {

template <int FLUX>
struct FluxM {
  static constexpr int m = (FLUX == WT_FLUX_EULER1D) ? 3 : 1;
};

// Tile geometry: T cells, T + 1 interfaces, m threads per interface (one per field)
template <int T, int M>
struct Tile1D {
  static constexpr int W = (T + 9) & ~1;              // staged window: T + 6 cells + alignment slack, even
  static constexpr int NI = T + 1;
  static constexpr int NT = ((M * NI + 31) / 32) * 32;
  // shared-memory layout in doubles
  static constexpr int kBar = 0;
  static constexpr int kUin = 2;
  static constexpr int kUn = kUin + M * W;
  static constexpr int kF = kUn + M * W;
  static constexpr int kVel = kF + M * W;
  static constexpr int kH = kVel + W;
  static constexpr int kSr = kH + W;
  static constexpr int kL = kSr + W;
  static constexpr int kRs = kL + 9 * NI;
  static constexpr int kFs = kRs + 3 * NI;
  static constexpr int kHf = kFs + M * NI;
  static constexpr int kRed = kHf + M * NI;
  static constexpr int kTotal = kRed + 4 * 32;
  static constexpr size_t bytes = sizeof(double) * kTotal;
};

// ---------------------------------------------------------------------------------------
// Boundary fill: copies the caller's state into the padded layout and writes the ghost
// cells (periodic, outflow, reflective with the normal momentum negated).
// ---------------------------------------------------------------------------------------
__global__ void pack1d_kernel(const double* __restrict__ src, long long src_stride, double* __restrict__ dst,
                              long long n, long long pitch, int m, int bc_lo, int bc_hi, int flip_comp);
__global__ void unpack1d_kernel(const double* __restrict__ src, long long pitch, double* __restrict__ dst,
                                long long dst_stride, long long n, int m);

// ---------------------------------------------------------------------------------------
// alpha_s of a padded state into ctl->amax[slot]
// ---------------------------------------------------------------------------------------
template <class MATH, int FLUX>
__global__ void __launch_bounds__(256) alpha1d_kernel(const double* __restrict__ u, long long n, long long pitch,
                                                      double gamma, double adv, Ctl* ctl, int slot) {
  constexpr int M = FluxM<FLUX>::m;
  __shared__ double red[4 * 32];
  double v[M];
#pragma unroll
  for (int s = 0; s < M; ++s) v[s] = 0.0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    if (FLUX == WT_FLUX_EULER1D) {
      double U[3] = {u[j + G], u[pitch + j + G], u[2 * pitch + j + G]};
      double lam[3];
      MATH::euler_speeds(U, gamma, lam);
      if (!finite3(U)) flag_error(ctl, WT_ERR_NONPHYSICAL);
#pragma unroll
      for (int s = 0; s < M; ++s) v[s] = (v[s] < lam[s]) ? lam[s] : v[s];
    } else {
      double x = u[j + G];
      double lam = (FLUX == WT_FLUX_ADVECTION) ? fabs(adv) : fabs(x);
      if (!isfinite(x)) flag_error(ctl, WT_ERR_NONPHYSICAL);
      v[0] = (v[0] < lam) ? lam : v[0];
    }
  }
  block_max_atomic<M>(v, red, ctl->amax[slot]);
}

// alpha_s of every problem of a batch: blockIdx.y is the problem
template <class MATH, int FLUX>
__global__ void __launch_bounds__(256) alpha1d_batched_kernel(const double* __restrict__ u, long long pitch,
                                                              const BatchSeg* __restrict__ segs, double gamma,
                                                              double adv, Ctl* ctl) {
  constexpr int M = FluxM<FLUX>::m;
  __shared__ double red[4 * 32];
  const BatchSeg sg = segs[blockIdx.y];
  Ctl* c = ctl + blockIdx.y;
  const double* up = u + sg.poff;
  double v[M];
#pragma unroll
  for (int s = 0; s < M; ++s) v[s] = 0.0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < sg.n;
       j += (long long)gridDim.x * blockDim.x) {
    if (FLUX == WT_FLUX_EULER1D) {
      double U[3] = {up[j + G], up[pitch + j + G], up[2 * pitch + j + G]};
      double lam[3];
      MATH::euler_speeds(U, gamma, lam);
      if (!finite3(U)) flag_error(c, WT_ERR_NONPHYSICAL);
#pragma unroll
      for (int s = 0; s < M; ++s) v[s] = (v[s] < lam[s]) ? lam[s] : v[s];
    } else {
      double x = up[j + G];
      double lam = (FLUX == WT_FLUX_ADVECTION) ? fabs(adv) : fabs(x);
      if (!isfinite(x)) flag_error(c, WT_ERR_NONPHYSICAL);
      v[0] = (v[0] < lam) ? lam : v[0];
    }
  }
  block_max_atomic<M>(v, red, c->amax[0]);
}

// ---------------------------------------------------------------------------------------
// Fused RHS + RK stage (1D).  One CTA per tile of T cells.
//   A  bulk-copy the stage input (and u^n for stages 2, 3) over cells j0-3 .. j0+T+2
//   B  per cell: physical flux (and velocity, enthalpy, sqrt(rho) for Euler)
//   C0 per interface: Roe average and left eigenvectors (Euler)
//   C1 per (interface, field): projection, Lax-Friedrichs split, WENO-theta on both sides
//   D  per interface: back-projection to the interface flux h_{j+1/2}
//   E  per cell: flux difference, RK combine, ghost images, wave speeds of the new state
// ---------------------------------------------------------------------------------------
template <class MATH, int FLUX, int STAGE, int T>
__device__ __forceinline__ bool stage1d_tile(const Stage1DArgs& a, const long long j0, const bool first_tile, double* sm,
                                             uint32_t& phase) {
  constexpr int M = FluxM<FLUX>::m;
  using TL = Tile1D<T, M>;
  constexpr int W = TL::W, NI = TL::NI, NT = TL::NT;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TL::kBar);
  double* s_uin = sm + TL::kUin;
  double* s_un = sm + TL::kUn;
  double* s_f = sm + TL::kF;
  double* s_vel = sm + TL::kVel;
  double* s_H = sm + TL::kH;
  double* s_sr = sm + TL::kSr;
  double* s_L = sm + TL::kL;
  double* s_rs = sm + TL::kRs;
  double* s_F = sm + TL::kFs;
  double* s_h = sm + TL::kHf;
  double* s_red = sm + TL::kRed;

  const int tid = threadIdx.x;
  Ctl* ctl = a.ctl;
  const long long n = a.n;
  if (j0 >= n) return true;
  const int Tc = (int)((n - j0 < T) ? (n - j0) : T);
  const int ni = Tc + 1;
  // ---- step control: is this step active, and its dt
  double dt = 0.0;
  if (STAGE != STAGE_RHS) {
    if (STAGE == STAGE_RK1) {
      const bool act = (ctl->status == 0) && (ctl->t < ctl->t_final);
      if (!act) {
        if (first_tile && tid == 0) ctl->active = 0;
        return true;
      }
    } else if (ctl->active == 0) {
      return true;
    }
    if (first_tile && tid < 8) ctl->amax[(STAGE + 2) % 3][tid] = 0ull;
  }
  const int slot_in = (STAGE == STAGE_RHS) ? 0 : STAGE;
  double alpha[M];
#pragma unroll
  for (int s = 0; s < M; ++s) alpha[s] = bits_to_double(ctl->amax[slot_in][s]);
  if (STAGE == STAGE_RK1) {
    const double smax = (FLUX == WT_FLUX_EULER1D) ? ((alpha[0] < alpha[M - 1]) ? alpha[M - 1] : alpha[0]) : alpha[0];
    dt = ctl->dt_fixed > 0.0 ? ctl->dt_fixed : MATH::cfl_dt(ctl->cfl, a.dx, smax);
    const double rem = ctl->t_final - ctl->t;
    if (rem < dt) dt = rem;
    if (first_tile && tid == 0) {
      ctl->dt = dt;
      ctl->active = 1;
    }
  } else if (STAGE != STAGE_RHS) {
    dt = ctl->dt;
  }

  // ---- A: stage the window [j0 - 3, j0 + Tc + 3) of every plane (16-byte aligned start)
  const long long s0 = j0 & ~1LL;
  const int off = (int)(j0 - s0);
  const int cells = Tc + 2 * G;
  const int len = (off + cells + 1) & ~1;
  constexpr bool kNeedUn = (STAGE == STAGE_RK2 || STAGE == STAGE_RK3);
  if (tid == 0) {
    const uint32_t bytes = (uint32_t)len * 8u;
    mbar_arrive_expect_tx(bar, bytes * (kNeedUn ? 2 * M : M));
#pragma unroll
    for (int c = 0; c < M; ++c) bulk_g2s(s_uin + c * W, a.uin + c * a.pitch + s0, bytes, bar);
    if (kNeedUn) {
#pragma unroll
      for (int c = 0; c < M; ++c) bulk_g2s(s_un + c * W, a.un + c * a.pitch + s0, bytes, bar);
    }
  }
  const bool ok = mbar_wait_bounded(bar, phase);
  if (__syncthreads_or(ok ? 0 : 1)) {
    if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
    mbar_wait_bounded(bar, phase);
    return false;
  }
  phase ^= 1u;

  // ---- B: per-cell quantities
  for (int k = tid; k < cells; k += NT) {
    if (FLUX == WT_FLUX_EULER1D) {
      double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
      double f[3], u, H, sr, p;
      MATH::euler_cell(U, a.gamma, f, u, H, sr, p);
      if (!finite3(U)) flag_error(ctl, WT_ERR_NONPHYSICAL);
      s_f[k] = f[0];
      s_f[W + k] = f[1];
      s_f[2 * W + k] = f[2];
      s_vel[k] = u;
      s_H[k] = H;
      s_sr[k] = sr;
    } else {
      const double x = s_uin[off + k];
      if (!isfinite(x)) flag_error(ctl, WT_ERR_NONPHYSICAL);
      s_f[k] = (FLUX == WT_FLUX_ADVECTION) ? MATH::flux_advection(a.adv_speed, x) : MATH::flux_burgers(x);
    }
  }
  __syncthreads();

  // ---- C0: Roe average and left eigenvectors per interface (interface i: cells i+2 | i+3)
  if (FLUX == WT_FLUX_EULER1D) {
    for (int i = tid; i < ni; i += NT) {
      double L[9], rs[3];
      MATH::roe(s_sr[i + 2], s_vel[i + 2], s_H[i + 2], s_sr[i + 3], s_vel[i + 3], s_H[i + 3], a.gamma, L, rs);
#pragma unroll
      for (int e = 0; e < 9; ++e) s_L[e * NI + i] = L[e];
#pragma unroll
      for (int e = 0; e < 3; ++e) s_rs[e * NI + i] = rs[e];
    }
    __syncthreads();
  }

  // ---- C1: per (interface, field) reconstruction on both sides
  for (int item = tid; item < M * ni; item += NT) {
    const int s = item / ni;
    const int i = item - s * ni;
    double vp[6], vm[6];
    if (FLUX == WT_FLUX_EULER1D) {
      double l[3] = {s_L[(3 * s) * NI + i], s_L[(3 * s + 1) * NI + i], s_L[(3 * s + 2) * NI + i]};
      double al = (s == 0) ? alpha[0] : ((s == 1) ? alpha[1] : alpha[M - 1]);
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) {
        const int k = i + kk;
        double f[3] = {s_f[k], s_f[W + k], s_f[2 * W + k]};
        double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
        MATH::project3(l, f, U, al, vp[kk], vm[kk]);
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) MATH::project1(s_f[i + kk], s_uin[off + i + kk], alpha[0], vp[kk], vm[kk]);
    }
    double qm[6];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) qm[kk] = vm[5 - kk];
    const double Fp = MATH::weno(vp, a.eps, a.alpha_R);
    const double Fm = MATH::weno(qm, a.eps, a.alpha_R);
    s_F[s * NI + i] = Fp + Fm;
  }
  __syncthreads();

  // ---- D: interface fluxes h_{j+1/2} = R (F+ + F-)
  const double* hsrc = s_F;
  if (FLUX == WT_FLUX_EULER1D) {
    for (int i = tid; i < ni; i += NT) {
      double rs[3] = {s_rs[i], s_rs[NI + i], s_rs[2 * NI + i]};
      double F[3] = {s_F[i], s_F[NI + i], s_F[2 * NI + i]};
      double h[3];
      MATH::backproject(rs, F, h);
#pragma unroll
      for (int c = 0; c < 3; ++c) s_h[c * NI + i] = h[c];
    }
    __syncthreads();
    hsrc = s_h;
  }

  // ---- E: flux difference, RK combine, ghost images, wave speeds
  double vmax[M];
#pragma unroll
  for (int s = 0; s < M; ++s) vmax[s] = 0.0;
  for (int t = tid; t < Tc; t += NT) {
    const long long j = j0 + t;
    double uo[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const double L = MATH::flux_diff(hsrc[c * NI + t + 1], hsrc[c * NI + t], a.dx, a.inv_dx);
      if (STAGE == STAGE_RHS) {
        a.Lout[c * a.lout_stride + j] = L;
      } else {
        const double us = s_uin[c * W + off + t + G];
        const double un = kNeedUn ? s_un[c * W + off + t + G] : us;
        uo[c] = MATH::template rk<(STAGE == STAGE_RHS ? 0 : STAGE)>(un, us, dt, L);
      }
    }
    if (STAGE != STAGE_RHS) {
#pragma unroll
      for (int c = 0; c < M; ++c) a.uout[c * a.pitch + j + G] = uo[c];
      // ghost images of this cell in the output
      if (j < G || j >= n - G) {
#pragma unroll
        for (int c = 0; c < M; ++c) {
          double* o = a.uout + c * a.pitch;
          const double v = uo[c];
          const double vr = (c == 1) ? -v : v;
          if (a.bc_hi == WT_BC_PERIODIC && j < G) o[n + j + G] = v;
          if (a.bc_lo == WT_BC_PERIODIC && j >= n - G) o[j - n + G] = v;
          if (a.bc_lo == WT_BC_OUTFLOW && j == 0) o[0] = o[1] = o[2] = v;
          if (a.bc_hi == WT_BC_OUTFLOW && j == n - 1) o[n + 3] = o[n + 4] = o[n + 5] = v;
          if (a.bc_lo == WT_BC_REFLECTIVE && j < G) o[2 - j] = vr;
          if (a.bc_hi == WT_BC_REFLECTIVE && j >= n - G) o[2 * n + 2 - j] = vr;
        }
      }
      if (FLUX == WT_FLUX_EULER1D) {
        double lam[3];
        MATH::euler_speeds(uo, a.gamma, lam);
        if (!finite3(uo)) flag_error(ctl, WT_ERR_NONPHYSICAL);
#pragma unroll
        for (int s = 0; s < M; ++s) vmax[s] = (vmax[s] < lam[s]) ? lam[s] : vmax[s];
      } else {
        const double lam = (FLUX == WT_FLUX_ADVECTION) ? fabs(a.adv_speed) : fabs(uo[0]);
        if (!isfinite(uo[0])) flag_error(ctl, WT_ERR_NONPHYSICAL);
        vmax[0] = (vmax[0] < lam) ? lam : vmax[0];
      }
    }
  }
  if (STAGE != STAGE_RHS) {
    block_max_atomic<M>(vmax, s_red, ctl->amax[(STAGE + 1) % 3]);
    if (STAGE == STAGE_RK3 && first_tile && tid == 0) {
      ctl->t = ctl->t + dt;
      ctl->steps = ctl->steps + 1;
    }
  }
  return true;
}

template <class MATH, int FLUX, int STAGE, int T>
__global__ void __launch_bounds__(Tile1D<T, FluxM<FLUX>::m>::NT) stage1d_kernel(const Stage1DArgs a) {
  using TL = Tile1D<T, FluxM<FLUX>::m>;
  extern __shared__ __align__(16) double sm[];
  pdl_launch_dependents();
  if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t*>(sm + TL::kBar), 1);
  __syncthreads();
  pdl_wait();
  uint32_t phase = 0;
  stage1d_tile<MATH, FLUX, STAGE, T>(a, (long long)blockIdx.x * T, blockIdx.x == 0, sm, phase);
}

// Batched stage: a persistent grid walks a table of (problem, tile) work items over many
// independent problems, each with its own grid, boundary conditions, alphas and dt.
template <class MATH, int FLUX, int STAGE, int T>
__global__ void __launch_bounds__(Tile1D<T, FluxM<FLUX>::m>::NT) stage1d_batched_kernel(const BatchArgs b) {
  using TL = Tile1D<T, FluxM<FLUX>::m>;
  extern __shared__ __align__(16) double sm[];
  pdl_launch_dependents();
  if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t*>(sm + TL::kBar), 1);
  __syncthreads();
  pdl_wait();
  uint32_t phase = 0;
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    const int2 item = b.tiles[t];
    const BatchSeg sg = b.segs[item.x];
    Stage1DArgs a;
    a.uin = b.uin + sg.poff;
    a.un = b.un + sg.poff;
    a.uout = b.uout + sg.poff;
    a.Lout = nullptr;
    a.n = sg.n;
    a.pitch = b.pitch;
    a.lout_stride = 0;
    a.dx = sg.dx;
    a.inv_dx = sg.inv_dx;
    a.gamma = b.gamma;
    a.adv_speed = b.adv_speed;
    a.eps = b.eps;
    a.alpha_R = b.alpha_R;
    a.bc_lo = sg.bc_lo;
    a.bc_hi = sg.bc_hi;
    a.ctl = b.ctl + item.x;
    const long long j0 = (long long)item.y * T;
    if (!stage1d_tile<MATH, FLUX, STAGE, T>(a, j0, j0 == 0, sm, phase)) return;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Host-side launchers, instantiated per policy
// ---------------------------------------------------------------------------------------

// Launch with programmatic stream serialization: the kernel may start while its predecessor in
// the stream finishes, and waits for it with griddepcontrol.wait before touching its outputs.
template <class K, class A>
cudaError_t launch_pdl(K kern, dim3 grid, dim3 block, size_t smem, cudaStream_t st, const A& arg) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, arg);
}
template <class MATH, int FLUX, int STAGE, int T>
cudaError_t launch_stage1d_t(const Stage1DArgs& a, cudaStream_t st) {
  using TL = Tile1D<T, FluxM<FLUX>::m>;
  static_assert(TL::bytes <= 48 * 1024, "tile exceeds the default dynamic shared memory limit");
  auto kern = stage1d_kernel<MATH, FLUX, STAGE, T>;
  const unsigned grid = (unsigned)((a.n + T - 1) / T);
  return launch_pdl(kern, dim3(grid), dim3(TL::NT), TL::bytes, st, a);
}

template <class MATH, int FLUX, int T>
cudaError_t launch_stage1d_flux(int stage, const Stage1DArgs& a, cudaStream_t st) {
  switch (stage) {
    case STAGE_RK1: return launch_stage1d_t<MATH, FLUX, STAGE_RK1, T>(a, st);
    case STAGE_RK2: return launch_stage1d_t<MATH, FLUX, STAGE_RK2, T>(a, st);
    case STAGE_RK3: return launch_stage1d_t<MATH, FLUX, STAGE_RK3, T>(a, st);
    case STAGE_RHS: return launch_stage1d_t<MATH, FLUX, STAGE_RHS, T>(a, st);
  }
  return cudaErrorInvalidValue;
}

template <class MATH>
cudaError_t launch_stage1d_policy(int flux, int stage, int tile, const Stage1DArgs& a, cudaStream_t st) {
  if (flux == WT_FLUX_EULER1D) {
    if (tile == 31) return launch_stage1d_flux<MATH, WT_FLUX_EULER1D, 31>(stage, a, st);
    if (tile == 63) return launch_stage1d_flux<MATH, WT_FLUX_EULER1D, 63>(stage, a, st);
    if (tile == 127) return launch_stage1d_flux<MATH, WT_FLUX_EULER1D, 127>(stage, a, st);
  } else if (flux == WT_FLUX_ADVECTION) {
    if (tile == 63) return launch_stage1d_flux<MATH, WT_FLUX_ADVECTION, 63>(stage, a, st);
    if (tile == 127) return launch_stage1d_flux<MATH, WT_FLUX_ADVECTION, 127>(stage, a, st);
  } else if (flux == WT_FLUX_BURGERS) {
    if (tile == 63) return launch_stage1d_flux<MATH, WT_FLUX_BURGERS, 63>(stage, a, st);
    if (tile == 127) return launch_stage1d_flux<MATH, WT_FLUX_BURGERS, 127>(stage, a, st);
  }
  return cudaErrorInvalidValue;
}

template <class MATH>
cudaError_t launch_alpha1d_policy(int flux, const double* u, long long n, long long pitch, double gamma, double adv,
                                  Ctl* ctl, int slot, cudaStream_t st) {
  long long blocks = (n + 255) / 256;
  if (blocks > 1216) blocks = 1216;  // 8 per SM is plenty for a grid-stride reduction
  if (blocks < 1) blocks = 1;
  if (flux == WT_FLUX_EULER1D)
    alpha1d_kernel<MATH, WT_FLUX_EULER1D><<<(unsigned)blocks, 256, 0, st>>>(u, n, pitch, gamma, adv, ctl, slot);
  else if (flux == WT_FLUX_ADVECTION)
    alpha1d_kernel<MATH, WT_FLUX_ADVECTION><<<(unsigned)blocks, 256, 0, st>>>(u, n, pitch, gamma, adv, ctl, slot);
  else if (flux == WT_FLUX_BURGERS)
    alpha1d_kernel<MATH, WT_FLUX_BURGERS><<<(unsigned)blocks, 256, 0, st>>>(u, n, pitch, gamma, adv, ctl, slot);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <class MATH, int FLUX, int STAGE, int T>
cudaError_t launch_stage1d_batched_t(const BatchArgs& b, int grid, cudaStream_t st) {
  using TL = Tile1D<T, FluxM<FLUX>::m>;
  return launch_pdl(stage1d_batched_kernel<MATH, FLUX, STAGE, T>, dim3(grid), dim3(TL::NT), TL::bytes, st, b);
}

template <class MATH, int FLUX, int T>
cudaError_t launch_stage1d_batched_flux(int stage, const BatchArgs& b, int grid, cudaStream_t st) {
  switch (stage) {
    case STAGE_RK1: return launch_stage1d_batched_t<MATH, FLUX, STAGE_RK1, T>(b, grid, st);
    case STAGE_RK2: return launch_stage1d_batched_t<MATH, FLUX, STAGE_RK2, T>(b, grid, st);
    case STAGE_RK3: return launch_stage1d_batched_t<MATH, FLUX, STAGE_RK3, T>(b, grid, st);
  }
  return cudaErrorInvalidValue;
}

template <class MATH>
cudaError_t launch_stage1d_batched_policy(int flux, int stage, int tile, const BatchArgs& b, int grid,
                                          cudaStream_t st) {
  if (flux == WT_FLUX_EULER1D) {
    if (tile == 31) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 31>(stage, b, grid, st);
    if (tile == 63) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 63>(stage, b, grid, st);
    if (tile == 127) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 127>(stage, b, grid, st);
  } else if (flux == WT_FLUX_ADVECTION) {
    if (tile == 63) return launch_stage1d_batched_flux<MATH, WT_FLUX_ADVECTION, 63>(stage, b, grid, st);
    if (tile == 127) return launch_stage1d_batched_flux<MATH, WT_FLUX_ADVECTION, 127>(stage, b, grid, st);
  } else if (flux == WT_FLUX_BURGERS) {
    if (tile == 63) return launch_stage1d_batched_flux<MATH, WT_FLUX_BURGERS, 63>(stage, b, grid, st);
    if (tile == 127) return launch_stage1d_batched_flux<MATH, WT_FLUX_BURGERS, 127>(stage, b, grid, st);
  }
  return cudaErrorInvalidValue;
}

template <class MATH, int FLUX, int T>
int batched_occupancy_t() {
  using TL = Tile1D<T, FluxM<FLUX>::m>;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage1d_batched_kernel<MATH, FLUX, STAGE_RK2, T>, TL::NT,
                                                    TL::bytes) != cudaSuccess)
    return 0;
  return nb;
}

template <class MATH>
int batched_occupancy_policy(int flux, int tile) {
  if (flux == WT_FLUX_EULER1D) {
    if (tile == 31) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 31>();
    if (tile == 63) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 63>();
    if (tile == 127) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 127>();
  } else if (flux == WT_FLUX_ADVECTION) {
    if (tile == 63) return batched_occupancy_t<MATH, WT_FLUX_ADVECTION, 63>();
    if (tile == 127) return batched_occupancy_t<MATH, WT_FLUX_ADVECTION, 127>();
  } else if (flux == WT_FLUX_BURGERS) {
    if (tile == 63) return batched_occupancy_t<MATH, WT_FLUX_BURGERS, 63>();
    if (tile == 127) return batched_occupancy_t<MATH, WT_FLUX_BURGERS, 127>();
  }
  return 0;
}

template <class MATH>
cudaError_t launch_alpha1d_batched_policy(int flux, const double* u, long long pitch, const BatchSeg* segs, int nprob,
                                          long long maxn, double gamma, double adv, Ctl* ctl, cudaStream_t st) {
  long long bx = (maxn + 255) / 256;
  if (bx > 64) bx = 64;
  dim3 grid((unsigned)(bx < 1 ? 1 : bx), (unsigned)nprob);
  if (flux == WT_FLUX_EULER1D)
    alpha1d_batched_kernel<MATH, WT_FLUX_EULER1D><<<grid, 256, 0, st>>>(u, pitch, segs, gamma, adv, ctl);
  else if (flux == WT_FLUX_ADVECTION)
    alpha1d_batched_kernel<MATH, WT_FLUX_ADVECTION><<<grid, 256, 0, st>>>(u, pitch, segs, gamma, adv, ctl);
  else if (flux == WT_FLUX_BURGERS)
    alpha1d_batched_kernel<MATH, WT_FLUX_BURGERS><<<grid, 256, 0, st>>>(u, pitch, segs, gamma, adv, ctl);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace wt
