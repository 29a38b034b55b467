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

// Tile geometry: T cells, T + 1 interfaces, m threads per interface (one per field), or with
// SPLIT = 2 (the step-blocked tiles) a pair of adjacent threads per (interface, field), one
// per side of the reconstruction (two warps per SMSP where the tile fills one warp per SMSP).
// IPT > 1 (stage and batched tiles): each thread carries IPT (interface, field) items, so the
// tile has about a 1/IPT of the threads and each thread IPT times the work of every phase.
// LATE (the stage and batched tiles, kStage): the eigenvector buffer, dead once phase C1 is
// done, also holds the interface fluxes h of phase D and the window of u^n, which is copied in
// after phase C1 (stages 2, 3) instead of with the stage input, so a tile needs about a sixth
// less shared memory and one more tile fits on an SM.
// DP (the fast policy's 1D Euler tiles, MATH::kDiffProj): the differences of f and u between
// neighbouring cells, taken once per stage after phase C0; those of f go to the planes of the
// per-cell Roe inputs (dead once phase C0 is done), those of u to planes of their own.
template <int T, int M, int SPLIT = 1, int IPT = 1, bool LATE = false, bool DP = false>
struct Tile1D {
  static_assert(IPT == 1 || SPLIT == 1, "thread pairs carry one item");
  static_assert(!LATE || SPLIT == 1, "the late u^n window is for the stage tiles");
  static constexpr int W = (T + 9) & ~1;              // staged window: T + 6 cells + alignment slack, even
  static constexpr int NI = T + 1;
  static constexpr int NT = SPLIT * ((M * NI + 32 * IPT - 1) / (32 * IPT)) * 32;
  // shared-memory layout in doubles
  static constexpr int kBar = 0;
  static constexpr int kUin = 2;
  static constexpr int kF = kUin + (LATE ? 1 : 2) * M * W;
  static constexpr int kVel = kF + M * W;
  static constexpr int kH = kVel + W;
  static constexpr int kSr = kH + W;
  static constexpr int kL = kSr + W;
  static constexpr int kRs = kL + 9 * NI;
  static constexpr int kFs = kRs + 3 * NI;       // F+ [M][NI], then F- [M][NI]
  static constexpr int kHf = LATE ? kL : kFs + 2 * M * NI;
  static constexpr int kUn = LATE ? kL + M * NI : kUin + M * W;
  static_assert(!LATE || (M * NI + M * W <= 9 * NI && (kUn % 2) == 0), "h and u^n fit the eigenvector buffer");
  // (resident and step-blocked tiles, latency-bound: f's differences get planes of their own
  // and are taken during phase C0)
  static constexpr int kDu = LATE ? kFs + 2 * M * NI : kHf + M * NI;  // DP: [M][W] u_{k+1} - u_k
  static constexpr int kDf = LATE ? kVel : kDu + M * W;               // DP: [M][W] f_{k+1} - f_k
  static_assert(!DP || M == 3, "differences first: 1D Euler tiles");
  static constexpr int kRed = kDu + (DP ? (LATE ? 1 : 2) * M * W : 0);
  static constexpr int kQn = kRed + 4 * 32;      // queue length (int)
  // queue of reconstructions still to be completed: one slot per thread, fewer if the tile
  // would pass 48 KB (the rest are completed in place).  A record holds the weights' inputs
  // (9 doubles), or with SPLIT = 2 a stencil's differences (15 doubles, FastMath::kDeferRec)
  static constexpr int REC = (SPLIT == 2) ? 15 : 9;
  static constexpr int kQ = kQn + 2;             // queue records [REC][QCAP]
  static constexpr int kQFit = ((48 * 1024 / 8 - kQ) * 2) / (2 * REC + 1);
  static constexpr int QCAP = (kQFit < NT ? kQFit : NT) & ~1;
  static constexpr int kQi = kQ + REC * QCAP;    // record destinations (int)
  static constexpr int kTotal = kQi + QCAP / 2;
  static constexpr size_t bytes = sizeof(double) * kTotal;
};

// the tile of a policy and flux: differences first where the policy takes them (1D Euler)
template <class MATH, int FLUX, int T, int SPLIT = 1, int IPT = 1, bool LATE = false>
using TileOf = Tile1D<T, FluxM<FLUX>::m, SPLIT, IPT, LATE, MATH::kDiffProj && FLUX == WT_FLUX_EULER1D>;

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
  unsigned long long v[M];
#pragma unroll
  for (int s = 0; s < M; ++s) v[s] = 0ull;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    if (FLUX == WT_FLUX_EULER1D) {
      double U[3] = {u[j + G], u[pitch + j + G], u[2 * pitch + j + G]};
      double lam[3];
      MATH::euler_speeds(U, gamma, lam);
      if (!finite3(U)) flag_error(ctl, WT_ERR_NONPHYSICAL);
#pragma unroll
      for (int s = 0; s < M; ++s) key_max(v[s], lam[s]);
    } else {
      double x = u[j + G];
      double lam = (FLUX == WT_FLUX_ADVECTION) ? fabs(adv) : fabs(x);
      if (!isfinite(x)) flag_error(ctl, WT_ERR_NONPHYSICAL);
      key_max(v[0], lam);
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
  unsigned long long v[M];
#pragma unroll
  for (int s = 0; s < M; ++s) v[s] = 0ull;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < sg.n;
       j += (long long)gridDim.x * blockDim.x) {
    if (FLUX == WT_FLUX_EULER1D) {
      double U[3] = {up[j + G], up[pitch + j + G], up[2 * pitch + j + G]};
      double lam[3];
      MATH::euler_speeds(U, gamma, lam);
      if (!finite3(U)) flag_error(c, WT_ERR_NONPHYSICAL);
#pragma unroll
      for (int s = 0; s < M; ++s) key_max(v[s], lam[s]);
    } else {
      double x = up[j + G];
      double lam = (FLUX == WT_FLUX_ADVECTION) ? fabs(adv) : fabs(x);
      if (!isfinite(x)) flag_error(c, WT_ERR_NONPHYSICAL);
      key_max(v[0], lam);
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
// How a tile's stage sits in its kernel:
//   kStage        one launch per stage; the window is bulk-copied in, outputs go to global memory
//   kResident     persistent kernel: the stage output of the tile's cells also stays in shared
//                 memory (s_uin, and s_un after the last stage); halos are exchanged per stage
//   kStepBlocked  persistent kernel whose tiles carry 9 redundant halo cells per side, so the
//                 three stages of an RK step need no halo exchange: the computed range shrinks
//                 by 3 cells per side per stage, only the tile's own cells contribute to the
//                 alphas, and only the last stage writes global memory
enum { kStage = 0, kResident = 1, kStepBlocked = 2 };

// Gathers the alpha mailbox words of `ncta` CTAs from one stage slot (4 words per CTA) with a
// bounded wait (`limit` SM clocks) until every word carries the parity bit `pbit`; called by a
// whole warp.  Lane l takes CTAs l, l + 32, ...; a CTA's four words are one 32-byte load
// (`slot` is 32-byte aligned), and all loads of a round are issued before any is tested, so a
// polling round costs one trip to L2 however many CTAs a lane covers.  After the first round
// only the CTAs whose words do not all carry the parity yet are read again.  On return every
// lane holds the maxima of words 0..M-1 (keys) in mk and the OR of words 3 in stv (its own
// CTAs' only; the caller reduces it).  Returns 1, or 0 (every lane) if the wait gave up.
template <int M>
__device__ __forceinline__ int gather_alpha_words(const unsigned long long* slot, int ncta, unsigned long long pbit,
                                                  long long limit, unsigned long long (&mk)[M],
                                                  unsigned long long& stv) {
  constexpr int kPL = 5;  // CTAs per lane in one batch (160 CTAs, more in further batches)
  const unsigned long long low63 = ~(1ull << 63);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int f = 0; f < M; ++f) mk[f] = 0ull;
  stv = 0ull;
  int ok = 1;
  const long long start = clock64();
  for (int base = 0; base < ncta && ok; base += 32 * kPL) {
    unsigned long long w[kPL][4];
    unsigned int need = 0u;  // CTAs of this batch whose words are not all there yet
#pragma unroll
    for (int q = 0; q < kPL; ++q) {
#pragma unroll
      for (int e = 0; e < 4; ++e) w[q][e] = pbit;
      if (base + 32 * q + lane < ncta) need |= 1u << q;
    }
    while (need != 0u) {
#pragma unroll
      for (int q = 0; q < kPL; ++q)
        if (need & (1u << q)) ld_relaxed_v4_u64(slot + 4 * (base + 32 * q + lane), w[q]);
#pragma unroll
      for (int q = 0; q < kPL; ++q) {
        bool ready = true;
#pragma unroll
        for (int e = 0; e < 4; ++e) ready = ready && ((w[q][e] ^ pbit) >> 63) == 0ull;
        if (ready) need &= ~(1u << q);
      }
      if (need != 0u && clock64() - start > limit) {
        ok = 0;
        break;
      }
    }
#pragma unroll
    for (int q = 0; q < kPL; ++q) {
#pragma unroll
      for (int f = 0; f < M; ++f) {
        const unsigned long long k = w[q][f] & low63;
        mk[f] = (mk[f] < k) ? k : mk[f];
      }
      stv |= w[q][3] & low63;
    }
  }
  ok = __all_sync(0xffffffffu, ok);
#pragma unroll
  for (int f = 0; f < M; ++f) mk[f] = warp_max_key_redux(mk[f]);
  return ok;
}

// How a step-blocked stage obtains its alphas and hands on its output.  The alphas come
// from a mailbox of 8-byte words, four per CTA and stage slot: the keys of the CTA's maxima
// and, at a step's first stage, whether it has seen a failure, each with the step's parity
// in bit 63.  Every CTA writes its words, then reads every CTA's words of the slot until
// all carry this step's parity (a word with the other parity is still the previous
// step's); the words are single-copy atomic, so no fence or arrival counter is needed.
// clear >= 0 marks the first CTA (it records dt).  first_stage: the stage opens an RK step,
// whose dt (from these alphas, cfl or dt_fixed, clipped at t_final) is set after the wait.
// Stage 3 also writes u^{n+1} of the CTA's own cells to the halo mailbox, as two words
// (high and low 32 bits of the double) tagged with `tag` in their upper 32 bits.
struct AlphaWait {
  unsigned long long target;
  int slot, clear;
  int first_stage;
  double cfl, dt_fixed, t, t_final;
  unsigned long long* amb;   // alpha mailbox [3][gridDim.x][4]
  unsigned long long par;    // parity of the step (0 or 1)
  unsigned long long* hmb_hi;
  unsigned long long* hmb_lo;
  unsigned int tag;
};

// Phases B-E of one stage over the cells [js, js + Ts) whose window [js - 3, js + Ts + 3) is
// in shared memory at s_uin[off...] (s_un for stages 2 and 3), with the stage's dt.  The
// wave speeds of the cells of [own_lo, own_hi) go to the alpha ring: in kStage and kResident
// those of the stage output (phase E, next slot, atomics at the end of the stage); in
// kStepBlocked those of the stage input (phase B, this stage's slot of the alpha mailbox,
// written and then gathered by the last warp while the others go on).  Returns false if a
// wait for the alphas timed out (the flag word then holds 2) or, at the first stage of a
// step-blocked RK step, if some CTA has seen a failure (flag word 3): the step is not taken.
template <class MATH, int FLUX, int STAGE, int T, int MODE, int IPT = 1, bool REC = false>
__device__ __forceinline__ bool stage1d_compute(const Stage1DArgs& a, const long long js, const int Ts, const int off,
                                                const long long own_lo, const long long own_hi,
                                                double (&alpha)[FluxM<FLUX>::m], double& dt, double* sm,
                                                const AlphaWait aw, uint32_t* phase = nullptr) {
  constexpr int M = FluxM<FLUX>::m;
  // step-blocked tiles split each reconstruction pair over two threads (see phase C1)
  constexpr int SPLIT = (MODE == kStepBlocked) ? 2 : 1;
  static_assert(IPT == 1 || MODE != kStepBlocked, "the step-blocked tiles carry one item per thread pair");
  constexpr bool LATE = (MODE == kStage);
  using TL = TileOf<MATH, FLUX, T, SPLIT, IPT, LATE>;
  constexpr int W = TL::W, NI = TL::NI, NT = TL::NT;
  constexpr bool DP = MATH::kDiffProj && FLUX == WT_FLUX_EULER1D;  // differences first (phase C1)
  static_assert(NT * IPT >= SPLIT * M * NI, "IPT (interface, field) items per thread (one per thread pair with SPLIT = 2)");
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
  const int Tc = Ts;
  const int ni = Tc + 1;
  const int cells = Tc + 2 * G;
  constexpr bool kNeedUn = (STAGE == STAGE_RK2 || STAGE == STAGE_RK3);

  // ---- B: per-cell quantities (step-blocked: also ghost images of the stage input).
  // Step-blocked: the last warp (the speed warp) meanwhile takes the wave speeds of the CTA's
  // own cells, writes their maxima to this stage's slot of the alpha mailbox, gathers every
  // CTA's words (gather_alpha_words) and leaves the alphas in shared memory (s_alpha,
  // s_aflag).  Its lanes release the other warps from phase B first (named barrier 1).
  constexpr int kSW = NT / 32 - 1;  // the speed warp (step-blocked)
  unsigned long long* s_alpha = reinterpret_cast<unsigned long long*>(s_red);
  int* s_aflag = reinterpret_cast<int*>(sm + TL::kQn) + 1;
  if (tid == 0) *reinterpret_cast<int*>(sm + TL::kQn) = 0;
  if (MODE == kStepBlocked && (tid >> 5) == kSW) {
    const int lane = tid & 31;
    named_barrier_arrive(1, NT);  // phase B does not wait for the speeds
    unsigned long long vb[M];
#pragma unroll
    for (int f = 0; f < M; ++f) vb[f] = 0ull;
    const int own0 = off + (int)(own_lo - js) + G;  // window position of the first own cell
    const int nown = (int)(own_hi - own_lo);
    for (int q = lane; q < nown; q += 32) {
      double U[M];
#pragma unroll
      for (int c = 0; c < M; ++c) U[c] = s_uin[c * W + own0 + q];
      if (FLUX == WT_FLUX_EULER1D) {
        double lam[3];
        MATH::euler_speeds(U, a.gamma, lam);
#pragma unroll
        for (int f = 0; f < M; ++f) key_max(vb[f], lam[f]);
      } else {
        key_max(vb[0], (FLUX == WT_FLUX_ADVECTION) ? fabs(a.adv_speed) : fabs(U[0]));
      }
    }
#pragma unroll
    for (int f = 0; f < M; ++f) vb[f] = warp_max_key_redux(vb[f]);
    // publish: words 0..M-1 the keys of this CTA's maxima, word 3 (first stage) its view of
    // the status, all with the step's parity in bit 63
    const unsigned long long pbit = aw.par << 63;
    unsigned long long* slot = aw.amb + (size_t)STAGE * 4 * gridDim.x;
    if (lane < 4) {
      unsigned long long w = 0ull;
#pragma unroll
      for (int f = 0; f < M; ++f)
        if (lane == f) w = vb[f];
      if (lane == 3 && aw.first_stage) w = (__ldcg(&ctl->status) != 0) ? 1ull : 0ull;
      st_relaxed_u64(slot + 4 * blockIdx.x + lane, w | pbit);
    }
    // gather every CTA's words of this slot, bounded wait
    unsigned long long mk[M], stv = 0ull;
    const int ok = gather_alpha_words<M>(slot, (int)gridDim.x, pbit, kWaitLimit, mk, stv);
    const bool stop = __any_sync(0xffffffffu, stv != 0ull) && aw.first_stage;
    if (lane == 0) {
#pragma unroll
      for (int f = 0; f < M; ++f) s_alpha[f] = mk[f];
      *s_aflag = !ok ? 2 : (stop ? 3 : 1);
    }
  } else {
    const int nb = (MODE == kStepBlocked) ? NT - 32 : NT;  // threads of phase B
    for (int k = tid; k < cells; k += nb) {
      double U[M];
#pragma unroll
      for (int c = 0; c < M; ++c) U[c] = s_uin[c * W + off + k];
      if (MODE == kStepBlocked) {
        // a ghost cell of a non-periodic end takes the image of the stage input
        const long long x = js - G + k;
        const bool lo_g = x < 0 && a.bc_lo != WT_BC_PERIODIC, hi_g = x >= n && a.bc_hi != WT_BC_PERIODIC;
        if (lo_g || hi_g) {
          const int bc = hi_g ? a.bc_hi : a.bc_lo;
          const long long xs = (bc == WT_BC_OUTFLOW) ? (hi_g ? n - 1 : 0) : (hi_g ? 2 * n - 1 - x : -1 - x);
          const int ks = k + (int)(xs - x);
#pragma unroll
          for (int c = 0; c < M; ++c) {
            const double v = s_uin[c * W + off + ks];
            U[c] = (bc == WT_BC_REFLECTIVE && c == 1) ? -v : v;
            s_uin[c * W + off + k] = U[c];
          }
        }
      }
      if (FLUX == WT_FLUX_EULER1D) {
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
        const double xv = U[0];
        if (!isfinite(xv)) flag_error(ctl, WT_ERR_NONPHYSICAL);
        s_f[k] = (FLUX == WT_FLUX_ADVECTION) ? MATH::flux_advection(a.adv_speed, xv) : MATH::flux_burgers(xv);
      }
    }
    if (MODE == kStepBlocked) named_barrier_sync(1, NT);
  }
  if (MODE != kStepBlocked) __syncthreads();
  // step-blocked scalar fluxes have no phase C0: the alphas are awaited here
  if (MODE == kStepBlocked && FLUX != WT_FLUX_EULER1D) __syncthreads();
  // Step-blocked: where the speed warp holds no phase-C1 item (stages whose items fit in the
  // other warps), phase C0 closes without it, so the other warps' alpha-free products overlap
  // its gather; it joins them before the alphas are read.  The condition is the same for
  // every thread of the block.
  const bool sw_free = MODE == kStepBlocked && SPLIT * M * ni <= NT - 32;
  auto c0_barrier = [&]() {
    if (!sw_free) {
      __syncthreads();
    } else if ((tid >> 5) != kSW) {
      named_barrier_sync(2, NT - 32);
    }
  };

  // ---- C0: Roe average and left eigenvectors per interface (interface i: cells i+2 | i+3);
  // with MATH::kRoeRows one row of the matrix per thread
  if (FLUX == WT_FLUX_EULER1D && MATH::kRoeRows) {
    if (tid < 3 * ni) {
      const int row = tid / ni, i = tid - row * ni;
      double l[3], rs[3];
      MATH::roe_row(s_sr[i + 2], s_vel[i + 2], s_H[i + 2], s_sr[i + 3], s_vel[i + 3], s_H[i + 3], a.gamma, row, l, rs);
#pragma unroll
      for (int e = 0; e < 3; ++e) s_L[(3 * row + e) * NI + i] = l[e];
      if (row == 0) {
#pragma unroll
        for (int e = 0; e < 3; ++e) s_rs[e * NI + i] = rs[e];
      }
    }
    c0_barrier();
  } else if (FLUX == WT_FLUX_EULER1D) {
    for (int i = tid; i < ni; i += NT) {
      double L[9], rs[3];
      MATH::roe(s_sr[i + 2], s_vel[i + 2], s_H[i + 2], s_sr[i + 3], s_vel[i + 3], s_H[i + 3], a.gamma, L, rs);
#pragma unroll
      for (int e = 0; e < 9; ++e) s_L[e * NI + i] = L[e];
#pragma unroll
      for (int e = 0; e < 3; ++e) s_rs[e * NI + i] = rs[e];
    }
    if constexpr (DP && MODE != kStage) {
      // differences k = i + 2 by the thread of interface i, the four outer ones (k = 0, 1,
      // Tc + 3, Tc + 4) by the next four threads, none of them the speed warp (static_assert
      // below)
      const int k = tid < ni ? tid + 2 : (tid < ni + 2 ? tid - ni : Tc + 3 + (tid - ni - 2));
      if (tid < ni + 4) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sm[TL::kDf + c * W + k] = s_f[c * W + k + 1] - s_f[c * W + k];
          sm[TL::kDu + c * W + k] = s_uin[c * W + off + k + 1] - s_uin[c * W + off + k];
        }
      }
    }
    c0_barrier();
  }
  static_assert(!DP || MODE == kStage || NI + 4 <= NT - (MODE == kStepBlocked ? 32 : 0),
                "outer differences fit the C0 threads");
  // DP: the differences of f and u between neighbouring window cells (f's over the per-cell
  // Roe inputs, read for the last time in phase C0), by the threads of phase C0
  double* s_df = sm + TL::kDf;
  double* s_du = sm + TL::kDu;
  if constexpr (DP && MODE == kStage) {
    if (!(sw_free && (tid >> 5) == kSW)) {
      const int np = sw_free ? NT - 32 : NT;
      for (int k = tid; k < cells - 1; k += np) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s_df[c * W + k] = s_f[c * W + k + 1] - s_f[c * W + k];
          s_du[c * W + k] = s_uin[c * W + off + k + 1] - s_uin[c * W + off + k];
        }
      }
    }
    c0_barrier();
  }

  // ---- C1: per (interface, field) reconstruction on both sides.  The projections onto the
  // characteristic field split into the alpha-free products (l.f, l.u), taken first, and the
  // Lax-Friedrichs combination.  A side whose stencil is not restricted (Eq. (be_res)) queues
  // its weight evaluation, which a second pass spreads over full warps instead of diverging
  // inside the first.  SPLIT = 2: the threads 2k (+ side) and 2k + 1 (- side) share item k;
  // each takes the products of three of the six stencil cells and the two swap them by a
  // shuffle, so each thread runs half the chain of the SPLIT = 1 item with the same operations.
  int* s_qn = reinterpret_cast<int*>(sm + TL::kQn);
  double* s_q = sm + TL::kQ;
  int* s_qi = reinterpret_cast<int*>(sm + TL::kQi);
  constexpr int QCAP = TL::QCAP;
  const int it = (SPLIT == 2) ? (tid >> 1) : tid;
  const int side2 = (SPLIT == 2) ? (tid & 1) : 0;
  const bool has_item = it < M * ni;
  const int s = has_item ? it / ni : 0;
  const int i = it - s * ni;
  // pa, pb: (l.f, l.u) of the stencil cells i .. i + 5 (window index), in the order of the
  // side's stencil with SPLIT = 2 (the - side reads the cells mirrored, Eq. (flux_split_lf))
  double pa[6], pb[6];
  // DP: (da_k, db_k) the products of the stencil's cell differences, (a2, b2) and (a3, b3) those
  // of its two centre cells (MATH::side_diffs); with SPLIT = 2 the + thread takes the centre
  // cell 2 and differences 0, 1, the - thread cell 3 and differences 4, 3, and the pair swaps them
  double da[5], db[5], a2 = 0.0, b2 = 0.0, a3 = 0.0, b3 = 0.0;
  auto proj_cell = [&](const double* l, const int k, double& x, double& y) {
    double f[3] = {s_f[k], s_f[W + k], s_f[2 * W + k]};
    double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
    MATH::project3_ab(l, f, U, x, y);
  };
  auto proj_diff = [&](const double* l, const int k, double& x, double& y) {
    double f[3] = {s_df[k], s_df[W + k], s_df[2 * W + k]};
    double U[3] = {s_du[k], s_du[W + k], s_du[2 * W + k]};
    MATH::project3_ab(l, f, U, x, y);
  };
  if constexpr (DP && SPLIT == 2) {
    double o[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (has_item) {
      double l[3] = {s_L[(3 * s) * NI + i], s_L[(3 * s + 1) * NI + i], s_L[(3 * s + 2) * NI + i]};
      proj_cell(l, i + 2 + side2, o[0], o[1]);
      proj_diff(l, side2 ? i + 4 : i, o[2], o[3]);
      proj_diff(l, side2 ? i + 3 : i + 1, o[4], o[5]);
    }
    if ((tid >> 5) * 32 < SPLIT * M * ni) {
      double p[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) p[r] = __shfl_xor_sync(0xffffffffu, o[r], 1);
      // the side's stencil order: its own products are differences 0, 1 (+ side) or 4, 3
      // (- side, mirrored), its partner's the other two in reverse, and difference 2 is
      // a3 - a2 on both sides (the partner's centre minus its own, negated on the - side)
      const unsigned long long sg = side2 ? 0x8000000000000000ull : 0ull;
      da[0] = o[2];
      db[0] = o[3];
      da[1] = o[4];
      db[1] = o[5];
      da[4] = p[2];
      db[4] = p[3];
      da[3] = p[4];
      db[3] = p[5];
      da[2] = flip_sign(p[0] - o[0], sg);
      db[2] = flip_sign(p[1] - o[1], sg);
      a2 = o[0];  // the own centre cell's products
      b2 = o[1];
    }
  } else if constexpr (DP) {
    if (has_item && IPT == 1) {
      double l[3] = {s_L[(3 * s) * NI + i], s_L[(3 * s + 1) * NI + i], s_L[(3 * s + 2) * NI + i]};
      proj_cell(l, i + 2, a2, b2);
      proj_cell(l, i + 3, a3, b3);
      proj_diff(l, i, da[0], db[0]);
      proj_diff(l, i + 1, da[1], db[1]);
      proj_diff(l, i + 3, da[3], db[3]);
      proj_diff(l, i + 4, da[4], db[4]);
      da[2] = a3 - a2;
      db[2] = b3 - b2;
    }
  } else if constexpr (SPLIT == 2) {
    double oa[3] = {0.0, 0.0, 0.0}, ob[3] = {0.0, 0.0, 0.0};
    if (has_item) {
      if (FLUX == WT_FLUX_EULER1D) {
        double l[3] = {s_L[(3 * s) * NI + i], s_L[(3 * s + 1) * NI + i], s_L[(3 * s + 2) * NI + i]};
#pragma unroll
        for (int h = 0; h < 3; ++h) {
          const int k = i + (side2 ? 5 - h : h);
          double f[3] = {s_f[k], s_f[W + k], s_f[2 * W + k]};
          double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
          MATH::project3_ab(l, f, U, oa[h], ob[h]);
        }
      } else {
#pragma unroll
        for (int h = 0; h < 3; ++h) {
          const int k = i + (side2 ? 5 - h : h);
          MATH::project1_ab(s_f[k], s_uin[off + k], oa[h], ob[h]);
        }
      }
    }
    // own cells take stencil places 0..2; the partner's, mirrored, places 5..3 (every warp
    // with items takes part as a whole)
    if ((tid >> 5) * 32 < SPLIT * M * ni) {
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        pa[h] = oa[h];
        pb[h] = ob[h];
        pa[5 - h] = __shfl_xor_sync(0xffffffffu, oa[h], 1);
        pb[5 - h] = __shfl_xor_sync(0xffffffffu, ob[h], 1);
      }
    }
  } else if (has_item && IPT == 1) {
    if (FLUX == WT_FLUX_EULER1D) {
      double l[3] = {s_L[(3 * s) * NI + i], s_L[(3 * s + 1) * NI + i], s_L[(3 * s + 2) * NI + i]};
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) {
        const int k = i + kk;
        double f[3] = {s_f[k], s_f[W + k], s_f[2 * W + k]};
        double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
        MATH::project3_ab(l, f, U, pa[kk], pb[kk]);
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) MATH::project1_ab(s_f[i + kk], s_uin[off + i + kk], pa[kk], pb[kk]);
    }
  }
  if (MODE == kStepBlocked) {
    // the speed warp holds the alphas of every CTA: it finished before the end of phase C0,
    // or joins the others here
    if (sw_free) __syncthreads();
    if (*s_aflag != 1) return false;
#pragma unroll
    for (int f = 0; f < M; ++f) alpha[f] = bits_to_double(s_alpha[f]);
    if (aw.first_stage) {
      const double smax = (FLUX == WT_FLUX_EULER1D) ? ((alpha[0] < alpha[M - 1]) ? alpha[M - 1] : alpha[0]) : alpha[0];
      dt = aw.dt_fixed > 0.0 ? aw.dt_fixed : MATH::cfl_dt(aw.cfl, a.dx, smax);
      const double rem = aw.t_final - aw.t;
      if (rem < dt) dt = rem;
      if (aw.clear >= 0 && tid == 0) ctl->dt = dt;
    }
  }
  // REC (the adjoint's recording forward pass): each reconstruction's branch flags, bit 0 restricted
  // (Eq. (be_res)), bit 1 theta = 1 (Eq. (tau_we6)), kept in the reduction buffer until the
  // records are written (phase E reuses it afterwards)
  unsigned char* s_fl = reinterpret_cast<unsigned char*>(s_red);
  static_assert(!REC || (2 * M * NI <= 4 * 32 * 8 && MODE == kStage), "flags fit the reduction buffer");
  // one reconstruction (stencil q) into s_F[dst], or into the queue
  auto reconstruct = [&](const double* q, const int dst) {
    if constexpr (MATH::kSplitWeno && MODE == kStepBlocked) {
      // a stencil the FP32 screen does not settle is deferred whole to the quad pass, so the
      // long FP64 path never diverges inside the warps of this pass
      double rec[TL::REC];
      double out;
      if (MATH::weno_front(q, a.eps, a.alpha_R, out, rec)) {
        s_F[dst] = out;
      } else {
        const int slot = atomicAdd(s_qn, 1);
        if (slot < QCAP) {
#pragma unroll
          for (int r = 0; r < TL::REC; ++r) s_q[r * QCAP + slot] = rec[r];
          s_qi[slot] = dst;
        } else {
          s_F[dst] = MATH::weno(q, a.eps, a.alpha_R);
        }
      }
    } else if constexpr (MATH::kSplitWeno) {
      typename MATH::WenoPart w;
      double out;
      if (MATH::weno_begin(q, a.eps, a.alpha_R, out, w)) {
        s_F[dst] = out;
        if constexpr (REC) s_fl[dst] = (unsigned char)(1 | (w.theta1 ? 2 : 0));
      } else {
        if constexpr (REC) s_fl[dst] = (unsigned char)(w.theta1 ? 2 : 0);
        const int slot = atomicAdd(s_qn, 1);
        if (slot < QCAP) {
#pragma unroll
          for (int k = 0; k < 4; ++k) s_q[k * QCAP + slot] = w.e[k];
          s_q[4 * QCAP + slot] = w.tau;
#pragma unroll
          for (int k = 0; k < 4; ++k) s_q[(5 + k) * QCAP + slot] = w.fh[k];
          s_qi[slot] = dst | (w.theta1 ? (1 << 30) : 0);
        } else {
          s_F[dst] = MATH::weno_finish(w);
        }
      }
    } else if constexpr (REC) {
      bool r, t;
      s_F[dst] = MATH::weno_flags(q, a.eps, a.alpha_R, r, t);
      s_fl[dst] = (unsigned char)((r ? 1 : 0) | (t ? 2 : 0));
    } else {
      s_F[dst] = MATH::weno(q, a.eps, a.alpha_R);
    }
  };
  if constexpr (DP) {
    // differences first: the reconstructions from their stencils' differences and q_2
    // (step-blocked: sg negates the result of a - side thread, which reconstructs its stencil
    // negated; its queue record carries bit 30)
    auto reconstruct_d = [&](const double* d, const double q2, const int dst, const unsigned long long sg = 0ull) {
      double out;
      if constexpr (MODE == kStepBlocked) {
        double rec[TL::REC];
        if (MATH::weno_front_d(d, q2, a.eps, a.alpha_R, out, rec)) {
          s_F[dst] = flip_sign(out, sg);
        } else {
          const int slot = atomicAdd(s_qn, 1);
          if (slot < QCAP) {
#pragma unroll
            for (int r = 0; r < TL::REC; ++r) s_q[r * QCAP + slot] = rec[r];
            s_qi[slot] = dst | (sg ? (1 << 30) : 0);
          } else {
            s_F[dst] = flip_sign(MATH::weno_d(d, q2, a.eps, a.alpha_R), sg);
          }
        }
      } else {
        typename MATH::WenoPart w;
        if (MATH::weno_begin_d(d, q2, a.eps, a.alpha_R, out, w)) {
          s_F[dst] = out;
          if constexpr (REC) s_fl[dst] = (unsigned char)(1 | (w.theta1 ? 2 : 0));
        } else {
          if constexpr (REC) s_fl[dst] = (unsigned char)(w.theta1 ? 2 : 0);
          const int slot = atomicAdd(s_qn, 1);
          if (slot < QCAP) {
#pragma unroll
            for (int k = 0; k < 4; ++k) s_q[k * QCAP + slot] = w.e[k];
            s_q[4 * QCAP + slot] = w.tau;
#pragma unroll
            for (int k = 0; k < 4; ++k) s_q[(5 + k) * QCAP + slot] = w.fh[k];
            s_qi[slot] = dst | (w.theta1 ? (1 << 30) : 0);
          } else {
            s_F[dst] = MATH::weno_finish(w);
          }
        }
      }
    };
    if constexpr (IPT > 1) {
      for (int it2 = tid; it2 < M * ni; it2 += NT) {
        const int s2 = it2 / ni, i2 = it2 - s2 * ni;
        double l[3] = {s_L[(3 * s2) * NI + i2], s_L[(3 * s2 + 1) * NI + i2], s_L[(3 * s2 + 2) * NI + i2]};
        double ea[5], eb[5], c2a, c2b, c3a, c3b;
        proj_cell(l, i2 + 2, c2a, c2b);
        proj_cell(l, i2 + 3, c3a, c3b);
        proj_diff(l, i2, ea[0], eb[0]);
        proj_diff(l, i2 + 1, ea[1], eb[1]);
        proj_diff(l, i2 + 3, ea[3], eb[3]);
        proj_diff(l, i2 + 4, ea[4], eb[4]);
        ea[2] = c3a - c2a;
        eb[2] = c3b - c2b;
        const double al = (s2 == 0) ? alpha[0] : ((s2 == 1) ? alpha[1] : alpha[M - 1]);
        double d[5], q2;
        MATH::side_diffs(ea, eb, c2a, c2b, c3a, c3b, al, false, d, q2);
        reconstruct_d(d, q2, s2 * NI + i2);
        MATH::side_diffs(ea, eb, c2a, c2b, c3a, c3b, al, true, d, q2);
        reconstruct_d(d, q2, M * NI + s2 * NI + i2);
      }
    } else if (has_item) {
      const double al = (s == 0) ? alpha[0] : ((s == 1) ? alpha[1] : alpha[M - 1]);
      double d[5], q2;
      if constexpr (SPLIT == 2) {
        // The - side reconstructs its stencil negated: the reconstruction is odd in its data bit
        // for bit (squares and comparisons do not see the sign; every other step is a rounded
        // linear operation, and round-to-nearest is symmetric), so -weno(-d, -q2) is the value
        // of MATH::side_diffs' stencil.  Its differences are then alpha-combined like the + side's,
        // with -alpha, from the side-ordered products, and no selects are needed.
        const unsigned long long sg = side2 ? 0x8000000000000000ull : 0ull;
        const double sa = flip_sign(al, sg);
#pragma unroll
        for (int k = 0; k < 5; ++k) d[k] = fma(sa, db[k], da[k]);
        q2 = fma(al, b2, flip_sign(a2, sg));  // + side: a2 + alpha b2; - side: alpha b3 - a3
        reconstruct_d(d, q2, side2 * (M * NI) + s * NI + i, sg);
      } else {
        MATH::side_diffs(da, db, a2, b2, a3, b3, al, false, d, q2);
        reconstruct_d(d, q2, s * NI + i);
        MATH::side_diffs(da, db, a2, b2, a3, b3, al, true, d, q2);
        reconstruct_d(d, q2, M * NI + s * NI + i);
      }
    }
  } else if constexpr (IPT > 1) {
    // several items per thread: projection and both reconstructions of each item in turn, with
    // the operations of the one-item path
    for (int it2 = tid; it2 < M * ni; it2 += NT) {
      const int s2 = it2 / ni, i2 = it2 - s2 * ni;
      double qa[6], qb[6];
      if (FLUX == WT_FLUX_EULER1D) {
        double l[3] = {s_L[(3 * s2) * NI + i2], s_L[(3 * s2 + 1) * NI + i2], s_L[(3 * s2 + 2) * NI + i2]};
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) {
          const int k = i2 + kk;
          double f[3] = {s_f[k], s_f[W + k], s_f[2 * W + k]};
          double U[3] = {s_uin[off + k], s_uin[W + off + k], s_uin[2 * W + off + k]};
          MATH::project3_ab(l, f, U, qa[kk], qb[kk]);
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) MATH::project1_ab(s_f[i2 + kk], s_uin[off + i2 + kk], qa[kk], qb[kk]);
      }
      const double al = (s2 == 0) ? alpha[0] : ((s2 == 1) ? alpha[1] : alpha[M - 1]);
      double vp[6], vm[6];
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) MATH::project_v(qa[kk], qb[kk], al, vp[kk], vm[kk]);
      double qm[6];
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) qm[kk] = vm[5 - kk];
      reconstruct(vp, s2 * NI + i2);
      reconstruct(qm, M * NI + s2 * NI + i2);
    }
  } else if (has_item) {
    const double al = (s == 0) ? alpha[0] : ((s == 1) ? alpha[1] : alpha[M - 1]);
    if constexpr (SPLIT == 2) {
      double q[6];
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) q[kk] = MATH::project_side(pa[kk], pb[kk], al, side2 != 0);
      reconstruct(q, side2 * (M * NI) + s * NI + i);
    } else {
      double vp[6], vm[6];
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) MATH::project_v(pa[kk], pb[kk], al, vp[kk], vm[kk]);
      double qm[6];
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) qm[kk] = vm[5 - kk];
      reconstruct(vp, s * NI + i);
      reconstruct(qm, M * NI + s * NI + i);
    }
  }
  __syncthreads();
  // LATE: phase C1 no longer reads the eigenvectors, so the window of u^n (stages 2, 3) is copied
  // into their buffer now; it lands while the queued weights and phase D run
  [[maybe_unused]] uint64_t* s_bar = reinterpret_cast<uint64_t*>(sm + TL::kBar);
  if constexpr (LATE && kNeedUn) {
    if (tid == 0) {
      const uint32_t late_bytes = (uint32_t)(((off + Tc + 2 * G + 1) & ~1) * 8);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the generic reads of the buffer
      mbar_arrive_expect_tx(s_bar, late_bytes * M);
      const long long s0 = js & ~1LL;
#pragma unroll
      for (int c = 0; c < M; ++c) bulk_g2s(s_un + c * W, a.un + c * a.pitch + s0, late_bytes, s_bar);
    }
  }
  if constexpr (MATH::kSplitWeno) {
    const int nq = min(*s_qn, QCAP);  // the same for every thread of the block
    if (nq > 0 && MODE == kStepBlocked) {
      // a quad of lanes per deferred stencil (FastMath::weno_back_quad): lane k forms
      // indicator k and weight k, the quad shares them by shuffles, and its lane 0 holds the
      // result.  The tiles holding a shock carry the queue, and every CTA waits for them at
      // the next alpha exchange.
      for (int base = 0; base < nq; base += NT / 4) {
        const int t = base + (tid >> 2), k = tid & 3;
        if (t < nq) {  // the same for the four lanes of a quad
          double rec[TL::REC];
#pragma unroll
          for (int r = 0; r < TL::REC; ++r) rec[r] = s_q[r * QCAP + t];
          const unsigned qmask = 0xfu << (tid & 28);
          const double out = MATH::weno_back_quad(k, rec, a.eps, a.alpha_R, qmask);
          const int qi = s_qi[t];  // bit 30: a negated - side stencil
          if (k == 0) s_F[qi & ((1 << 30) - 1)] = flip_sign(out, (qi >> 30) & 1 ? 0x8000000000000000ull : 0ull);
        }
      }
      __syncthreads();
    } else if (nq > 0) {
      for (int t = tid; t < nq; t += NT) {
        typename MATH::WenoPart w;
#pragma unroll
        for (int k = 0; k < 4; ++k) w.e[k] = s_q[k * QCAP + t];
        w.tau = s_q[4 * QCAP + t];
#pragma unroll
        for (int k = 0; k < 4; ++k) w.fh[k] = s_q[(5 + k) * QCAP + t];
        const int d = s_qi[t];
        w.theta1 = (d >> 30) & 1;
        s_F[d & ((1 << 30) - 1)] = MATH::weno_finish(w);
      }
      __syncthreads();
    }
  }

  // REC: the records of the tile's interfaces (slot js + i for interface js - 1 + i; a tile
  // shares its first interface with its left neighbour, which writes the same values)
  if constexpr (REC) {
    for (int i = tid; i < ni; i += NT) {
      double* r = a.rec + (size_t)(js + i) * kAdjRec;
      unsigned long long fl = 0ull;
#pragma unroll
      for (int side = 0; side < 2; ++side)
#pragma unroll
        for (int f = 0; f < 3; ++f)
          fl |= (unsigned long long)s_fl[side * (M * NI) + f * NI + i] << (2 * (3 * side + f));
      r[0] = s_rs[i];
      r[1] = s_rs[NI + i];
      r[2] = s_F[i] + s_F[3 * NI + i];
      r[3] = s_F[NI + i] + s_F[4 * NI + i];
      r[4] = s_F[2 * NI + i] + s_F[5 * NI + i];
      r[5] = __longlong_as_double((long long)fl);
    }
    __syncthreads();  // the flags' buffer is the reduction buffer of phase E
  }

  // ---- D: interface fluxes h_{j+1/2} = R (F+ + F-)
  const double* hsrc = s_F;
  if (FLUX == WT_FLUX_EULER1D) {
    for (int i = tid; i < ni; i += NT) {
      double rs[3] = {s_rs[i], s_rs[NI + i], s_rs[2 * NI + i]};
      double F[3] = {s_F[i] + s_F[3 * NI + i], s_F[NI + i] + s_F[4 * NI + i], s_F[2 * NI + i] + s_F[5 * NI + i]};
      double h[3];
      MATH::backproject(rs, F, h);
#pragma unroll
      for (int c = 0; c < 3; ++c) s_h[c * NI + i] = h[c];
    }
    __syncthreads();
    hsrc = s_h;
  }

  // LATE: the window of u^n has landed before phase E reads it (bounded wait)
  if constexpr (LATE && kNeedUn) {
    const bool ok = mbar_wait_bounded(s_bar, *phase);
    if (__syncthreads_or(ok ? 0 : 1)) {
      if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
      mbar_wait_bounded(s_bar, *phase);
      return false;
    }
    *phase ^= 1u;
  }
  // ---- E: flux difference, RK combine, ghost images, wave speeds.  Step-blocked: one
  // (cell, component) per thread, and no wave speeds (phase B of the next stage takes them).
  if (MODE == kStepBlocked && STAGE != STAGE_RHS) {
    for (int idx = tid; idx < M * Tc; idx += NT) {
      const int c = idx / Tc, t = idx - c * Tc;
      const long long j = js + t;
      const double hp = (FLUX == WT_FLUX_EULER1D) ? hsrc[c * NI + t + 1] : hsrc[t + 1] + hsrc[NI + t + 1];
      const double hm = (FLUX == WT_FLUX_EULER1D) ? hsrc[c * NI + t] : hsrc[t] + hsrc[NI + t];
      const double L = MATH::flux_diff(hp, hm, a.dx, a.inv_dx);
      const double us = s_uin[c * W + off + t + G];
      const double un = kNeedUn ? s_un[c * W + off + t + G] : us;
      const double v = MATH::template rk<(STAGE == STAGE_RHS ? 0 : STAGE)>(un, us, dt, L);
      s_uin[c * W + off + t + G] = v;
      if (STAGE == STAGE_RK3) {
        s_un[c * W + off + t + G] = v;
        if (j >= own_lo && j < own_hi) {
          if (!isfinite(v)) flag_error(ctl, WT_ERR_NONPHYSICAL);
          double* o = a.uout + c * a.pitch;
          o[j + G] = v;
          // the halo mailbox: u^{n+1} for the neighbours' next step, two tagged words
          {
            const unsigned long long b = (unsigned long long)__double_as_longlong(v);
            const unsigned long long tg = (unsigned long long)aw.tag << 32;
            st_relaxed_u64(aw.hmb_hi + c * a.pitch + j, tg | (b >> 32));
            st_relaxed_u64(aw.hmb_lo + c * a.pitch + j, tg | (b & 0xffffffffull));
          }
          // ghost images of this cell in the output
          if (j < G || j >= n - G) {
            const double vr = (c == 1) ? -v : v;
            if (a.bc_hi == WT_BC_PERIODIC && j < G) o[n + j + G] = v;
            if (a.bc_lo == WT_BC_PERIODIC && j >= n - G) o[j - n + G] = v;
            if (a.bc_lo == WT_BC_OUTFLOW && j == 0) o[0] = o[1] = o[2] = v;
            if (a.bc_hi == WT_BC_OUTFLOW && j == n - 1) o[n + 3] = o[n + 4] = o[n + 5] = v;
            if (a.bc_lo == WT_BC_REFLECTIVE && j < G) o[2 - j] = vr;
            if (a.bc_hi == WT_BC_REFLECTIVE && j >= n - G) o[2 * n + 2 - j] = vr;
          }
        }
      }
    }
    __syncthreads();
    return true;
  }
  unsigned long long vmax[M];
#pragma unroll
  for (int f = 0; f < M; ++f) vmax[f] = 0ull;
  // Euler stage tiles (throughput-bound): the wave speeds of the stage output are screened in FP32
  // (euler_speeds_screen) and kept in the dead buffer of the reconstructions (s_lam, +inf
  // where the screen does not apply); the FP64 speeds are then taken only for the cells that
  // can hold a maximum of the tile (below)
  constexpr bool kScreen = FLUX == WT_FLUX_EULER1D && MODE == kStage && STAGE != STAGE_RHS;
  float* s_lam = reinterpret_cast<float*>(s_F);
  float m32[3] = {0.0f, 0.0f, 0.0f};
  const float g32 = f32_hi(a.gamma * (a.gamma - 1.0));
  for (int t = tid; t < Tc; t += NT) {
    const long long j = js + t;
    const bool own = (MODE != kStepBlocked) || (j >= own_lo && j < own_hi);
    double uo[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      // scalar fluxes: h = F+ + F- directly from the reconstruction
      const double hp = (FLUX == WT_FLUX_EULER1D) ? hsrc[c * NI + t + 1] : hsrc[t + 1] + hsrc[NI + t + 1];
      const double hm = (FLUX == WT_FLUX_EULER1D) ? hsrc[c * NI + t] : hsrc[t] + hsrc[NI + t];
      const double L = MATH::flux_diff(hp, hm, a.dx, a.inv_dx);
      if (STAGE == STAGE_RHS) {
        a.Lout[c * a.lout_stride + j] = L;
      } else {
        const double us = s_uin[c * W + off + t + G];
        const double un = kNeedUn ? s_un[c * W + off + t + G] : us;
        uo[c] = MATH::template rk<(STAGE == STAGE_RHS ? 0 : STAGE)>(un, us, dt, L);
      }
    }
    if (STAGE != STAGE_RHS) {
      if (MODE != kStage) {
#pragma unroll
        for (int c = 0; c < M; ++c) {
          s_uin[c * W + off + t + G] = uo[c];
          if (STAGE == STAGE_RK3) s_un[c * W + off + t + G] = uo[c];
        }
      }
      if (own && (MODE != kStepBlocked || STAGE == STAGE_RK3)) {
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
      }
      if (own && MODE == kStepBlocked) {
        if (FLUX == WT_FLUX_EULER1D ? !finite3(uo) : !isfinite(uo[0])) flag_error(ctl, WT_ERR_NONPHYSICAL);
      } else if (own) {
        if constexpr (kScreen) {
          if (!finite3(uo)) flag_error(ctl, WT_ERR_NONPHYSICAL);
          float l32[3];
          const bool ok = euler_speeds_screen(uo, g32, l32);
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            s_lam[f * NI + t] = ok ? l32[f] : INFINITY;
            if (ok) m32[f] = fmaxf(m32[f], l32[f]);
          }
          // the FP64 pass reads the output back
#pragma unroll
          for (int c = 0; c < M; ++c) s_uin[c * W + off + t + G] = uo[c];
        } else if (FLUX == WT_FLUX_EULER1D) {
          double lam[3];
          MATH::euler_speeds(uo, a.gamma, lam);
          if (!finite3(uo)) flag_error(ctl, WT_ERR_NONPHYSICAL);
#pragma unroll
          for (int f = 0; f < M; ++f) key_max(vmax[f], lam[f]);
        } else {
          const double lam = (FLUX == WT_FLUX_ADVECTION) ? fabs(a.adv_speed) : fabs(uo[0]);
          if (!isfinite(uo[0])) flag_error(ctl, WT_ERR_NONPHYSICAL);
          key_max(vmax[0], lam);
        }
      }
    }
  }
  if constexpr (kScreen) {
    // The tile's FP32 maxima m_s.  With e = 2^-14.6 max(m_0, m_2) bounding every cell's error
    // in lam_0, lam_2 (|u| + c <= max(lam_0, lam_2) + its error), a cell holding the FP64
    // maximum of field 0 or 2 has lam_s >= m_s - 2 e; for field 1 (no cancellation, error
    // 2.3 * 2^-20 relative) lam_1 >= m_1 (1 - 2^-17.8), and where m_1 = 0 every screened cell
    // has m = 0, |u| = 0 exactly.  Margins 2^-12 and 2^-16 are taken.  A candidate for field 1
    // only takes |u| (MATH::speed_u), one for field 0 or 2 the sound speed as well; a cell whose
    // state equals its left neighbour's bit for bit has the same speeds and is skipped (a run
    // of equal states is decided by its first cell, which has the same screen values).
    float* s_lm = s_lam + 3 * NI;  // [3][32] warp maxima
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      float v = m32[f];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) s_lm[f * 32 + warp] = v;
    }
    __syncthreads();
    float tm[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int f = 0; f < 3; ++f)
      for (int w = 0; w < NT / 32; ++w) tm[f] = fmaxf(tm[f], s_lm[f * 32 + w]);
    const float smx = fmaxf(tm[0], tm[2]);
    const float thr0 = tm[0] - 0x1p-12f * smx, thr2 = tm[2] - 0x1p-12f * smx;
    const float thr1 = tm[1] * (1.0f - 0x1p-16f);
    for (int t = tid; t < Tc; t += NT) {
      const float l0 = s_lam[t], l1 = s_lam[NI + t], l2 = s_lam[2 * NI + t];
      const bool c02 = l0 >= thr0 || l2 >= thr2;
      if (c02 || (l1 > 0.0f && l1 >= thr1)) {
        const int k = off + t + G;
        double U[3] = {s_uin[k], s_uin[W + k], s_uin[2 * W + k]};
        bool dup = t > 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          dup = dup && __double_as_longlong(U[c]) == __double_as_longlong(s_uin[c * W + k - 1]);
        if (!dup) {
          double u, ir;
          key_max(vmax[1], MATH::speed_u(U, u, ir));
          if (c02) {
            double a0, a2;
            MATH::speed_c(U, a.gamma, u, ir, a0, a2);
            key_max(vmax[0], a0);
            key_max(vmax[2], a2);
          }
        }
      }
    }
  }
  if (MODE == kStepBlocked) {
    __syncthreads();
  } else if (STAGE != STAGE_RHS) {
    block_max_atomic<M>(vmax, s_red, ctl->amax[(STAGE + 1) % 3]);
  }
  return true;
}

template <class MATH, int FLUX, int STAGE, int T, int IPT = 1, bool REC = false>
__device__ __forceinline__ bool stage1d_tile(const Stage1DArgs& a, const long long j0, const bool first_tile, double* sm,
                                             uint32_t& phase) {
  constexpr int M = FluxM<FLUX>::m;
  using TL = TileOf<MATH, FLUX, T, 1, IPT, true>;
  constexpr int W = TL::W;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TL::kBar);
  double* s_uin = sm + TL::kUin;
  int* s_run = reinterpret_cast<int*>(sm + TL::kQn) + 1;
  const int tid = threadIdx.x;
  Ctl* ctl = a.ctl;
  const long long n = a.n;
  if (j0 >= n) return true;
  const int Tc = (int)((n - j0 < T) ? (n - j0) : T);

  // ---- A: stage the window [j0 - 3, j0 + Tc + 3) of every plane (16-byte aligned start).
  // The copies are issued first and overlap the reads of the control block below.
  const long long s0 = j0 & ~1LL;
  const int off = (int)(j0 - s0);
  const int cells = Tc + 2 * G;
  const int len = (off + cells + 1) & ~1;
  constexpr bool kNeedUn = (STAGE == STAGE_RK2 || STAGE == STAGE_RK3);
  // (u^n of stages 2 and 3 is copied later, into the eigenvector buffer: Tile1D LATE)
  if (tid == 0) {
    const uint32_t bytes = (uint32_t)len * 8u;
    mbar_arrive_expect_tx(bar, bytes * M);
#pragma unroll
    for (int c = 0; c < M; ++c) bulk_g2s(s_uin + c * W, a.uin + c * a.pitch + s0, bytes, bar);
  }

  // ---- step control: is this step active (decided by thread 0 for the whole block), its dt
  if (tid == 0) {
    int run = 1;
    if (STAGE == STAGE_RK1) run = (ctl->status == 0) && (ctl->t < ctl->t_final);
    if (STAGE == STAGE_RK2 || STAGE == STAGE_RK3) run = ctl->active != 0;
    if (STAGE == STAGE_RK1 && !run && first_tile) ctl->active = 0;
    *s_run = run;
  }
  double dt = 0.0;
  double alpha[M];
  const int slot_in = (STAGE == STAGE_RHS) ? 0 : STAGE;
#pragma unroll
  for (int s = 0; s < M; ++s) alpha[s] = bits_to_double(ctl->amax[slot_in][s]);
  if (STAGE == STAGE_RK1) {
    const double smax = (FLUX == WT_FLUX_EULER1D) ? ((alpha[0] < alpha[M - 1]) ? alpha[M - 1] : alpha[0]) : alpha[0];
    dt = ctl->dt_fixed > 0.0 ? ctl->dt_fixed : MATH::cfl_dt(ctl->cfl, a.dx, smax);
    const double rem = ctl->t_final - ctl->t;
    if (rem < dt) dt = rem;
  } else if (STAGE != STAGE_RHS) {
    dt = ctl->dt;
  }

  // every copy completes before the block moves on (or leaves)
  const bool ok = mbar_wait_bounded(bar, phase);
  if (__syncthreads_or(ok ? 0 : 1)) {
    if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
    mbar_wait_bounded(bar, phase);
    return false;
  }
  phase ^= 1u;
  if (!*s_run) return true;
  if (STAGE != STAGE_RHS && first_tile && tid < 8) ctl->amax[(STAGE + 2) % 3][tid] = 0ull;
  if (STAGE == STAGE_RK1 && first_tile && tid == 0) {
    ctl->dt = dt;
    ctl->active = 1;
  }

  if (!stage1d_compute<MATH, FLUX, STAGE, T, kStage, IPT, REC>(a, j0, Tc, off, j0, j0 + Tc, alpha, dt, sm,
                                                              AlphaWait{0ull, 0, -1, 0, 0.0, 0.0, 0.0, 0.0}, &phase))
    return false;
  if (STAGE != STAGE_RHS) {
    if (STAGE == STAGE_RK3 && first_tile && tid == 0) {
      ctl->t = ctl->t + dt;
      ctl->steps = ctl->steps + 1;
    }
  }
  return true;
}

template <class MATH, int FLUX, int STAGE, int T>
__global__ void __launch_bounds__(Tile1D<T, FluxM<FLUX>::m, 1, 1, true>::NT) stage1d_kernel(const Stage1DArgs a) {
  using TL = TileOf<MATH, FLUX, T, 1, 1, true>;
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
template <class MATH, int FLUX, int STAGE, int T, int IPT, bool REC = false>
__global__ void __launch_bounds__(Tile1D<T, FluxM<FLUX>::m, 1, IPT, true>::NT) stage1d_batched_kernel(const BatchArgs b) {
  using TL = TileOf<MATH, FLUX, T, 1, IPT, true>;
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
    a.rec = REC ? b.rec + (size_t)b.rec_off[item.x] * kAdjRec : nullptr;
    const long long j0 = (long long)item.y * T;
    if (!stage1d_tile<MATH, FLUX, STAGE, T, IPT, REC>(a, j0, j0 == 0, sm, phase)) return;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Persistent RK3 integration of one problem: a cooperative grid with one CTA per tile runs
// p.n_steps steps (fewer once t_final is reached or a failure was flagged), three stages per
// step, with a grid barrier after each stage instead of a kernel boundary.  Each CTA keeps
// its tile resident in shared memory: its own cells of the stage input and of u^n stay
// there from stage to stage, and only the three halo cells on each side are read back from
// the neighbours' stage outputs.  Every stage writes its output and ghost images to global
// memory as in the stage kernels, so the buffers hold the same values on exit.  dt and t
// are computed by every CTA from the same alphas, so all CTAs take the same decisions; the
// stop decision of a step is the OR of one vote per CTA (status seen before the step's last
// barrier), read after that barrier.
// ---------------------------------------------------------------------------------------
template <class MATH, int FLUX, int T>
__device__ __forceinline__ void load_halos(const double* uin, long long pitch, long long j0, int Tc, double* s_uin) {
  constexpr int M = FluxM<FLUX>::m;
  constexpr int W = Tile1D<T, M>::W;
  const int tid = threadIdx.x;
  if (tid < 2 * G * M) {
    const int c = tid / (2 * G), h = tid - c * (2 * G);
    const int k = (h < G) ? h : Tc + h;  // window index: 0..2 and Tc+3..Tc+5
    s_uin[c * W + k] = __ldcg(uin + c * pitch + j0 + k);
  }
  __syncthreads();
}

template <class MATH, int FLUX, int T>
__global__ void __launch_bounds__(Tile1D<T, FluxM<FLUX>::m>::NT, 3) persist1d_kernel(const PersistArgs p) {
  constexpr int M = FluxM<FLUX>::m;
  using TL = TileOf<MATH, FLUX, T>;
  constexpr int W = TL::W, NT = TL::NT;
  extern __shared__ __align__(16) double sm[];
  double* s_uin = sm + TL::kUin;
  double* s_un = sm + TL::kUn;
  const int tid = threadIdx.x;
  Ctl* ctl = p.a[0].ctl;
  const long long n = p.a[0].n, pitch = p.a[0].pitch;
  const long long j0 = (long long)blockIdx.x * T;
  const int Tc = (int)((n - j0 < T) ? (n - j0) : T);
  const int cells = Tc + 2 * G;
  const bool first = blockIdx.x == 0;
  unsigned long long nbar = 0;
  const unsigned long long nblk = gridDim.x;

  // window of u^n: stage input and u^n
  for (int idx = tid; idx < M * cells; idx += NT) {
    const int c = idx / cells, k = idx - c * cells;
    const double v = __ldcg(p.a[0].uin + c * pitch + j0 + k);
    s_uin[c * W + k] = v;
    s_un[c * W + k] = v;
  }
  const double t_final = __ldcg(&ctl->t_final), cfl = __ldcg(&ctl->cfl), dt_fixed = __ldcg(&ctl->dt_fixed);
  double t = __ldcg(&ctl->t);
  // status as it stands before any block of this launch can flag a failure
  bool stop = __ldcg(&ctl->status) != 0;
  if (!grid_barrier(&ctl->gbar, (++nbar) * nblk)) {
    if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
    return;
  }

  for (long long step = 0; step < p.n_steps; ++step) {
    if (stop || !(t < t_final)) break;
    double alpha[M];
    double dt;
    // ---- RK1 (alphas of u^n in slot 0)
#pragma unroll
    for (int s = 0; s < M; ++s) alpha[s] = bits_to_double(__ldcg(&ctl->amax[0][s]));
    {
      const double smax = (FLUX == WT_FLUX_EULER1D) ? ((alpha[0] < alpha[M - 1]) ? alpha[M - 1] : alpha[0]) : alpha[0];
      dt = dt_fixed > 0.0 ? dt_fixed : MATH::cfl_dt(cfl, p.a[0].dx, smax);
      const double rem = t_final - t;
      if (rem < dt) dt = rem;
    }
    if (first && tid < 8) ctl->amax[2][tid] = 0ull;
    if (first && tid == 0) ctl->dt = dt;
    stage1d_compute<MATH, FLUX, STAGE_RK1, T, kResident>(p.a[0], j0, Tc, 0, j0, j0 + Tc, alpha, dt, sm,
                                                         AlphaWait{0ull, 0, -1, 0, 0.0, 0.0, 0.0, 0.0});
    if (!grid_barrier(&ctl->gbar, (++nbar) * nblk)) {
      if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
      return;
    }
    load_halos<MATH, FLUX, T>(p.a[1].uin, pitch, j0, Tc, s_uin);
    // ---- RK2
#pragma unroll
    for (int s = 0; s < M; ++s) alpha[s] = bits_to_double(__ldcg(&ctl->amax[1][s]));
    if (first && tid < 8) ctl->amax[0][tid] = 0ull;
    stage1d_compute<MATH, FLUX, STAGE_RK2, T, kResident>(p.a[1], j0, Tc, 0, j0, j0 + Tc, alpha, dt, sm,
                                                         AlphaWait{0ull, 0, -1, 0, 0.0, 0.0, 0.0, 0.0});
    if (!grid_barrier(&ctl->gbar, (++nbar) * nblk)) {
      if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
      return;
    }
    load_halos<MATH, FLUX, T>(p.a[2].uin, pitch, j0, Tc, s_uin);
    // ---- RK3
#pragma unroll
    for (int s = 0; s < M; ++s) alpha[s] = bits_to_double(__ldcg(&ctl->amax[2][s]));
    if (first && tid < 8) ctl->amax[1][tid] = 0ull;
    stage1d_compute<MATH, FLUX, STAGE_RK3, T, kResident>(p.a[2], j0, Tc, 0, j0, j0 + Tc, alpha, dt, sm,
                                                         AlphaWait{0ull, 0, -1, 0, 0.0, 0.0, 0.0, 0.0});
    t = t + dt;
    const int v = (int)(step % 3);
    if (tid == 0) {
      if (first) {
        ctl->t = t;
        ctl->steps = ctl->steps + 1;
      }
      if (__ldcg(&ctl->status) != 0) atomicOr(&ctl->vote[v], 1u);
    }
    if (!grid_barrier(&ctl->gbar, (++nbar) * nblk)) {
      if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
      return;
    }
    stop = __ldcg(&ctl->vote[v]) != 0;
    if (first && tid == 0) ctl->vote[(v + 2) % 3] = 0u;
    load_halos<MATH, FLUX, T>(p.a[0].uin, pitch, j0, Tc, s_uin);
  }
}

// ---------------------------------------------------------------------------------------
// Step-blocked persistent RK3 integration: one CTA per tile of T cells, on at most one tile
// per SM.  At the start of a step each CTA holds u^n over its cells and 9 halo cells per
// side (3 per stage); it computes stage 1 over its cells and 6 halo cells per side, stage 2
// over 3 per side and stage 3 over its own cells, so the only exchange between neighbours
// is the halo reload at the start of a step.  The halo cells are computed with exactly the
// arithmetic, alphas and dt of their owners.  Non-periodic ends: the computed range stops
// at the boundary and phase B re-images the ghost cells from the stage input.
// Exchanges go through tagged mailboxes, with no fence, counter or grid barrier per step:
//   halos   stage 3 writes u^{n+1} of the CTA's own cells as two words tagged with the
//           step; the next step polls the 9 halo cells per side until their tags match;
//   alphas  phase B of each stage: the speed warp writes the maxima of the CTA's own cells
//           of the stage input, tagged with the step's parity, and gathers every CTA's, all
//           while the other warps do the alpha-free work (cell quantities, Roe matrices,
//           the (l.f, l.u) products).  dt follows from the alphas of the first stage.
// Stop decisions: t_final is seen identically by every CTA; a failure seen by any CTA
// (its status view, published with the first stage's alphas) stops every CTA before it
// takes that step, so the state in global memory is the last completed step's.
// ---------------------------------------------------------------------------------------
template <class MATH, int FLUX, int T>
__device__ __forceinline__ void sb_load_window(const double* un, long long pitch, long long n, long long x0, int k_lo,
                                               int k_hi, bool per_lo, bool per_hi, double* s_uin, double* s_un, int W) {
  constexpr int M = FluxM<FLUX>::m;
  const int span = k_hi - k_lo;
  for (int idx = threadIdx.x; idx < M * span; idx += blockDim.x) {
    const int c = idx / span, k = k_lo + (idx - c * span);
    const long long x = x0 + k;
    long long src;
    if (x < 0) {
      if (per_lo) src = ((x % n) + n) % n;
      else if (x >= -G) src = x;
      else continue;
    } else if (x >= n) {
      if (per_hi) src = x % n;
      else if (x < n + G) src = x;
      else continue;
    } else {
      src = x;
    }
    const double v = __ldcg(un + c * pitch + src + G);
    s_uin[c * W + k] = v;
    s_un[c * W + k] = v;
  }
}

// Halo cells of u^n at the start of a step (window positions [0, E0) and [Tc + E0, Tc + 2 E0))
// from the halo mailbox: words tagged `tag`, polled with a bounded wait.  Ghost cells of a
// non-periodic end are skipped: phase B re-images them from the stage input.  Returns false
// for every thread of the block if a wait timed out.
template <int M>
__device__ __forceinline__ bool sb_mailbox_halo(const unsigned long long* hi, const unsigned long long* lo,
                                                long long pitch, long long n, long long x0, int Tc, int E0,
                                                bool per_lo, bool per_hi, unsigned int tag, double* s_uin,
                                                double* s_un, int W, long long limit = kWaitLimit) {
  int bad = 0;
  const int nh = 2 * E0;
  for (int idx = threadIdx.x; idx < M * nh; idx += blockDim.x) {
    const int c = idx / nh, h = idx - c * nh;
    const int k = (h < E0) ? h : Tc + h;
    const long long x = x0 + k;
    long long src;
    if (x < 0) {
      if (!per_lo) continue;
      src = ((x % n) + n) % n;
    } else if (x >= n) {
      if (!per_hi) continue;
      src = x % n;
    } else {
      src = x;
    }
    const unsigned long long* ph = hi + c * pitch + src;
    const unsigned long long* pl = lo + c * pitch + src;
    const long long start = clock64();
    unsigned long long wh, wl;
    for (;;) {
      wh = ld_relaxed_u64(ph);
      wl = ld_relaxed_u64(pl);
      if ((unsigned int)(wh >> 32) == tag && (unsigned int)(wl >> 32) == tag) break;
      if (clock64() - start > limit) {
        bad = 1;
        break;
      }
    }
    const double v = __longlong_as_double((long long)((wh << 32) | (wl & 0xffffffffull)));
    s_uin[c * W + k] = v;
    s_un[c * W + k] = v;
  }
  return __syncthreads_or(bad) == 0;
}

// one CTA per SM (the launch checks that the grid is co-resident)
template <class MATH, int FLUX, int T>
__global__ void __launch_bounds__(Tile1D<T + 4 * G, FluxM<FLUX>::m, 2>::NT, 1) stepblock1d_kernel(const PersistArgs p) {
  constexpr int M = FluxM<FLUX>::m;
  constexpr int E0 = 3 * G;   // halo cells per side at the start of a step
  constexpr int TB = T + 4 * G;  // cells computed in stage 1: T + 2 * (E0 - G)
  using TL = TileOf<MATH, FLUX, TB, 2>;
  constexpr int W = TL::W;
  static_assert(W >= T + 2 * E0, "window of a step");
  extern __shared__ __align__(16) double sm[];
  double* s_uin = sm + TL::kUin;
  double* s_un = sm + TL::kUn;
  const int tid = threadIdx.x;
  Ctl* ctl = p.a[0].ctl;
  const long long n = p.a[0].n, pitch = p.a[0].pitch;
  const long long j0 = (long long)blockIdx.x * T;
  const int Tc = (int)((n - j0 < T) ? (n - j0) : T);
  const long long x0 = j0 - E0;
  const int wcells = Tc + 2 * E0;
  const int bc_lo = p.a[0].bc_lo, bc_hi = p.a[0].bc_hi;
  const bool per_lo = bc_lo == WT_BC_PERIODIC, per_hi = bc_hi == WT_BC_PERIODIC;
  const bool first = blockIdx.x == 0;
  const unsigned long long nblk = gridDim.x;
  unsigned long long* gbar = &ctl->gbar;
  unsigned long long nbar = 0;

  sb_load_window<MATH, FLUX, T>(p.a[0].uin, pitch, n, x0, 0, wcells, per_lo, per_hi, s_uin, s_un, W);
  const double t_final = __ldcg(&ctl->t_final), cfl = __ldcg(&ctl->cfl), dt_fixed = __ldcg(&ctl->dt_fixed);
  double t = __ldcg(&ctl->t);
  // status as it stands before any block of this launch can flag a failure
  bool stop = __ldcg(&ctl->status) != 0;
  grid_arrive(gbar);
  if (!grid_wait(gbar, (++nbar) * nblk)) {
    if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
    return;
  }

  // computed range of a stage with e halo cells per side, clipped at non-periodic ends
  auto range = [&](int e, long long& lo, int& Ts, int& off) {
    long long l = j0 - e, h = j0 + Tc + e;
    if (!per_lo && l < 0) l = 0;
    if (!per_hi && h > n) h = n;
    lo = l;
    Ts = (int)(h - l);
    off = (int)(l - G - x0);
  };

  const int* s_aflag = reinterpret_cast<const int*>(sm + TL::kQn) + 1;
  for (long long step = 0;; ++step) {
    if (step >= p.n_steps || stop || !(t < t_final)) break;
    if (step > 0) {
      // halo cells of u^n: the neighbours' stage-3 words of the previous step
      if (!sb_mailbox_halo<M>(p.hmb_hi, p.hmb_lo, pitch, n, x0, Tc, E0, per_lo, per_hi, (unsigned int)step, s_uin,
                              s_un, W)) {
        if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
        return;
      }
    }
    __syncthreads();

    const unsigned long long par = (unsigned long long)((~step) & 1);  // the mailboxes start zeroed
    double alpha[M], dt = 0.0;
    long long lo;
    int Ts, off;
    // ---- RK1: alphas of u^n (slot 0), then dt; a failure seen by any CTA stops here
    range(2 * G, lo, Ts, off);
    if (!stage1d_compute<MATH, FLUX, STAGE_RK1, TB, kStepBlocked>(
            p.a[0], lo, Ts, off, j0, j0 + Tc, alpha, dt, sm,
            AlphaWait{0ull, 0, first ? 2 : -1, 1, cfl, dt_fixed, t, t_final, p.amb, par, nullptr, nullptr, 0u})) {
      if (*s_aflag != 3 && tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
      return;
    }
    // ---- RK2: alphas of u1 (slot 1)
    range(G, lo, Ts, off);
    if (!stage1d_compute<MATH, FLUX, STAGE_RK2, TB, kStepBlocked>(
            p.a[1], lo, Ts, off, j0, j0 + Tc, alpha, dt, sm,
            AlphaWait{0ull, 1, -1, 0, 0.0, 0.0, 0.0, 0.0, p.amb, par, nullptr, nullptr, 0u})) {
      if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
      return;
    }
    // ---- RK3: alphas of u2 (slot 2); u^{n+1} of the CTA's cells to global memory and to the
    // halo mailbox (tag step + 1)
    range(0, lo, Ts, off);
    if (!stage1d_compute<MATH, FLUX, STAGE_RK3, TB, kStepBlocked>(
            p.a[2], lo, Ts, off, j0, j0 + Tc, alpha, dt, sm,
            AlphaWait{0ull, 2, -1, 0, 0.0, 0.0, 0.0, 0.0, p.amb, par, p.hmb_hi, p.hmb_lo, (unsigned int)(step + 1)})) {
      if (tid == 0) flag_error(ctl, WT_ERR_TIMEOUT);
      return;
    }
    t = t + dt;
    if (first && tid == 0) {
      ctl->t = t;
      ctl->steps = ctl->steps + 1;
    }
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
  using TL = TileOf<MATH, FLUX, T, 1, 1, true>;
  static_assert(TL::bytes <= 48 * 1024, "tile exceeds the default dynamic shared memory limit");
  auto kern = stage1d_kernel<MATH, FLUX, STAGE, T>;
  const unsigned grid = (unsigned)((a.n + T - 1) / T);
  return launch_pdl(kern, dim3(grid), dim3(TL::NT), TL::bytes, st, a);
}

// Cooperative launch of the persistent kernel (grid = number of tiles, all co-resident)
template <class MATH, int FLUX, int T>
cudaError_t launch_persist1d_t(const PersistArgs& p, int grid, cudaStream_t st) {
  using TL = TileOf<MATH, FLUX, T>;
  static_assert(TL::bytes <= 48 * 1024, "tile exceeds the default dynamic shared memory limit");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(TL::NT);
  cfg.dynamicSmemBytes = TL::bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, persist1d_kernel<MATH, FLUX, T>, p);
}

// CTAs of the persistent kernel that fit on the device at once (0: no cooperative launch)
template <class MATH, int FLUX, int T>
int persist1d_capacity_t() {
  using TL = TileOf<MATH, FLUX, T>;
  int dev = 0, sms = 0, coop = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persist1d_kernel<MATH, FLUX, T>, TL::NT, TL::bytes) !=
      cudaSuccess)
    return 0;
  return per * sms;
}

// Cooperative launch of the step-blocked kernel (grid = number of tiles of T cells)
template <class MATH, int FLUX, int T>
cudaError_t launch_stepblock1d_t(const PersistArgs& p, int grid, cudaStream_t st) {
  using TL = TileOf<MATH, FLUX, T + 4 * G, 2>;
  static_assert(TL::bytes <= 48 * 1024, "tile exceeds the default dynamic shared memory limit");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(TL::NT);
  cfg.dynamicSmemBytes = TL::bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, stepblock1d_kernel<MATH, FLUX, T>, p);
}

template <class MATH, int FLUX, int T>
int stepblock1d_capacity_t() {
  using TL = TileOf<MATH, FLUX, T + 4 * G, 2>;
  int dev = 0, sms = 0, coop = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stepblock1d_kernel<MATH, FLUX, T>, TL::NT, TL::bytes) !=
      cudaSuccess)
    return 0;
  return per * sms;
}

template <class MATH>
int stepblock1d_capacity_policy(int flux) {
  switch (flux) {
    case WT_FLUX_EULER1D: return stepblock1d_capacity_t<MATH, WT_FLUX_EULER1D, 27>();
    case WT_FLUX_ADVECTION: return stepblock1d_capacity_t<MATH, WT_FLUX_ADVECTION, 51>();
    case WT_FLUX_BURGERS: return stepblock1d_capacity_t<MATH, WT_FLUX_BURGERS, 51>();
  }
  return 0;
}

template <class MATH>
cudaError_t launch_stepblock1d_policy(int flux, const PersistArgs& p, int grid, cudaStream_t st) {
  switch (flux) {
    case WT_FLUX_EULER1D: return launch_stepblock1d_t<MATH, WT_FLUX_EULER1D, 27>(p, grid, st);
    case WT_FLUX_ADVECTION: return launch_stepblock1d_t<MATH, WT_FLUX_ADVECTION, 51>(p, grid, st);
    case WT_FLUX_BURGERS: return launch_stepblock1d_t<MATH, WT_FLUX_BURGERS, 51>(p, grid, st);
  }
  return cudaErrorInvalidValue;
}

// tiles with a persistent kernel: 31 and 63 (Euler), 63 (scalar fluxes); 0 for the others
template <class MATH>
int persist1d_capacity_policy(int flux, int tile) {
  if (flux == WT_FLUX_EULER1D) {
    if (tile == 31) return persist1d_capacity_t<MATH, WT_FLUX_EULER1D, 31>();
    if (tile == 63) return persist1d_capacity_t<MATH, WT_FLUX_EULER1D, 63>();
    return 0;
  }
  if (tile != 63) return 0;
  if (flux == WT_FLUX_ADVECTION) return persist1d_capacity_t<MATH, WT_FLUX_ADVECTION, 63>();
  if (flux == WT_FLUX_BURGERS) return persist1d_capacity_t<MATH, WT_FLUX_BURGERS, 63>();
  return 0;
}

template <class MATH>
cudaError_t launch_persist1d_policy(int flux, int tile, const PersistArgs& p, int grid, cudaStream_t st) {
  if (flux == WT_FLUX_EULER1D) {
    if (tile == 31) return launch_persist1d_t<MATH, WT_FLUX_EULER1D, 31>(p, grid, st);
    if (tile == 63) return launch_persist1d_t<MATH, WT_FLUX_EULER1D, 63>(p, grid, st);
    return cudaErrorInvalidValue;
  }
  if (tile != 63) return cudaErrorInvalidValue;
  if (flux == WT_FLUX_ADVECTION) return launch_persist1d_t<MATH, WT_FLUX_ADVECTION, 63>(p, grid, st);
  if (flux == WT_FLUX_BURGERS) return launch_persist1d_t<MATH, WT_FLUX_BURGERS, 63>(p, grid, st);
  return cudaErrorInvalidValue;
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

template <class MATH, int FLUX, int STAGE, int T, int IPT, bool REC = false>
cudaError_t launch_stage1d_batched_t(const BatchArgs& b, int grid, cudaStream_t st) {
  using TL = TileOf<MATH, FLUX, T, 1, IPT, true>;
  static_assert(TL::bytes <= 48 * 1024, "tile exceeds the default dynamic shared memory limit");
  return launch_pdl(stage1d_batched_kernel<MATH, FLUX, STAGE, T, IPT, REC>, dim3(grid), dim3(TL::NT), TL::bytes, st,
                    b);
}

// the adjoint's recording forward stage: 1D Euler, 127-cell tiles, six items per thread
template <class MATH>
cudaError_t launch_stage1d_batched_record_policy(int stage, const BatchArgs& b, int grid, cudaStream_t st) {
  switch (stage) {
    case STAGE_RK1: return launch_stage1d_batched_t<MATH, WT_FLUX_EULER1D, STAGE_RK1, 127, 6, true>(b, grid, st);
    case STAGE_RK2: return launch_stage1d_batched_t<MATH, WT_FLUX_EULER1D, STAGE_RK2, 127, 6, true>(b, grid, st);
    case STAGE_RK3: return launch_stage1d_batched_t<MATH, WT_FLUX_EULER1D, STAGE_RK3, 127, 6, true>(b, grid, st);
  }
  return cudaErrorInvalidValue;
}

template <class MATH, int FLUX, int T, int IPT = 1>
cudaError_t launch_stage1d_batched_flux(int stage, const BatchArgs& b, int grid, cudaStream_t st) {
  switch (stage) {
    case STAGE_RK1: return launch_stage1d_batched_t<MATH, FLUX, STAGE_RK1, T, IPT>(b, grid, st);
    case STAGE_RK2: return launch_stage1d_batched_t<MATH, FLUX, STAGE_RK2, T, IPT>(b, grid, st);
    case STAGE_RK3: return launch_stage1d_batched_t<MATH, FLUX, STAGE_RK3, T, IPT>(b, grid, st);
  }
  return cudaErrorInvalidValue;
}

// tile: the batched tile code, cells per tile + 1000 x (items per thread - 1) (wt_launch.h)
template <class MATH>
cudaError_t launch_stage1d_batched_policy(int flux, int stage, int tile, const BatchArgs& b, int grid,
                                          cudaStream_t st) {
  if (flux == WT_FLUX_EULER1D) {
    if (tile == 31) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 31>(stage, b, grid, st);
    if (tile == 63) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 63>(stage, b, grid, st);
    if (tile == 127) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 127>(stage, b, grid, st);
    if (tile == 1063) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 63, 2>(stage, b, grid, st);
    if (tile == 1127) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 127, 2>(stage, b, grid, st);
    if (tile == 2127) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 127, 3>(stage, b, grid, st);
    if (tile == 3127) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 127, 4>(stage, b, grid, st);
    if (tile == 5127) return launch_stage1d_batched_flux<MATH, WT_FLUX_EULER1D, 127, 6>(stage, b, grid, st);
  } else if (flux == WT_FLUX_ADVECTION) {
    if (tile == 63) return launch_stage1d_batched_flux<MATH, WT_FLUX_ADVECTION, 63>(stage, b, grid, st);
    if (tile == 127) return launch_stage1d_batched_flux<MATH, WT_FLUX_ADVECTION, 127>(stage, b, grid, st);
  } else if (flux == WT_FLUX_BURGERS) {
    if (tile == 63) return launch_stage1d_batched_flux<MATH, WT_FLUX_BURGERS, 63>(stage, b, grid, st);
    if (tile == 127) return launch_stage1d_batched_flux<MATH, WT_FLUX_BURGERS, 127>(stage, b, grid, st);
  }
  return cudaErrorInvalidValue;
}

template <class MATH, int FLUX, int T, int IPT = 1>
int batched_occupancy_t() {
  using TL = TileOf<MATH, FLUX, T, 1, IPT, true>;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage1d_batched_kernel<MATH, FLUX, STAGE_RK2, T, IPT>,
                                                    TL::NT, TL::bytes) != cudaSuccess)
    return 0;
  return nb;
}

template <class MATH>
int batched_occupancy_policy(int flux, int tile) {
  if (flux == WT_FLUX_EULER1D) {
    if (tile == 31) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 31>();
    if (tile == 63) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 63>();
    if (tile == 127) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 127>();
    if (tile == 1063) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 63, 2>();
    if (tile == 1127) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 127, 2>();
    if (tile == 2127) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 127, 3>();
    if (tile == 3127) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 127, 4>();
    if (tile == 5127) return batched_occupancy_t<MATH, WT_FLUX_EULER1D, 127, 6>();
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
