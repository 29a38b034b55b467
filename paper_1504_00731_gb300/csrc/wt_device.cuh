// Device-side building blocks shared by the WENO-theta kernels: the control block kept in
// the workspace, bulk-copy (TMA) staging with bounded mbarrier waits, block-wide maxima,
// and ghost-cell index maps.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/weno_theta.h"

namespace wt {

constexpr int G = 3;  // ghost cells per side: the stencil of an interface is {j-2 .. j+3}

// Per-run control block, resident in the workspace.  Lax-Friedrichs constants are kept
// as the bit patterns of non-negative doubles so that atomicMax on unsigned 64-bit
// integers is an exact maximum.  A ring of three slots lets stage s read slot s, fill
// slot s+1 and clear slot s+2 without a separate launch.
struct Ctl {
  unsigned long long amax[3][8];  // [slot][dir * 4 + field]
  unsigned long long cfl2d[3];    // 2D: max_j ((|u|+c)/dx + (|v|+c)/dy) per slot
  double t;                       // time reached
  double dt;                      // step of the current RK step
  double t_final;
  double cfl;
  double dt_fixed;
  long long steps;
  int status;                     // first device-detected failure (wt_status), 0 if none
  int active;                     // 1 while the current step is being taken
  int pad[2];
  // persistent kernel: grid-barrier arrivals of the launch, and per-step stop votes (ring of 3)
  unsigned long long gbar;
  unsigned int vote[3];
  int pad2;
};

__device__ __forceinline__ void flag_error(Ctl* ctl, int code) {
  if (ctl) atomicCAS(&ctl->status, 0, code);
}

// The state must stay finite.  Negative pressure (or density) in an intermediate RK stage
// is not an error: the scheme has no positivity limiter and a literal evaluation carries
// on through it (the sound speed there is NaN and drops out of the alpha maxima).
__device__ __forceinline__ bool finite3(const double* U) { return isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]); }

// Programmatic dependent launch: let the next kernel in the stream start its prologue now,
// and wait (in hardware) until the previous kernel has completed and its writes are visible.
// Both are no-ops for a kernel launched without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------------------
// Bulk copies global -> shared (cp.async.bulk, completion on an mbarrier)
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// dst, src 16-byte aligned; bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after `limit` SM clock cycles (default 2^31, about one second).
constexpr long long kWaitLimit = 1LL << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = kWaitLimit) {
  const long long start = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - start > limit) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Block-wide maxima of wave speeds, on bit patterns.  Speeds are non-negative, and
// non-negative doubles order like their bit patterns, so the maxima run on the integer
// pipe instead of the narrow FP64 one.  A NaN speed (the sound speed of a finite state
// whose pressure went negative) maps to key 0 and so drops out of the maximum.
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long speed_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return b > 0x7FF0000000000000ull ? 0ull : b;
}
__device__ __forceinline__ void key_max(unsigned long long& acc, double x) {
  const unsigned long long k = speed_key(x);
  acc = (acc < k) ? k : acc;
}

__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (v < w) ? w : v;
  }
  return v;
}

// The same maximum (every lane of a full warp) from two 32-bit warp reductions: the largest
// high word, then the largest low word among the lanes that hold it.  A shorter dependent
// chain than five shuffle rounds, for the alpha exchange of the step-blocked kernel.
__device__ __forceinline__ unsigned long long warp_max_key_redux(unsigned long long v) {
  const unsigned hi = (unsigned)(v >> 32);
  const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? (unsigned)v : 0u);
  return ((unsigned long long)mh << 32) | ml;
}

// x with its sign bit XORed with that of sg (0 or -0.0's pattern): an exact negation on the
// integer pipe
__device__ __forceinline__ double flip_sign(double x, unsigned long long sg) {
  return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(x) ^ sg));
}

// ---------------------------------------------------------------------------------------
// FP32 screen of the 1D Euler wave speeds, so that a tile takes the FP64 speeds of only the
// cells that can hold its maxima.  The FP64 maxima over those cells are the maxima over all.
// ---------------------------------------------------------------------------------------

// The high 32 bits of a double as a float: sign, exponent rebiased, the top 20 bits of the
// mantissa, so |f32_hi(x) - x| < 2^-20 |x| for 2^-126 <= |x| < 2^128 (0 below).  Integer pipe.
__device__ __forceinline__ float f32_hi(double x) {
  const int hi = __double2hiint(x);
  const int mag = hi & 0x7fffffff;
  return mag < 0x38100000 ? 0.0f : __int_as_float(((mag - 0x38000000) << 3) | (hi & 0x80000000));
}

// lam = (|u - c|, |u|, |u + c|) of U = (rho, m, E) in FP32, g = gamma (gamma - 1) (a float
// within 2^-20 of it).  Returns false, and leaves lam unset, unless rho and E lie in
// [2^-60, 2^60], m is 0 or 2^-100 <= |m| <= 2^60, and the internal energy E - m u / 2 is at
// least E / 16.  Otherwise, with d = 2^-20 (each input within d of its value) and every FP32
// operation within 2^-22: 1 / rho within 1.1 d; u within 2.2 d of m / rho (relative, so
// lam[1] is within 2.3 d of |u|); m u / 2 within 3.3 d, hence the internal energy within
// 4.3 d E absolute, at most 69 d relative; c^2 = g (E - m u / 2) / rho within 71 d and c
// within 36 d; so lam[0], lam[2] are within 37 d (|u| + c) < 2^-14.7 (|u| + c) of the exact
// speeds.  The FP64 speeds are within a few 2^-53 of those.
__device__ __forceinline__ bool euler_speeds_screen(const double* U, float g, float* lam) {
  const float r = f32_hi(U[0]), m = f32_hi(U[1]), E = f32_hi(U[2]);
  const float am = fabsf(m);
  if (!(r >= 0x1p-60f && r <= 0x1p60f && E >= 0x1p-60f && E <= 0x1p60f && am <= 0x1p60f &&
        (am >= 0x1p-100f || (__double_as_longlong(U[1]) << 1) == 0)))
    return false;
  const float ir = __frcp_rn(r);
  const float u = m * ir;
  const float pe = fmaf(-0.5f * m, u, E);
  if (!(pe >= 0.0625f * E)) return false;
  const float c2 = (g * pe) * ir;
  const float c = c2 * rsqrtf(c2);
  lam[0] = fabsf(u - c);
  lam[1] = fabsf(u);
  lam[2] = fabsf(u + c);
  return true;
}

// Reduces K keys per thread to the block maximum and folds it into dst[k] with one
// atomicMax per block.  scratch: >= K * 32 doubles of shared memory.
template <int K>
__device__ __forceinline__ void block_max_atomic(unsigned long long (&v)[K], double* scratch_d,
                                                 unsigned long long* dst) {
  unsigned long long* scratch = reinterpret_cast<unsigned long long*>(scratch_d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const unsigned long long w = warp_max_key(v[k]);
    if (lane == 0) scratch[k * 32 + warp] = w;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    unsigned long long m = 0ull;
    for (int w = 0; w < nw; ++w) {
      const unsigned long long x = scratch[threadIdx.x * 32 + w];
      m = (m < x) ? x : m;
    }
    atomicMax(&dst[threadIdx.x], m);
  }
}

// Named CTA barrier `id` over `count` threads: arrive without waiting, or arrive and wait
__device__ __forceinline__ void named_barrier_arrive(int id, int count) {
  asm volatile("barrier.cta.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_barrier_sync(int id, int count) {
  asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// ---------------------------------------------------------------------------------------
// Grid-wide barrier of a cooperative (co-resident) grid.  ctr counts arrivals from 0 at the
// launch; the k-th barrier of the launch (k = 1, 2, ...) waits for k * gridDim.x of them.
// The stores of the block before the barrier are visible to every block after it (fence +
// release by arrival, acquire by the waiting thread, then a CTA barrier).  Data written
// during the launch by other blocks must be read around L1 (ld.global.cg).  The wait is
// bounded: false (for every thread of the block) once about 2^31 clocks have passed.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Relaxed gpu-scope 8-byte accesses: single-copy atomic and coherent per location, so a
// reader sees either the old or the new word.  The mailboxes of the step-blocked kernel
// carry a tag inside each word and need no fence.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Four relaxed 8-byte words from a 32-byte aligned address in one request.  Each word is
// single-copy atomic on its own; the four are not read as one atomic unit.
__device__ __forceinline__ void ld_relaxed_v4_u64(const unsigned long long* p, unsigned long long (&w)[4]) {
  asm volatile("ld.relaxed.gpu.global.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3])
               : "l"(p)
               : "memory");
}

// arrival: every thread's earlier stores are ordered before it (CTA barrier, then a gpu fence)
__device__ __forceinline__ void grid_arrive(unsigned long long* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1ull);
  }
}

// wait for `target` arrivals; false for every thread of the block on timeout
__device__ __forceinline__ bool grid_wait(const unsigned long long* ctr, unsigned long long target,
                                          long long limit = kWaitLimit) {
  int bad = 0;
  if (threadIdx.x == 0) {
    const long long start = clock64();
    while (ld_acquire_u64(ctr) < target) {
      if (clock64() - start > limit) {
        bad = 1;
        break;
      }
    }
    __threadfence();
  }
  return __syncthreads_or(bad) == 0;
}

__device__ __forceinline__ bool grid_barrier(unsigned long long* ctr, unsigned long long target) {
  grid_arrive(ctr);
  return grid_wait(ctr, target);
}

__device__ __forceinline__ double bits_to_double(unsigned long long b) { return __longlong_as_double((long long)b); }

// ---------------------------------------------------------------------------------------
// Ghost cells: interior index of the cell whose value ghost index g (g < 0 or g >= n)
// takes, and whether the normal momentum flips sign.
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ long long ghost_source(long long g, long long n, int bc_lo, int bc_hi, bool* flip) {
  *flip = false;
  if (g < 0) {
    if (bc_lo == WT_BC_PERIODIC) return g + n;
    if (bc_lo == WT_BC_OUTFLOW) return 0;
    *flip = true;
    return -g - 1;
  }
  if (bc_hi == WT_BC_PERIODIC) return g - n;
  if (bc_hi == WT_BC_OUTFLOW) return n - 1;
  *flip = true;
  return 2 * n - 1 - g;
}

}  // namespace wt
