// Fast-arithmetic instantiations of the 1D kernels, plus the boundary-fill (pack) and
// unpack kernels, which do no arithmetic.
#define WT_ADJOINT_COMMON_KERNELS
#include <cstdlib>

#include "wt_kernels.cuh"
#include "wt_kernels2d.cuh"
#include "wt_adjoint.cuh"
#include "wt_math_fast.cuh"

namespace wt {

__global__ void pack1d_kernel(const double* __restrict__ src, long long src_stride, double* __restrict__ dst,
                              long long n, long long pitch, int m, int bc_lo, int bc_hi, int flip_comp) {
  const long long row = n + 2 * G;
  const long long total = (long long)m * row;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / row);
    const long long p = idx - (long long)c * row;
    const long long j = p - G;
    bool flip = false;
    const long long sj = (j >= 0 && j < n) ? j : ghost_source(j, n, bc_lo, bc_hi, &flip);
    double v = src[c * src_stride + sj];
    if (flip && c == flip_comp) v = -v;
    dst[c * pitch + p] = v;
  }
}

__global__ void unpack1d_kernel(const double* __restrict__ src, long long pitch, double* __restrict__ dst,
                                long long dst_stride, long long n, int m) {
  const long long total = (long long)m * n;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / n);
    const long long j = idx - (long long)c * n;
    dst[c * dst_stride + j] = src[c * pitch + j + G];
  }
}

static unsigned copy_grid(long long total) {
  long long b = (total + 255) / 256;
  if (b > 4864) b = 4864;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_pack1d(const double* src, long long src_stride, double* dst, long long n, long long pitch, int m,
                          int bc_lo, int bc_hi, int flip_comp, cudaStream_t st) {
  pack1d_kernel<<<copy_grid((long long)m * (n + 2 * G)), 256, 0, st>>>(src, src_stride, dst, n, pitch, m, bc_lo, bc_hi,
                                                                         flip_comp);
  return cudaGetLastError();
}

cudaError_t launch_unpack1d(const double* src, long long pitch, double* dst, long long dst_stride, long long n, int m,
                            cudaStream_t st) {
  unpack1d_kernel<<<copy_grid((long long)m * n), 256, 0, st>>>(src, pitch, dst, dst_stride, n, m);
  return cudaGetLastError();
}

__global__ void pack1d_batched_kernel(const double* __restrict__ src, long long src_stride, double* __restrict__ dst,
                                      long long pitch, const BatchSeg* __restrict__ segs, int m, int flip_comp) {
  const BatchSeg sg = segs[blockIdx.y];
  const long long row = sg.n + 2 * G;
  const long long total = (long long)m * row;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / row);
    const long long p = idx - (long long)c * row;
    const long long j = p - G;
    bool flip = false;
    const long long sj = (j >= 0 && j < sg.n) ? j : ghost_source(j, sg.n, sg.bc_lo, sg.bc_hi, &flip);
    double v = src[c * src_stride + sg.uoff + sj];
    if (flip && c == flip_comp) v = -v;
    dst[c * pitch + sg.poff + p] = v;
  }
}

// skip (may be null): problems whose control block carries a failure are not written, so the
// destination keeps what it held (the caller's input state)
__global__ void unpack1d_batched_kernel(const double* __restrict__ src, long long pitch, double* __restrict__ dst,
                                        long long dst_stride, const BatchSeg* __restrict__ segs, int m,
                                        const Ctl* __restrict__ skip) {
  if (skip && skip[blockIdx.y].status != 0) return;
  const BatchSeg sg = segs[blockIdx.y];
  const long long total = (long long)m * sg.n;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / sg.n);
    const long long j = idx - (long long)c * sg.n;
    dst[c * dst_stride + sg.uoff + j] = src[c * pitch + sg.poff + j + G];
  }
}

__global__ void gather_t_kernel(const Ctl* __restrict__ ctl, int nprob, double* __restrict__ t_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob) t_out[p] = ctl[p].t;
}

__global__ void gather_status_kernel(const Ctl* __restrict__ ctl, int nprob, int* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob) out[p] = ctl[p].status;
}

static dim3 batched_grid(long long maxn, int m, int nprob) {
  long long bx = ((long long)m * (maxn + 2 * G) + 255) / 256;
  if (bx > 64) bx = 64;
  return dim3((unsigned)(bx < 1 ? 1 : bx), (unsigned)nprob);
}

cudaError_t launch_pack1d_batched(const double* src, long long src_stride, double* dst, long long pitch,
                                  const BatchSeg* segs, int nprob, long long maxn, int m, int flip_comp, cudaStream_t st) {
  pack1d_batched_kernel<<<batched_grid(maxn, m, nprob), 256, 0, st>>>(src, src_stride, dst, pitch, segs, m, flip_comp);
  return cudaGetLastError();
}

cudaError_t launch_unpack1d_batched(const double* src, long long pitch, double* dst, long long dst_stride,
                                    const BatchSeg* segs, int nprob, long long maxn, int m, cudaStream_t st,
                                    const Ctl* skip_failed) {
  unpack1d_batched_kernel<<<batched_grid(maxn, m, nprob), 256, 0, st>>>(src, pitch, dst, dst_stride, segs, m,
                                                                        skip_failed);
  return cudaGetLastError();
}

cudaError_t launch_gather_status(const Ctl* ctl, int nprob, int* out, cudaStream_t st) {
  gather_status_kernel<<<(nprob + 255) / 256, 256, 0, st>>>(ctl, nprob, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_t(const Ctl* ctl, int nprob, double* t_out, cudaStream_t st) {
  gather_t_kernel<<<(nprob + 255) / 256, 256, 0, st>>>(ctl, nprob, t_out);
  return cudaGetLastError();
}

cudaError_t launch_persist1d_fast(int flux, int tile, const PersistArgs& p, int grid, cudaStream_t st) {
  return launch_persist1d_policy<FastMath>(flux, tile, p, grid, st);
}

int persist1d_capacity_fast(int flux, int tile) { return persist1d_capacity_policy<FastMath>(flux, tile); }

cudaError_t launch_stepblock1d_fast(int flux, const PersistArgs& p, int grid, cudaStream_t st) {
  return launch_stepblock1d_policy<FastMath>(flux, p, grid, st);
}

int stepblock1d_capacity_fast(int flux) { return stepblock1d_capacity_policy<FastMath>(flux); }

cudaError_t launch_stage1d_fast(int flux, int stage, int tile, const Stage1DArgs& a, cudaStream_t st) {
  return launch_stage1d_policy<FastMath>(flux, stage, tile, a, st);
}

cudaError_t launch_alpha1d_fast(int flux, const double* u, long long n, long long pitch, double gamma, double adv,
                                Ctl* ctl, int slot, cudaStream_t st) {
  return launch_alpha1d_policy<FastMath>(flux, u, n, pitch, gamma, adv, ctl, slot, st);
}

cudaError_t launch_stage1d_batched_fast(int flux, int stage, int tile, const BatchArgs& b, int grid, cudaStream_t st) {
  return launch_stage1d_batched_policy<FastMath>(flux, stage, tile, b, grid, st);
}

cudaError_t launch_stage1d_batched_record_fast(int stage, const BatchArgs& b, int grid, cudaStream_t st) {
  return launch_stage1d_batched_record_policy<FastMath>(stage, b, grid, st);
}

cudaError_t launch_alpha1d_batched_fast(int flux, const double* u, long long pitch, const BatchSeg* segs, int nprob,
                                        long long maxn, double gamma, double adv, Ctl* ctl, cudaStream_t st) {
  return launch_alpha1d_batched_policy<FastMath>(flux, u, pitch, segs, nprob, maxn, gamma, adv, ctl, st);
}

int stage1d_batched_occupancy_fast(int flux, int tile) { return batched_occupancy_policy<FastMath>(flux, tile); }

__global__ void pack2d_kernel(const double* __restrict__ src, double* __restrict__ dst, long long nx, long long ny,
                              long long rowp, long long planep, int bxl, int bxh, int byl, int byh) {
  const long long W = nx + 2 * G, Hh = ny + 2 * G;
  const long long per = W * Hh;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < 4 * per;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / per);
    const long long k = idx - (long long)c * per;
    const long long py = k / W, px = k - py * W;
    long long x = px - G, y = py - G;
    bool fx = false, fy = false;
    if (x < 0 || x >= nx) x = ghost_source(x, nx, bxl, bxh, &fx);
    if (y < 0 || y >= ny) y = ghost_source(y, ny, byl, byh, &fy);
    double v = src[(c * ny + y) * nx + x];
    if ((fx && c == 1) || (fy && c == 2)) v = -v;  // reflective: normal momentum flips
    dst[c * planep + py * rowp + px] = v;
  }
}

__global__ void unpack2d_kernel(const double* __restrict__ src, double* __restrict__ dst, long long nx, long long ny,
                                long long rowp, long long planep) {
  const long long per = nx * ny;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < 4 * per;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / per);
    const long long k = idx - (long long)c * per;
    const long long y = k / nx, x = k - y * nx;
    dst[idx] = src[c * planep + (y + G) * rowp + x + G];
  }
}

cudaError_t launch_pack2d(const double* src, double* dst, long long nx, long long ny, long long rowp, long long planep,
                          int bxl, int bxh, int byl, int byh, cudaStream_t st) {
  pack2d_kernel<<<copy_grid(4 * (nx + 2 * G) * (ny + 2 * G)), 256, 0, st>>>(src, dst, nx, ny, rowp, planep, bxl, bxh,
                                                                            byl, byh);
  return cudaGetLastError();
}

cudaError_t launch_unpack2d(const double* src, double* dst, long long nx, long long ny, long long rowp,
                            long long planep, cudaStream_t st) {
  unpack2d_kernel<<<copy_grid(4 * nx * ny), 256, 0, st>>>(src, dst, nx, ny, rowp, planep);
  return cudaGetLastError();
}

cudaError_t prepare_stage2d_fast() { return prepare_stage2d_policy<FastMath>(); }

cudaError_t launch_stage2d_fast(int stage, const Stage2DArgs& a, cudaStream_t st) {
  return launch_stage2d_policy<FastMath>(stage, a, st);
}

cudaError_t launch_alpha2d_fast(const double* u, long long nx, long long ny, long long rowp, long long planep,
                                double gamma, double dx, double dy, Ctl* ctl, int slot, cudaStream_t st) {
  return launch_alpha2d_policy<FastMath>(u, nx, ny, rowp, planep, gamma, dx, dy, ctl, slot, st);
}

cudaError_t prepare_adj_fast() { return prepare_adj_policy<FastMath>(); }

cudaError_t launch_adj_stage_fast(const AdjArgs& a, int grid, int code, cudaStream_t st) {
  return launch_adj_stage_policy<FastMath>(a, grid, code, st);
}

cudaError_t launch_adj_argmax_fast(const double* uin, long long pitch, const BatchSeg* segs, int nprob,
                                     long long maxn, const double* alpha, double gamma, int* arg, cudaStream_t st) {
  return launch_adj_argmax_policy<FastMath>(uin, pitch, segs, nprob, maxn, alpha, gamma, arg, st);
}

// The reverse tile: 63 cells with three (interface, field) items per thread (64 threads), the
// fastest of the compiled codes on the adjoint workload, unless WT_ADJ_TILE names another (31,
// 2031, 63, 1063, 2063).  The gradients agree to rounding: the per-tile partial sums of the
// alpha and dt derivatives are added in another order.
int adj_tile_code() {
  if (const char* e = getenv("WT_ADJ_TILE")) {
    const int c = atoi(e);
    if (c == 31 || c == 2031 || c == 63 || c == 1063 || c == 2063) return c;
  }
  return 2063;
}

cudaError_t launch_adj_gather(const GatherArgs& a, int nprob, long long maxn, cudaStream_t st) {
  long long bx = (maxn + 255) / 256;
  if (bx > 64) bx = 64;
  adj_gather_kernel<<<dim3((unsigned)(bx < 1 ? 1 : bx), (unsigned)nprob), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adj_apply(const double* uin, long long pitch, const BatchSeg* segs, const int* tstart,
                             const int* tcount, const double* partial, const double* alpha, const double* dt,
                             const int* arg, double* ubar, long long ustride, double* dtbar, int final_stage,
                             double gamma, int nprob, cudaStream_t st) {
  adj_apply_kernel<<<(nprob + 3) / 4, 128, 0, st>>>(uin, pitch, segs, tstart, tcount, partial, alpha, dt, arg, ubar,
                                                    ustride, dtbar, final_stage, gamma, nprob);
  return cudaGetLastError();
}

cudaError_t launch_adj_record(const Ctl* ctl, int slot, double* alpha_out, double* dt_out, int nprob, cudaStream_t st) {
  adj_record_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(ctl, slot, alpha_out, dt_out, nprob);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Self-test of the bounded waits: a grid-counter wait on a word nobody increments, an
// mbarrier wait for bulk-copy bytes that never arrive (no copy is issued, so nothing is in
// flight when the block leaves), a grid-counter wait that is already satisfied, and the
// step-blocked kernel's mailbox waits: halo words whose step tag never arrives, alpha words
// that never carry the step's parity, and alpha words already published.
// ---------------------------------------------------------------------------------------
__global__ void selftest_wait_kernel(int which, unsigned long long* word, unsigned long long* mbox, long long limit,
                                     int* result) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ double s_a[32], s_b[32];
  bool ok = true;
  if (which == 0 || which == 2) {
    ok = grid_wait(word, which == 0 ? 1ull : 0ull, limit);
  } else if (which == 1) {
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      mbar_arrive_expect_tx(&bar, 16u);
    }
    __syncthreads();
    ok = __syncthreads_or(mbar_wait_bounded(&bar, 0u, limit) ? 0 : 1) == 0;
  } else if (which == 3) {
    // one periodic cell whose halo words (zeroed: tag 0) are awaited with tag 1
    ok = sb_mailbox_halo<1>(mbox, mbox + 1, 1, 1, -1, 1, 1, true, true, 1u, s_a, s_b, 16, limit);
  } else {
    // one CTA's alpha words: zeroed (parity 0) and awaited with parity 1, or first published
    // with parity 1 by this warp
    const unsigned long long pbit = 1ull << 63;
    if (which == 5 && threadIdx.x < 4) st_relaxed_u64(mbox + threadIdx.x, pbit | (unsigned long long)threadIdx.x);
    __syncwarp();
    unsigned long long mk[3], stv;
    ok = gather_alpha_words<3>(mbox, 1, pbit, limit, mk, stv) != 0;
    if (ok) ok = mk[0] == 0ull && mk[1] == 1ull && mk[2] == 2ull;  // the published values
  }
  if (threadIdx.x == 0) *result = ok ? WT_OK : WT_ERR_TIMEOUT;
}

cudaError_t launch_selftest_wait(int which, unsigned long long* word, unsigned long long* mbox, long long limit,
                                 int* result, cudaStream_t st) {
  selftest_wait_kernel<<<1, 32, 0, st>>>(which, word, mbox, limit, result);
  return cudaGetLastError();
}

}  // namespace wt
