// Internal interface between the C ABI (wt_api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "wt_device.cuh"

namespace wt {

enum { STAGE_RK1 = 0, STAGE_RK2 = 1, STAGE_RK3 = 2, STAGE_RHS = 3 };

// Arguments of one fused RHS + RK stage launch over a 1D grid.
struct Stage1DArgs {
  const double* uin;     // stage input, padded planes [m][pitch], cell j at j + G
  const double* un;      // u^n, padded (stages 2 and 3)
  double* uout;          // stage output, padded (stages)
  double* Lout;          // L(u) output [m][lout_stride] (RHS mode)
  long long n;           // cells
  long long pitch;       // plane stride of the padded arrays (doubles, multiple of 32)
  long long lout_stride;
  double dx, inv_dx;
  double gamma, adv_speed, eps, alpha_R;
  int bc_lo, bc_hi;
  Ctl* ctl;
  // the adjoint's recording forward pass only (else null): one record of kAdjRec doubles per
  // interface, slot gi + 1 for interface gi = -1 .. n-1
  double* rec;
};

// Record of one interface and stage for the adjoint's reverse pass: Roe's mean velocity and
// enthalpy (from which the policy rebuilds the eigenvectors bit for bit), the characteristic
// fluxes F_s = F+_s + F-_s of the three fields, and the branch flags of the six
// reconstructions as the bit pattern of a double: bit 2 (3 side + s) set if restricted (Eq.
// (be_res)), bit 2 (3 side + s) + 1 set if theta = 1 (Eq. (tau_we6)); side 0 = +, 1 = -.
constexpr int kAdjRec = 6;

// Arguments of the persistent kernel: the three stages of an RK step and the steps to take
struct PersistArgs {
  Stage1DArgs a[3];
  long long n_steps;
  // step-blocked kernel only, zeroed before each launch: the alpha mailbox
  // [3 stages][grid][4] and the halo mailbox (high and low 32-bit halves of u^{n+1} of
  // every cell, [m][pitch] each, the step's tag in the upper 32 bits of each word)
  unsigned long long* amb;
  unsigned long long* hmb_hi;
  unsigned long long* hmb_lo;
};

// One problem of a batch: padded storage at poff in the workspace planes, caller storage
// at uoff in the caller's packed planes.
struct BatchSeg {
  long long poff;
  long long uoff;
  long long n;
  double dx, inv_dx;
  int bc_lo, bc_hi;
};

// Arguments of one batched stage launch.
struct BatchArgs {
  const double* uin;       // plane bases [m][pitch]; problem p starts at segs[p].poff
  const double* un;
  double* uout;
  long long pitch;
  const BatchSeg* segs;
  Ctl* ctl;                // [nprob]
  const int2* tiles;       // work items: (problem, tile index); tile j0 = index * T
  int ntiles;
  double gamma, adv_speed, eps, alpha_R;
  double* rec;             // recording forward pass of the adjoint only (else null): records
  const long long* rec_off;  // [nprob] first interface slot of each problem in rec
};

// tile: a tile code, cells per tile + 1000 x (items per thread - 1): 31, 63, 127 (Euler; 63, 127
// scalar) with one (interface, field) item per thread, 1063 and 1127 (Euler) with two,
// 2127, 3127 and 5127 (Euler) with three, four and six
cudaError_t launch_stage1d_batched_strict(int flux, int stage, int tile, const BatchArgs& b, int grid, cudaStream_t st);
cudaError_t launch_stage1d_batched_fast(int flux, int stage, int tile, const BatchArgs& b, int grid, cudaStream_t st);
// the adjoint's recording forward stage (1D Euler, tile code 5127): also writes b.rec
cudaError_t launch_stage1d_batched_record_strict(int stage, const BatchArgs& b, int grid, cudaStream_t st);
cudaError_t launch_stage1d_batched_record_fast(int stage, const BatchArgs& b, int grid, cudaStream_t st);
// resident CTAs per SM of the batched stage kernel (occupancy), 0 on error
int stage1d_batched_occupancy_strict(int flux, int tile);
int stage1d_batched_occupancy_fast(int flux, int tile);
cudaError_t launch_alpha1d_batched_strict(int flux, const double* u, long long pitch, const BatchSeg* segs, int nprob,
                                          long long maxn, double gamma, double adv, Ctl* ctl, cudaStream_t st);
cudaError_t launch_alpha1d_batched_fast(int flux, const double* u, long long pitch, const BatchSeg* segs, int nprob,
                                        long long maxn, double gamma, double adv, Ctl* ctl, cudaStream_t st);
cudaError_t launch_pack1d_batched(const double* src, long long src_stride, double* dst, long long pitch,
                                  const BatchSeg* segs, int nprob, long long maxn, int m, int flip_comp, cudaStream_t st);
// skip_failed (may be null): leave out the problems whose control block records a failure
cudaError_t launch_unpack1d_batched(const double* src, long long pitch, double* dst, long long dst_stride,
                                    const BatchSeg* segs, int nprob, long long maxn, int m, cudaStream_t st,
                                    const Ctl* skip_failed = nullptr);
cudaError_t launch_gather_t(const Ctl* ctl, int nprob, double* t_out, cudaStream_t st);
cudaError_t launch_gather_status(const Ctl* ctl, int nprob, int* out, cudaStream_t st);

// Arguments of one fused 2D stage launch.  Padded planes: cell (x, y) at (y + G) * rowp + x + G.
struct Stage2DArgs {
  const double* uin;
  const double* un;
  double* uout;
  double* Lout;          // RHS mode: [4][ny][nx]
  long long nx, ny;
  long long rowp;        // padded row stride (even)
  long long planep;      // padded plane stride
  double dx, dy, inv_dx, inv_dy;
  double gamma, eps, alpha_R;
  double gravity;        // g of the source terms (0: none)
  int bcx_lo, bcx_hi, bcy_lo, bcy_hi;
  Ctl* ctl;
};

cudaError_t prepare_stage2d_strict();
cudaError_t prepare_stage2d_fast();
cudaError_t launch_stage2d_strict(int stage, const Stage2DArgs& a, cudaStream_t st);
cudaError_t launch_stage2d_fast(int stage, const Stage2DArgs& a, cudaStream_t st);
cudaError_t launch_alpha2d_strict(const double* u, long long nx, long long ny, long long rowp, long long planep,
                                  double gamma, double dx, double dy, Ctl* ctl, int slot, cudaStream_t st);
cudaError_t launch_alpha2d_fast(const double* u, long long nx, long long ny, long long rowp, long long planep,
                                double gamma, double dx, double dy, Ctl* ctl, int slot, cudaStream_t st);
cudaError_t launch_pack2d(const double* src, double* dst, long long nx, long long ny, long long rowp, long long planep,
                          int bxl, int bxh, int byl, int byh, cudaStream_t st);
cudaError_t launch_unpack2d(const double* src, double* dst, long long nx, long long ny, long long rowp,
                            long long planep, cudaStream_t st);

// ---- discrete adjoint (1D Euler) -----------------------------------------------------
struct AdjArgs {  // one reverse RK stage over a tile table
  const double* uin;        // padded stage input planes [3][pitch]
  long long pitch;
  const BatchSeg* segs;     // uoff = offset of the problem in the [nprob][3][n] adjoint arrays, stride n
  const int2* tiles;        // (problem, tile index), tile width T
  int ntiles;
  long long ustride;        // n: component stride of the adjoint arrays
  const double* ubar_out;   // adjoint of the stage output
  const double* alpha;      // [nprob][4]: alphas of the stage input
  const double* dt;         // [nprob]
  double cL;                // weight of dt L in the stage: 1, 1/4, 2/3
  double gamma, eps, alpha_R;
  const long long* goff;    // [nprob]: first interface slot of the problem in G (n + 1 slots)
  double* G;                // [slots][36]: per interface, 6 cells x (fbar[3], Ubar[3])
  double* partial;          // [ntiles][4]: d/d alpha_s (3) and d/d dt of the tile
  const double* rec;        // [slots][kAdjRec] the forward stage's records (slots as G)
};

struct GatherArgs {  // per-cell gather of the interface contributions
  const double* uin;        // padded stage input planes (for the flux Jacobians)
  long long pitch;
  const BatchSeg* segs;
  const long long* goff;
  const double* G;
  long long ustride;
  const double* x;          // ubar_out
  double* out;
  double a_self;
  int accumulate;
  double* acc;              // may be null
  double a_acc;
  double gamma;
};

cudaError_t prepare_adj_strict();
cudaError_t prepare_adj_fast();
// code: the reverse tile, cells + 1000 x (items per thread - 1) (adj_tile_code)
cudaError_t launch_adj_stage_strict(const AdjArgs& a, int grid, int code, cudaStream_t st);
cudaError_t launch_adj_stage_fast(const AdjArgs& a, int grid, int code, cudaStream_t st);
cudaError_t launch_adj_argmax_strict(const double* uin, long long pitch, const BatchSeg* segs, int nprob,
                                     long long maxn, const double* alpha, double gamma, int* arg, cudaStream_t st);
cudaError_t launch_adj_argmax_fast(const double* uin, long long pitch, const BatchSeg* segs, int nprob, long long maxn,
                                   const double* alpha, double gamma, int* arg, cudaStream_t st);
cudaError_t launch_adj_gather(const GatherArgs& a, int nprob, long long maxn, cudaStream_t st);
cudaError_t launch_adj_apply(const double* uin, long long pitch, const BatchSeg* segs, const int* tstart,
                             const int* tcount, const double* partial, const double* alpha, const double* dt,
                             const int* arg, double* ubar, long long ustride, double* dtbar, int final_stage,
                             double gamma, int nprob, cudaStream_t st);
cudaError_t launch_adj_record(const Ctl* ctl, int slot, double* alpha_out, double* dt_out, int nprob, cudaStream_t st);
int adj_tile_code();

cudaError_t launch_selftest_wait(int which, unsigned long long* word, unsigned long long* mbox, long long limit,
                                 int* result, cudaStream_t st);

// Records a message for wt_last_error() on the calling thread and returns code.
int set_last_error(int code, const char* msg);

// Argument checks of the C ABI (WT_OK, or the status with wt_last_error() set), and the
// launch defaults every 1D RHS evaluation uses, so that entry points sharing them launch the
// same kernel instance on the same arguments.
int check_problem(const wt_problem* p);
int check_grid_1d(const wt_problem* p, const wt_grid* g);  // 2D grids too, for WT_FLUX_EULER2D
int default_tile(int flux, long long n);                  // stage-kernel tile for n cells
Stage1DArgs base_args(const wt_problem* p, long long n, double dx, long long pitch, Ctl* ctl);

cudaError_t launch_persist1d_strict(int flux, int tile, const PersistArgs& p, int grid, cudaStream_t st);
cudaError_t launch_persist1d_fast(int flux, int tile, const PersistArgs& p, int grid, cudaStream_t st);
int persist1d_capacity_strict(int flux, int tile);
// tile of the step-blocked kernel: 27 cells (Euler: 3 x 40 interface items = 4 warps in stage
// 1), 51 cells (scalar fluxes: 64 items = 2 warps)
inline int stepblock1d_tile(int flux) { return flux == WT_FLUX_EULER1D ? 27 : 51; }
cudaError_t launch_stepblock1d_strict(int flux, const PersistArgs& p, int grid, cudaStream_t st);
cudaError_t launch_stepblock1d_fast(int flux, const PersistArgs& p, int grid, cudaStream_t st);
int stepblock1d_capacity_strict(int flux);
int stepblock1d_capacity_fast(int flux);
int persist1d_capacity_fast(int flux, int tile);
cudaError_t launch_stage1d_strict(int flux, int stage, int tile, const Stage1DArgs& a, cudaStream_t st);
cudaError_t launch_stage1d_fast(int flux, int stage, int tile, const Stage1DArgs& a, cudaStream_t st);
cudaError_t launch_alpha1d_strict(int flux, const double* u, long long n, long long pitch, double gamma, double adv,
                                  Ctl* ctl, int slot, cudaStream_t st);
cudaError_t launch_alpha1d_fast(int flux, const double* u, long long n, long long pitch, double gamma, double adv,
                                Ctl* ctl, int slot, cudaStream_t st);
cudaError_t launch_pack1d(const double* src, long long src_stride, double* dst, long long n, long long pitch, int m,
                          int bc_lo, int bc_hi, int flip_comp, cudaStream_t st);
cudaError_t launch_unpack1d(const double* src, long long pitch, double* dst, long long dst_stride, long long n, int m,
                            cudaStream_t st);

}  // namespace wt
