// Strict-arithmetic instantiations of the 1D kernels.  Built with -fmad=false: no operation
// is contracted, so every result equals a literal binary64 evaluation of the paper's formulas.
#include "wt_kernels.cuh"
#include "wt_kernels2d.cuh"
#include "wt_adjoint.cuh"
#include "wt_math_strict.cuh"

namespace wt {

cudaError_t launch_persist1d_strict(int flux, int tile, const PersistArgs& p, int grid, cudaStream_t st) {
  return launch_persist1d_policy<StrictMath>(flux, tile, p, grid, st);
}

int persist1d_capacity_strict(int flux, int tile) { return persist1d_capacity_policy<StrictMath>(flux, tile); }

cudaError_t launch_stepblock1d_strict(int flux, const PersistArgs& p, int grid, cudaStream_t st) {
  return launch_stepblock1d_policy<StrictMath>(flux, p, grid, st);
}

int stepblock1d_capacity_strict(int flux) { return stepblock1d_capacity_policy<StrictMath>(flux); }

cudaError_t launch_stage1d_strict(int flux, int stage, int tile, const Stage1DArgs& a, cudaStream_t st) {
  return launch_stage1d_policy<StrictMath>(flux, stage, tile, a, st);
}

cudaError_t launch_alpha1d_strict(int flux, const double* u, long long n, long long pitch, double gamma, double adv,
                                  Ctl* ctl, int slot, cudaStream_t st) {
  return launch_alpha1d_policy<StrictMath>(flux, u, n, pitch, gamma, adv, ctl, slot, st);
}

cudaError_t launch_stage1d_batched_strict(int flux, int stage, int tile, const BatchArgs& b, int grid, cudaStream_t st) {
  return launch_stage1d_batched_policy<StrictMath>(flux, stage, tile, b, grid, st);
}

cudaError_t launch_stage1d_batched_record_strict(int stage, const BatchArgs& b, int grid, cudaStream_t st) {
  return launch_stage1d_batched_record_policy<StrictMath>(stage, b, grid, st);
}

cudaError_t launch_alpha1d_batched_strict(int flux, const double* u, long long pitch, const BatchSeg* segs, int nprob,
                                        long long maxn, double gamma, double adv, Ctl* ctl, cudaStream_t st) {
  return launch_alpha1d_batched_policy<StrictMath>(flux, u, pitch, segs, nprob, maxn, gamma, adv, ctl, st);
}

int stage1d_batched_occupancy_strict(int flux, int tile) { return batched_occupancy_policy<StrictMath>(flux, tile); }

cudaError_t prepare_stage2d_strict() { return prepare_stage2d_policy<StrictMath>(); }

cudaError_t launch_stage2d_strict(int stage, const Stage2DArgs& a, cudaStream_t st) {
  return launch_stage2d_policy<StrictMath>(stage, a, st);
}

cudaError_t launch_alpha2d_strict(const double* u, long long nx, long long ny, long long rowp, long long planep,
                                double gamma, double dx, double dy, Ctl* ctl, int slot, cudaStream_t st) {
  return launch_alpha2d_policy<StrictMath>(u, nx, ny, rowp, planep, gamma, dx, dy, ctl, slot, st);
}

cudaError_t prepare_adj_strict() { return prepare_adj_policy<StrictMath>(); }

cudaError_t launch_adj_stage_strict(const AdjArgs& a, int grid, int code, cudaStream_t st) {
  return launch_adj_stage_policy<StrictMath>(a, grid, code, st);
}

cudaError_t launch_adj_argmax_strict(const double* uin, long long pitch, const BatchSeg* segs, int nprob,
                                     long long maxn, const double* alpha, double gamma, int* arg, cudaStream_t st) {
  return launch_adj_argmax_policy<StrictMath>(uin, pitch, segs, nprob, maxn, alpha, gamma, arg, st);
}

}  // namespace wt
