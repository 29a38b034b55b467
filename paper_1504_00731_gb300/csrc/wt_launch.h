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
};

// Records a message for wt_last_error() on the calling thread and returns code.
int set_last_error(int code, const char* msg);

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
