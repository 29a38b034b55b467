// weno_theta_rhs_noalloc: L(u) for callers that cannot allocate device memory.
//
// Some callers have no way to hand the library a workspace: code that runs inside a
// region where a cudaMalloc is not allowed or would stall the device (a real-time loop
// that must not synchronise, a host program linked against this C ABI with no allocator
// of its own, a plug-in living under a host application's fixed memory budget).  For them
// this entry point keeps its scratch -- the control block and the padded copy of the state
// with its ghost cells -- in a fixed-size array of device memory that is part of the
// library image.  Every GPU that loads the library holds that array until the process
// exits.  The caller still passes the input u and the output L (both device memory).
//
// The array is shared by every call and keeps whatever the last call left in it; each call
// clears the part that must start at zero.  Calls whose GPU work overlaps in time (on
// different streams, or from different host threads) race on the array and give wrong
// results: serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "wt_launch.h"

namespace {

using namespace wt;

// Scratch capacity (WT_NOALLOC_SCRATCH_BYTES, 8 MiB): the control block plus m padded
// planes of pitch(n) = n + 6 rounded up to 32 doubles.
constexpr long long kScratchDoubles = WT_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr long long kCtlDoubles = 64;  // sizeof(Ctl) <= 512 bytes, keeps the planes 256-byte aligned
static_assert(sizeof(Ctl) <= kCtlDoubles * sizeof(double), "control block does not fit its slot");

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_setup_mu;
double* g_scratch_ptr[64] = {};  // device address of the array, per device

int set_error(int code, const char* msg) { return wt::set_last_error(code, msg); }

// largest n with m * pitch(n) <= capacity, pitch(n) = 32 * ceil((n + 6) / 32)
long long max_cells(int m) {
  const long long per_plane = (kScratchDoubles - kCtlDoubles) / m;
  return (per_plane / 32) * 32 - 2 * G;
}

// Device address of the scratch array on the current device, looked up once per device.
// The host-side name g_noalloc_scratch is only a stand-in and must never reach a kernel.
int scratch_for_device(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (dev < 0 || dev >= 64) return set_error(WT_ERR_CUDA, "device index out of range");
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return set_error(WT_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return WT_OK;
}

bool is_device_pointer(const void* p, int* dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *dev = a.device;
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int weno_theta_rhs_noalloc(const wt_problem* prob, const wt_grid* grid, const double* u, double* L, void* stream) {
  // the checks of weno_theta_rhs first, then the limits of this variant
  int rc = check_problem(prob);
  if (rc != WT_OK) return rc;
  if ((rc = check_grid_1d(prob, grid)) != WT_OK) return rc;
  if (!u || !L) return set_error(WT_ERR_ARG, "u and L must not be NULL");
  if (prob->flux == WT_FLUX_EULER2D)
    return set_error(WT_ERR_UNSUPPORTED, "weno_theta_rhs_noalloc supports the 1D fluxes only");
  const int m = prob->m;
  const long long n = grid->n[0];
  if (n > max_cells(m))
    return set_error(WT_ERR_ARG,
                     "n exceeds the built-in scratch array of WT_NOALLOC_SCRATCH_BYTES (at most 349498 cells for "
                     "Euler, 1048506 for a scalar flux); use weno_theta_rhs with a workspace");
  int dev_u = -1, dev_L = -1;
  if (!is_device_pointer(u, &dev_u) || !is_device_pointer(L, &dev_L) || dev_u != dev_L)
    return set_error(WT_ERR_ARG, "u and L must be device memory on the same GPU");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return set_error(WT_ERR_CUDA, "cudaGetDevice failed");
  if (cur != dev_u && cudaSetDevice(dev_u) != cudaSuccess) return set_error(WT_ERR_CUDA, "cudaSetDevice failed");
  double* base = nullptr;
  rc = scratch_for_device(dev_u, &base);
  if (rc == WT_OK) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Ctl* ctl = reinterpret_cast<Ctl*>(base);
    double* Un = base + kCtlDoubles;
    const long long pitch = ((n + 2 * G + 31) / 32) * 32;
    const double dx = (grid->hi[0] - grid->lo[0]) / (double)n;
    // the same arguments, tile and launches as weno_theta_rhs with a device workspace
    Stage1DArgs a = base_args(prob, n, dx, pitch, ctl);
    a.uin = Un;
    a.Lout = L;
    const bool strict = prob->mode == WT_MODE_STRICT;
    const int blo = prob->bc_lo[0], bhi = prob->bc_hi[0];
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), st);  // alpha slots and status start at zero
    if (e == cudaSuccess) e = launch_pack1d(u, n, Un, n, pitch, m, blo, bhi, 1, st);
    if (e == cudaSuccess)
      e = strict ? launch_alpha1d_strict(prob->flux, Un, n, pitch, prob->gamma, prob->adv_speed, ctl, 0, st)
                 : launch_alpha1d_fast(prob->flux, Un, n, pitch, prob->gamma, prob->adv_speed, ctl, 0, st);
    if (e == cudaSuccess)
      e = strict ? launch_stage1d_strict(prob->flux, STAGE_RHS, default_tile(prob->flux, n), a, st)
                 : launch_stage1d_fast(prob->flux, STAGE_RHS, default_tile(prob->flux, n), a, st);
    if (e != cudaSuccess) rc = set_error(WT_ERR_CUDA, cudaGetErrorString(e));
  }
  if (cur != dev_u) cudaSetDevice(cur);
  return rc;
}

}  // extern "C"
