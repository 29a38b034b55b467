// C ABI of the WENO-theta library (include/weno_theta.h): argument checks, workspace
// layout, host <-> device staging, and the RK step loop replayed from a CUDA graph.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "wt_launch.h"

namespace {

using namespace wt;

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define WT_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(WT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

// Argument checks and launch defaults shared with the no-allocation entry point (wt_launch.h).
namespace wt {

int expected_m(int flux) {
  switch (flux) {
    case WT_FLUX_ADVECTION:
    case WT_FLUX_BURGERS: return 1;
    case WT_FLUX_EULER1D: return 3;
    case WT_FLUX_EULER2D: return 4;
  }
  return -1;
}

bool bc_ok(int b) { return b == WT_BC_PERIODIC || b == WT_BC_OUTFLOW || b == WT_BC_REFLECTIVE; }

int check_problem(const wt_problem* p) {
  if (!p) return fail(WT_ERR_ARG, "problem is NULL");
  if (expected_m(p->flux) < 0) return fail(WT_ERR_ARG, "unknown flux %d", p->flux);
  if (p->m != expected_m(p->flux)) return fail(WT_ERR_ARG, "m = %d does not match flux %d", p->m, p->flux);
  if (p->mode != WT_MODE_FAST && p->mode != WT_MODE_STRICT) return fail(WT_ERR_ARG, "unknown mode %d", p->mode);
  if (p->launch != WT_LAUNCH_AUTO && p->launch != WT_LAUNCH_STAGES) return fail(WT_ERR_ARG, "unknown launch %d", p->launch);
  if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return fail(WT_ERR_ARG, "eps must be positive");
  if (!(p->alpha_R >= 0.0)) return fail(WT_ERR_ARG, "alpha_R must be >= 0");
  if ((p->flux == WT_FLUX_EULER1D || p->flux == WT_FLUX_EULER2D) && !(p->gamma > 1.0))
    return fail(WT_ERR_ARG, "gamma must exceed 1");
  if (p->flux == WT_FLUX_ADVECTION && !std::isfinite(p->adv_speed)) return fail(WT_ERR_ARG, "adv_speed not finite");
  for (int d = 0; d < 2; ++d)
    if (!bc_ok(p->bc_lo[d]) || !bc_ok(p->bc_hi[d])) return fail(WT_ERR_ARG, "unknown boundary condition");
  if ((p->flux == WT_FLUX_ADVECTION || p->flux == WT_FLUX_BURGERS) &&
      (p->bc_lo[0] == WT_BC_REFLECTIVE || p->bc_hi[0] == WT_BC_REFLECTIVE))
    return fail(WT_ERR_UNSUPPORTED, "reflective boundaries are defined for the Euler equations only");
  if ((p->bc_lo[0] == WT_BC_PERIODIC) != (p->bc_hi[0] == WT_BC_PERIODIC))
    return fail(WT_ERR_ARG, "a periodic boundary must be periodic at both ends");
  if (!std::isfinite(p->gravity)) return fail(WT_ERR_ARG, "gravity not finite");
  if (p->gravity != 0.0 && p->flux != WT_FLUX_EULER2D)
    return fail(WT_ERR_UNSUPPORTED, "gravity source terms are defined for the 2D Euler equations only");
  return WT_OK;
}

int check_grid_2d(const wt_problem* p, const wt_grid* g) {
  if (g->ndim != 2) return fail(WT_ERR_ARG, "ndim must be 2 for 2D Euler");
  for (int d = 0; d < 2; ++d) {
    if (g->n[d] < G) return fail(WT_ERR_ARG, "n[%d] = %lld is below the minimum of %d cells", d, (long long)g->n[d], G);
    if (g->n[d] > (1LL << 20)) return fail(WT_ERR_ARG, "n[%d] too large", d);
    if (!(g->hi[d] > g->lo[d]) || !std::isfinite(g->hi[d] - g->lo[d])) return fail(WT_ERR_ARG, "need lo < hi");
    if ((p->bc_lo[d] == WT_BC_PERIODIC) != (p->bc_hi[d] == WT_BC_PERIODIC))
      return fail(WT_ERR_ARG, "a periodic boundary must be periodic at both ends");
  }
  return WT_OK;
}

int check_grid_1d(const wt_problem* p, const wt_grid* g) {
  if (!g) return fail(WT_ERR_ARG, "grid is NULL");
  if (g->reserved != 0) return fail(WT_ERR_ARG, "reserved field must be 0");
  if (p->flux == WT_FLUX_EULER2D) return check_grid_2d(p, g);
  if (g->ndim != 1) return fail(WT_ERR_ARG, "ndim must be 1 for a 1D flux");
  if (g->n[0] < G) return fail(WT_ERR_ARG, "n = %lld is below the minimum of %d cells", (long long)g->n[0], G);
  if (g->n[0] > (1LL << 40)) return fail(WT_ERR_ARG, "n too large");
  if (!(g->hi[0] > g->lo[0]) || !std::isfinite(g->hi[0] - g->lo[0])) return fail(WT_ERR_ARG, "need lo < hi");
  return WT_OK;
}

int default_tile(int flux, long long n) {
  if (flux == WT_FLUX_EULER1D) {
    // about one CTA per SM for short grids, larger tiles once the grid fills the GPU
    if (n <= 152LL * 31) return 31;
    if (n <= 152LL * 4 * 63) return 63;
    return 127;
  }
  return n <= 152LL * 2 * 63 ? 63 : 127;
}

Stage1DArgs base_args(const wt_problem* p, long long n, double dx, long long pitch, Ctl* ctl) {
  Stage1DArgs a;
  memset(&a, 0, sizeof a);
  a.n = n;
  a.pitch = pitch;
  a.lout_stride = n;
  a.dx = dx;
  a.inv_dx = 1.0 / dx;
  a.gamma = p->gamma;
  a.adv_speed = p->adv_speed;
  a.eps = p->eps;
  a.alpha_R = p->alpha_R;
  a.bc_lo = p->bc_lo[0];
  a.bc_hi = p->bc_hi[0];
  a.ctl = ctl;
  return a;
}

}  // namespace wt

namespace {

constexpr size_t kAlign = 256;
// the step-blocked kernel reads each CTA's alpha words as one aligned 32-byte record
static_assert(kAlign % 32 == 0, "workspace regions must start 32-byte aligned");
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// padded plane stride: n + 2G rounded up to 32 doubles (256 bytes)
inline long long plane_pitch(long long n) { return ((n + 2 * G + 31) / 32) * 32; }

// Most CTAs of a step-blocked launch (one per SM), and the alpha mailbox words they use
constexpr long long kStepBlockMaxCtas = 1024;
inline long long stepblock_mailbox_words(long long ctas) { return 3 * 4 * ctas; }

// 1D workspace: [Ctl][alpha mailbox][Un][U1][U2][staging m*n][staging m*n].  The step-blocked
// kernel keeps its stage values on chip and uses U1, U2 as its halo mailbox.
struct Layout1D {
  size_t ctl, amb, un, u1, u2, st_in, st_out, total;
  long long pitch;
  long long amb_ctas;  // CTAs the alpha mailbox has room for
};

Layout1D layout_1d(int m, long long n) {
  Layout1D L;
  L.pitch = plane_pitch(n);
  const size_t plane = (size_t)m * L.pitch * sizeof(double);
  const size_t stage = (size_t)m * n * sizeof(double);
  // the step-blocked tiles hold at least 27 cells
  L.amb_ctas = (n + 26) / 27 < kStepBlockMaxCtas ? (n + 26) / 27 : kStepBlockMaxCtas;
  size_t o = 0;
  L.ctl = o;
  o = align_up(o + sizeof(Ctl));
  L.amb = o;
  o = align_up(o + (size_t)stepblock_mailbox_words(L.amb_ctas) * sizeof(unsigned long long));
  L.un = o;
  o = align_up(o + plane);
  L.u1 = o;
  o = align_up(o + plane);
  L.u2 = o;
  o = align_up(o + plane);
  L.st_in = o;
  o = align_up(o + stage);
  L.st_out = o;
  o = align_up(o + stage);
  L.total = o;
  return L;
}

// Device of a pointer, and whether it is device-accessible memory (device or managed).
int pointer_info(const void* p, bool* is_device, int* device) {
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *is_device = false;
    *device = -1;
    return WT_OK;
  }
  *is_device = (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
  *device = attr.device;
  return WT_OK;
}

// Host memory the driver has page-locked (or registered): asynchronous copies from and to it
// overlap kernels; copies of pageable memory do not.
bool pinned_host(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeHost;
}

// Makes the workspace's device current for the duration of a call.
struct DeviceGuard {
  int old = -1;
  bool changed = false;
  int enter(int dev) {
    if (cudaGetDevice(&old) != cudaSuccess) return fail(WT_ERR_CUDA, "cudaGetDevice failed");
    if (dev >= 0 && dev != old) {
      if (cudaSetDevice(dev) != cudaSuccess) return fail(WT_ERR_CUDA, "cudaSetDevice(%d) failed", dev);
      changed = true;
    }
    return WT_OK;
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(old);
  }
};

int check_ws(void* ws, size_t ws_bytes, size_t need, int* device) {
  if (!ws) return fail(WT_ERR_WORKSPACE, "workspace is NULL");
  if ((reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0) return fail(WT_ERR_WORKSPACE, "workspace not 256-byte aligned");
  if (ws_bytes < need) return fail(WT_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", ws_bytes, need);
  bool dev;
  pointer_info(ws, &dev, device);
  if (!dev) return fail(WT_ERR_WORKSPACE, "workspace is not device memory");
  return WT_OK;
}

cudaError_t launch_stage(const wt_problem* p, int stage, int tile, const Stage1DArgs& a, cudaStream_t st) {
  return p->mode == WT_MODE_STRICT ? launch_stage1d_strict(p->flux, stage, tile, a, st)
                                   : launch_stage1d_fast(p->flux, stage, tile, a, st);
}

cudaError_t launch_alpha(const wt_problem* p, const double* u, long long n, long long pitch, Ctl* ctl, int slot,
                         cudaStream_t st) {
  return p->mode == WT_MODE_STRICT ? launch_alpha1d_strict(p->flux, u, n, pitch, p->gamma, p->adv_speed, ctl, slot, st)
                                   : launch_alpha1d_fast(p->flux, u, n, pitch, p->gamma, p->adv_speed, ctl, slot, st);
}

// Copies the caller's state (host or device) into the padded planes with ghost cells.
int stage_in(const double* u, bool u_dev, double* staging, int m, long long n, long long pitch, double* Un,
             int bc_lo, int bc_hi, cudaStream_t st) {
  const double* src = u;
  if (!u_dev) {
    WT_CUDA(cudaMemcpyAsync(staging, u, sizeof(double) * m * n, cudaMemcpyHostToDevice, st));
    src = staging;
  }
  WT_CUDA(launch_pack1d(src, n, Un, n, pitch, m, bc_lo, bc_hi, 1, st));
  return WT_OK;
}

// --- CUDA graph of one RK step (three fused stage launches), cached per argument set
struct GraphEntry {
  Stage1DArgs a[3];
  int flux, mode, tile, device, nsteps;
  cudaGraphExec_t exec;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
cudaStream_t g_capture_stream[64] = {};
cudaStream_t g_copy_stream[64][2] = {};  // per device: copies to the device, copies back

bool same_args(const Stage1DArgs& x, const Stage1DArgs& y) { return memcmp(&x, &y, sizeof x) == 0; }

int get_step_graph(const wt_problem* p, int device, int tile, int nsteps, const Stage1DArgs a[3],
                   cudaGraphExec_t* out) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (auto& e : g_graphs) {
    if (e.device == device && e.flux == p->flux && e.mode == p->mode && e.tile == tile && e.nsteps == nsteps &&
        same_args(e.a[0], a[0]) && same_args(e.a[1], a[1]) && same_args(e.a[2], a[2])) {
      *out = e.exec;
      return WT_OK;
    }
  }
  if (device < 0 || device >= 64) return fail(WT_ERR_CUDA, "device index %d out of range", device);
  cudaStream_t& cs = g_capture_stream[device];
  if (!cs) WT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  WT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < nsteps; ++k)
    for (int s = 0; s < 3 && le == cudaSuccess; ++s) le = launch_stage(p, s, tile, a[s], cs);
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(cs, &graph);
  if (le != cudaSuccess) return fail(WT_ERR_CUDA, "stage launch during capture: %s", cudaGetErrorString(le));
  if (ee != cudaSuccess) return fail(WT_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ee));
  cudaGraphExec_t exec = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(WT_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
  if (g_graphs.size() >= 16) {
    cudaGraphExecDestroy(g_graphs.front().exec);
    g_graphs.erase(g_graphs.begin());
  }
  GraphEntry e;
  e.a[0] = a[0];
  e.a[1] = a[1];
  e.a[2] = a[2];
  e.flux = p->flux;
  e.mode = p->mode;
  e.tile = tile;
  e.device = device;
  e.nsteps = nsteps;
  e.exec = exec;
  g_graphs.push_back(e);
  *out = exec;
  return WT_OK;
}

Ctl make_ctl(double cfl, double dt_fixed, double t_final) {
  Ctl h;
  memset(&h, 0, sizeof h);
  h.t = 0.0;
  h.t_final = t_final;
  h.cfl = cfl;
  h.dt_fixed = dt_fixed;
  h.active = 1;
  return h;
}


// --- batched stepping -------------------------------------------------------------------

// Candidates of the batched autotuner, as tile codes: cells per tile + 1000 x (items per thread
// - 1).  Euler: tiles of 31, 63 and 127 cells with one (interface, field) item per thread, 63
// and 127 cells with two, 127 cells with three, four and six (fewer threads, more work each).
int tile_candidates(int flux, int* out) {
  if (flux == WT_FLUX_EULER1D) {
    out[0] = 31;
    out[1] = 63;
    out[2] = 127;
    out[3] = 1063;
    out[4] = 1127;
    out[5] = 2127;
    out[6] = 3127;
    out[7] = 5127;
    return 8;
  }
  out[0] = 63;
  out[1] = 127;
  return 2;
}

struct BatchLayout {
  size_t ctl, segs, tiles, un, u1, u2, st_u, st_o, st_t, total;
  long long pitch;
  long long max_tiles;
};

BatchLayout layout_batched(int m, int nprob, long long pitch, long long max_tiles, long long total_cells) {
  BatchLayout L;
  L.pitch = pitch;
  L.max_tiles = max_tiles;
  const size_t plane = (size_t)m * pitch * sizeof(double);
  size_t o = 0;
  L.ctl = o;
  o = align_up(o + sizeof(Ctl) * (size_t)nprob);
  L.segs = o;
  o = align_up(o + sizeof(BatchSeg) * (size_t)nprob);
  L.tiles = o;
  o = align_up(o + sizeof(int2) * (size_t)max_tiles);
  L.un = o;
  o = align_up(o + plane);
  L.u1 = o;
  o = align_up(o + plane);
  L.u2 = o;
  o = align_up(o + plane);
  L.st_u = o;
  o = align_up(o + sizeof(double) * (size_t)m * total_cells);
  L.st_o = o;  // results of a pipelined host call (the input stays in st_u until the call ends)
  o = align_up(o + sizeof(double) * (size_t)m * total_cells);
  L.st_t = o;
  o = align_up(o + sizeof(double) * (size_t)nprob);
  L.total = o;
  return L;
}

// upper bounds used by wt_workspace_bytes when only the batch totals are known
long long batched_pitch_bound(long long cells, int nprob) { return ((cells + 8LL * nprob + 31) / 32) * 32; }
long long batched_tiles_bound(long long cells, int nprob) { return cells / 31 + nprob; }

std::vector<int2> make_tiles(const std::vector<BatchSeg>& segs, int code) {
  const int T = code % 1000;  // cells per tile of the tile code
  std::vector<int2> t;
  // largest problems first, so the tail of the persistent loop is made of short work
  std::vector<int> order(segs.size());
  for (size_t i = 0; i < segs.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return segs[a].n > segs[b].n; });
  for (int p : order) {
    const long long nt = (segs[p].n + T - 1) / T;
    for (long long k = 0; k < nt; ++k) t.push_back(make_int2(p, (int)k));
  }
  return t;
}

struct BatchGraph {
  BatchArgs a[3];
  int flux, mode, tile, grid, device;
  cudaGraphExec_t exec;
};
std::vector<BatchGraph> g_bgraphs;
struct TuneEntry {
  int flux, mode, nprob, device;
  long long total, pitch;
  unsigned long long mix;  // hash of the segments' lengths and boundaries
  int tile;
};

// FNV-1a over the segments' lengths and boundary conditions: batches of the same size but a
// different mix of lengths get their own autotuning
unsigned long long segment_mix(const std::vector<BatchSeg>& segs) {
  unsigned long long h = 1469598103934665603ull;
  auto mixin = [&](unsigned long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xffull;
      h *= 1099511628211ull;
    }
  };
  for (const BatchSeg& s : segs) {
    mixin((unsigned long long)s.n);
    mixin((unsigned long long)(s.bc_lo * 4 + s.bc_hi));
  }
  return h;
}
std::vector<TuneEntry> g_tuned;

int batched_grid_size(const wt_problem* p, int tile, long long ntiles, int device) {
  int occ = p->mode == WT_MODE_STRICT ? stage1d_batched_occupancy_strict(p->flux, tile)
                                      : stage1d_batched_occupancy_fast(p->flux, tile);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  long long g = (long long)(occ > 0 ? occ : 1) * (sms > 0 ? sms : 1);
  if (g > ntiles) g = ntiles;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_batched_stage(const wt_problem* p, int stage, int tile, const BatchArgs& b, int grid,
                                 cudaStream_t st) {
  return p->mode == WT_MODE_STRICT ? launch_stage1d_batched_strict(p->flux, stage, tile, b, grid, st)
                                   : launch_stage1d_batched_fast(p->flux, stage, tile, b, grid, st);
}

int get_batched_graph(const wt_problem* p, int device, int tile, int grid, const BatchArgs a[3], cudaGraphExec_t* out) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (auto& e : g_bgraphs) {
    if (e.device == device && e.flux == p->flux && e.mode == p->mode && e.tile == tile && e.grid == grid &&
        !memcmp(&e.a[0], &a[0], sizeof(BatchArgs)) && !memcmp(&e.a[1], &a[1], sizeof(BatchArgs)) &&
        !memcmp(&e.a[2], &a[2], sizeof(BatchArgs))) {
      *out = e.exec;
      return WT_OK;
    }
  }
  if (device < 0 || device >= 64) return fail(WT_ERR_CUDA, "device index %d out of range", device);
  cudaStream_t& cs = g_capture_stream[device];
  if (!cs) WT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  WT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int s = 0; s < 3 && le == cudaSuccess; ++s) le = launch_batched_stage(p, s, tile, a[s], grid, cs);
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(cs, &graph);
  if (le != cudaSuccess) return fail(WT_ERR_CUDA, "batched stage launch during capture: %s", cudaGetErrorString(le));
  if (ee != cudaSuccess) return fail(WT_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ee));
  cudaGraphExec_t exec = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(WT_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
  if (g_bgraphs.size() >= 8) {
    cudaGraphExecDestroy(g_bgraphs.front().exec);
    g_bgraphs.erase(g_bgraphs.begin());
  }
  BatchGraph e;
  memcpy(e.a, a, sizeof e.a);
  e.flux = p->flux;
  e.mode = p->mode;
  e.tile = tile;
  e.grid = grid;
  e.device = device;
  e.exec = exec;
  g_bgraphs.push_back(e);
  *out = exec;
  return WT_OK;
}


// --- 2D ------------------------------------------------------------------------------------

// 2D workspace: [Ctl][Un][U1][U2][staging 4*nx*ny][staging 4*nx*ny]; padded planes with row
// stride rowp = nx + 6 rounded up to even and plane stride (ny + 6) * rowp rounded to 32.
struct Layout2D {
  size_t ctl, un, u1, u2, st_in, st_out, total;
  long long rowp, planep;
};

Layout2D layout_2d(long long nx, long long ny) {
  Layout2D L;
  L.rowp = ((nx + 2 * G + 1) / 2) * 2;
  L.planep = (((ny + 2 * G) * L.rowp + 31) / 32) * 32;
  const size_t planes = (size_t)4 * L.planep * sizeof(double);
  const size_t stage = (size_t)4 * nx * ny * sizeof(double);
  size_t o = 0;
  L.ctl = o;
  o = align_up(o + sizeof(Ctl));
  L.un = o;
  o = align_up(o + planes);
  L.u1 = o;
  o = align_up(o + planes);
  L.u2 = o;
  o = align_up(o + planes);
  L.st_in = o;
  o = align_up(o + stage);
  L.st_out = o;
  o = align_up(o + stage);
  L.total = o;
  return L;
}

Stage2DArgs base_args_2d(const wt_problem* p, const wt_grid* g, const Layout2D& lay, Ctl* ctl) {
  Stage2DArgs a;
  memset(&a, 0, sizeof a);
  a.nx = g->n[0];
  a.ny = g->n[1];
  a.rowp = lay.rowp;
  a.planep = lay.planep;
  a.dx = (g->hi[0] - g->lo[0]) / (double)g->n[0];
  a.dy = (g->hi[1] - g->lo[1]) / (double)g->n[1];
  a.inv_dx = 1.0 / a.dx;
  a.inv_dy = 1.0 / a.dy;
  a.gamma = p->gamma;
  a.eps = p->eps;
  a.alpha_R = p->alpha_R;
  a.gravity = p->gravity;
  a.bcx_lo = p->bc_lo[0];
  a.bcx_hi = p->bc_hi[0];
  a.bcy_lo = p->bc_lo[1];
  a.bcy_hi = p->bc_hi[1];
  a.ctl = ctl;
  return a;
}

cudaError_t launch_stage2d(const wt_problem* p, int stage, const Stage2DArgs& a, cudaStream_t st) {
  return p->mode == WT_MODE_STRICT ? launch_stage2d_strict(stage, a, st) : launch_stage2d_fast(stage, a, st);
}

cudaError_t launch_alpha2d(const wt_problem* p, const Stage2DArgs& a, const double* u, cudaStream_t st) {
  return p->mode == WT_MODE_STRICT
             ? launch_alpha2d_strict(u, a.nx, a.ny, a.rowp, a.planep, a.gamma, a.dx, a.dy, a.ctl, 0, st)
             : launch_alpha2d_fast(u, a.nx, a.ny, a.rowp, a.planep, a.gamma, a.dx, a.dy, a.ctl, 0, st);
}

struct Graph2D {
  Stage2DArgs a[3];
  int mode, device;
  cudaGraphExec_t exec;
};
std::vector<Graph2D> g_graphs2d;

int get_step_graph_2d(const wt_problem* p, int device, const Stage2DArgs a[3], cudaGraphExec_t* out) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (auto& e : g_graphs2d)
    if (e.device == device && e.mode == p->mode && !memcmp(e.a, a, sizeof e.a)) {
      *out = e.exec;
      return WT_OK;
    }
  if (device < 0 || device >= 64) return fail(WT_ERR_CUDA, "device index %d out of range", device);
  cudaStream_t& cs = g_capture_stream[device];
  if (!cs) WT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  WT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int s = 0; s < 3 && le == cudaSuccess; ++s) le = launch_stage2d(p, s, a[s], cs);
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(cs, &graph);
  if (le != cudaSuccess) return fail(WT_ERR_CUDA, "2D stage launch during capture: %s", cudaGetErrorString(le));
  if (ee != cudaSuccess) return fail(WT_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ee));
  cudaGraphExec_t exec = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(WT_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
  if (g_graphs2d.size() >= 8) {
    cudaGraphExecDestroy(g_graphs2d.front().exec);
    g_graphs2d.erase(g_graphs2d.begin());
  }
  Graph2D e;
  memcpy(e.a, a, sizeof e.a);
  e.mode = p->mode;
  e.device = device;
  e.exec = exec;
  g_graphs2d.push_back(e);
  *out = exec;
  return WT_OK;
}

int rhs_2d(const wt_problem* prob, const wt_grid* grid, const double* u, double* L, void* ws, size_t ws_bytes,
           void* stream) {
  int rc;
  const Layout2D lay = layout_2d(grid->n[0], grid->n[1]);
  int dev;
  if ((rc = check_ws(ws, ws_bytes, lay.total, &dev)) != WT_OK) return rc;
  DeviceGuard guard;
  if ((rc = guard.enter(dev)) != WT_OK) return rc;
  WT_CUDA(prob->mode == WT_MODE_STRICT ? prepare_stage2d_strict() : prepare_stage2d_fast());
  bool u_dev, L_dev;
  int d_u, d_L;
  pointer_info(u, &u_dev, &d_u);
  pointer_info(L, &L_dev, &d_L);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  Ctl* ctl = reinterpret_cast<Ctl*>(w + lay.ctl);
  double* Un = reinterpret_cast<double*>(w + lay.un);
  double* st_in = reinterpret_cast<double*>(w + lay.st_in);
  double* st_out = reinterpret_cast<double*>(w + lay.st_out);
  const long long cells = grid->n[0] * grid->n[1];
  Stage2DArgs a = base_args_2d(prob, grid, lay, ctl);
  WT_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
  const double* src = u;
  if (!u_dev) {
    WT_CUDA(cudaMemcpyAsync(st_in, u, sizeof(double) * 4 * cells, cudaMemcpyHostToDevice, st));
    src = st_in;
  }
  WT_CUDA(launch_pack2d(src, Un, a.nx, a.ny, a.rowp, a.planep, a.bcx_lo, a.bcx_hi, a.bcy_lo, a.bcy_hi, st));
  WT_CUDA(launch_alpha2d(prob, a, Un, st));
  a.uin = Un;
  a.Lout = L_dev ? L : st_out;
  WT_CUDA(launch_stage2d(prob, STAGE_RHS, a, st));
  if (!L_dev) WT_CUDA(cudaMemcpyAsync(L, st_out, sizeof(double) * 4 * cells, cudaMemcpyDeviceToHost, st));
  if (!u_dev || !L_dev) {
    WT_CUDA(cudaStreamSynchronize(st));
    int status = 0;
    WT_CUDA(cudaMemcpy(&status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) return fail(status, "device reported status %d (non-finite state)", status);
  }
  return WT_OK;
}

int step_2d(const wt_problem* prob, const wt_grid* grid, double* u, double cfl, double dt_fixed, double t_final,
            int64_t max_steps, double* t_reached, int64_t* steps, void* ws, size_t ws_bytes, void* stream) {
  int rc;
  const Layout2D lay = layout_2d(grid->n[0], grid->n[1]);
  int dev;
  if ((rc = check_ws(ws, ws_bytes, lay.total, &dev)) != WT_OK) return rc;
  DeviceGuard guard;
  if ((rc = guard.enter(dev)) != WT_OK) return rc;
  WT_CUDA(prob->mode == WT_MODE_STRICT ? prepare_stage2d_strict() : prepare_stage2d_fast());
  bool u_dev;
  int d_u;
  pointer_info(u, &u_dev, &d_u);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  Ctl* ctl = reinterpret_cast<Ctl*>(w + lay.ctl);
  double* Un = reinterpret_cast<double*>(w + lay.un);
  double* U1 = reinterpret_cast<double*>(w + lay.u1);
  double* U2 = reinterpret_cast<double*>(w + lay.u2);
  double* st_in = reinterpret_cast<double*>(w + lay.st_in);
  const long long cells = grid->n[0] * grid->n[1];
  const Ctl h = make_ctl(cfl, dt_fixed, t_final);
  WT_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st));
  Stage2DArgs base = base_args_2d(prob, grid, lay, ctl);
  const double* src = u;
  if (!u_dev) {
    WT_CUDA(cudaMemcpyAsync(st_in, u, sizeof(double) * 4 * cells, cudaMemcpyHostToDevice, st));
    src = st_in;
  }
  WT_CUDA(launch_pack2d(src, Un, base.nx, base.ny, base.rowp, base.planep, base.bcx_lo, base.bcx_hi, base.bcy_lo,
                        base.bcy_hi, st));
  WT_CUDA(launch_alpha2d(prob, base, Un, st));
  Stage2DArgs a[3] = {base, base, base};
  a[0].uin = Un;
  a[0].uout = U1;
  a[1].uin = U1;
  a[1].un = Un;
  a[1].uout = U2;
  a[2].uin = U2;
  a[2].un = Un;
  a[2].uout = Un;
  cudaGraphExec_t exec;
  if (max_steps > 0 && (rc = get_step_graph_2d(prob, dev, a, &exec)) != WT_OK) return rc;
  Ctl hc;
  int64_t launched = 0;
  const bool bounded_time = std::isfinite(t_final);
  const int64_t chunk = bounded_time ? 16 : max_steps;
  while (launched < max_steps) {
    int64_t k = max_steps - launched;
    if (k > chunk) k = chunk;
    for (int64_t i = 0; i < k; ++i) WT_CUDA(cudaGraphLaunch(exec, st));
    launched += k;
    if (bounded_time) {
      WT_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      WT_CUDA(cudaStreamSynchronize(st));
      if (hc.status != 0 || !(hc.t < hc.t_final)) break;
    }
  }
  WT_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  WT_CUDA(cudaStreamSynchronize(st));
  if (hc.status != 0) return fail(hc.status, "device reported status %d after %lld steps", hc.status, hc.steps);
  if (u_dev) {
    WT_CUDA(launch_unpack2d(Un, u, base.nx, base.ny, base.rowp, base.planep, st));
  } else {
    WT_CUDA(launch_unpack2d(Un, st_in, base.nx, base.ny, base.rowp, base.planep, st));
    WT_CUDA(cudaMemcpyAsync(u, st_in, sizeof(double) * 4 * cells, cudaMemcpyDeviceToHost, st));
  }
  WT_CUDA(cudaStreamSynchronize(st));
  if (t_reached) *t_reached = hc.t;
  if (steps) *steps = hc.steps;
  return WT_OK;
}


// --- discrete adjoint ----------------------------------------------------------------------

struct AdjLayout {
  size_t ctl, segs, tiles_f, tiles_r, tstart, tcount, goff, un, u1, u2, ckpt, segu, rec_a, rec_dt, rec, v[4], G,
      partial, arg, dtbar, staging, total;
  long long pitch;
};

int adjoint_layout(const wt_problem* prob, const wt_grid* grid, int nprob, int64_t n_steps, int K, AdjLayout* out) {
  int rc;
  if ((rc = check_problem(prob)) != WT_OK) return rc;
  if (prob->flux != WT_FLUX_EULER1D) return fail(WT_ERR_UNSUPPORTED, "the adjoint is implemented for 1D Euler");
  if ((rc = check_grid_1d(prob, grid)) != WT_OK) return rc;
  if (nprob < 1 || nprob > 65535) return fail(WT_ERR_ARG, "nprob = %d outside 1..65535", nprob);
  if (n_steps < 0) return fail(WT_ERR_ARG, "n_steps must be >= 0");
  if (K < 1) return fail(WT_ERR_ARG, "checkpoint_every must be >= 1");
  const long long n = grid->n[0];
  if (n > (1LL << 30)) return fail(WT_ERR_ARG, "n too large for the adjoint");
  const long long padded = ((n + 2 * G + 1) / 2) * 2;
  const long long P = ((padded * nprob + 31) / 32) * 32;
  const long long S = (n_steps + K - 1) / K;
  const long long Kseg = std::min<long long>(K, std::max<long long>(n_steps, 1));
  const long long ntf = (long long)nprob * ((n + 126) / 127);
  const long long ntr = (long long)nprob * ((n + 30) / 31);
  AdjLayout L;
  L.pitch = P;
  const size_t plane = sizeof(double) * 3 * (size_t)P;
  const size_t vec = sizeof(double) * 3 * (size_t)n * nprob;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.ctl = take(sizeof(Ctl) * nprob);
  L.segs = take(sizeof(BatchSeg) * nprob);
  L.tiles_f = take(sizeof(int2) * ntf);
  L.tiles_r = take(sizeof(int2) * ntr);
  L.tstart = take(sizeof(int) * nprob);
  L.tcount = take(sizeof(int) * nprob);
  L.goff = take(sizeof(long long) * nprob);
  L.un = take(plane);
  L.u1 = take(plane);
  L.u2 = take(plane);
  L.ckpt = take(plane * (size_t)std::max<long long>(S, 1));
  L.segu = take(plane * 3 * (size_t)Kseg);
  L.rec_a = take(sizeof(double) * 12 * nprob * (size_t)Kseg);
  L.rec_dt = take(sizeof(double) * nprob * (size_t)Kseg);
  // the recording forward pass's per-interface records of every stage of a segment
  L.rec = take(sizeof(double) * kAdjRec * (size_t)(n + 1) * nprob * 3 * (size_t)Kseg);
  for (int i = 0; i < 4; ++i) L.v[i] = take(vec);
  L.G = take(sizeof(double) * 36 * (size_t)(n + 1) * nprob);
  L.partial = take(sizeof(double) * 4 * (size_t)ntr);
  L.arg = take(sizeof(int) * 4 * nprob);
  L.dtbar = take(sizeof(double) * nprob);
  L.staging = take(vec);
  L.total = o;
  *out = L;
  return WT_OK;
}

// Reads the control block back, reports a device-detected failure, copies u^n to the caller.
int finish_step_1d(Ctl* ctl, double* Un, const Layout1D& lay, double* u, bool u_dev, double* st_in, int m,
                          long long n, double* t_reached, int64_t* steps, cudaStream_t st) {
  Ctl hc;
  WT_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  WT_CUDA(cudaStreamSynchronize(st));
  if (hc.status != 0) return fail(hc.status, "device reported status %d after %lld steps", hc.status, hc.steps);
  if (u_dev) {
    WT_CUDA(launch_unpack1d(Un, lay.pitch, u, n, n, m, st));
  } else {
    WT_CUDA(launch_unpack1d(Un, lay.pitch, st_in, n, n, m, st));
    WT_CUDA(cudaMemcpyAsync(u, st_in, sizeof(double) * m * n, cudaMemcpyDeviceToHost, st));
  }
  WT_CUDA(cudaStreamSynchronize(st));
  if (t_reached) *t_reached = hc.t;
  if (steps) *steps = hc.steps;
  return WT_OK;
}

}  // namespace

int wt::set_last_error(int code, const char* msg) { return fail(code, "%s", msg); }

extern "C" {

const char* wt_last_error(void) { return g_err.c_str(); }

size_t wt_workspace_bytes(const wt_problem* prob, const wt_grid* grid, int64_t batch_cells, int32_t nprob) {
  if (check_problem(prob) != WT_OK) return 0;
  if (grid) {
    if (check_grid_1d(prob, grid) != WT_OK) return 0;
    if (grid->ndim == 2) return layout_2d(grid->n[0], grid->n[1]).total;
    return layout_1d(prob->m, grid->n[0]).total;
  }
  if (prob->flux == WT_FLUX_EULER2D) {
    fail(WT_ERR_UNSUPPORTED, "batched stepping supports the 1D fluxes only");
    return 0;
  }
  if (batch_cells < 3 || nprob < 1 || nprob > 65535) {
    fail(WT_ERR_ARG, "need batch_cells >= 3 and 1 <= nprob <= 65535");
    return 0;
  }
  return layout_batched(prob->m, nprob, batched_pitch_bound(batch_cells, nprob),
                        batched_tiles_bound(batch_cells, nprob), batch_cells)
      .total;
}

int weno_theta_rhs(const wt_problem* prob, const wt_grid* grid, const double* u, double* L, void* ws, size_t ws_bytes,
                   void* stream) {
  int rc;
  if ((rc = check_problem(prob)) != WT_OK) return rc;
  if ((rc = check_grid_1d(prob, grid)) != WT_OK) return rc;
  if (!u || !L) return fail(WT_ERR_ARG, "u and L must not be NULL");
  if (grid->ndim == 2) return rhs_2d(prob, grid, u, L, ws, ws_bytes, stream);
  const int m = prob->m;
  const long long n = grid->n[0];
  const Layout1D lay = layout_1d(m, n);
  int dev;
  if ((rc = check_ws(ws, ws_bytes, lay.total, &dev)) != WT_OK) return rc;
  DeviceGuard guard;
  if ((rc = guard.enter(dev)) != WT_OK) return rc;
  bool u_dev, L_dev;
  int d_u, d_L;
  pointer_info(u, &u_dev, &d_u);
  pointer_info(L, &L_dev, &d_L);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  Ctl* ctl = reinterpret_cast<Ctl*>(w + lay.ctl);
  double* Un = reinterpret_cast<double*>(w + lay.un);
  double* st_in = reinterpret_cast<double*>(w + lay.st_in);
  double* st_out = reinterpret_cast<double*>(w + lay.st_out);
  const double dx = (grid->hi[0] - grid->lo[0]) / (double)n;

  WT_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
  if ((rc = stage_in(u, u_dev, st_in, m, n, lay.pitch, Un, prob->bc_lo[0], prob->bc_hi[0], st)) != WT_OK) return rc;
  WT_CUDA(launch_alpha(prob, Un, n, lay.pitch, ctl, 0, st));
  Stage1DArgs a = base_args(prob, n, dx, lay.pitch, ctl);
  a.uin = Un;
  a.Lout = L_dev ? L : st_out;
  WT_CUDA(launch_stage(prob, STAGE_RHS, default_tile(prob->flux, n), a, st));
  if (!L_dev) {
    WT_CUDA(cudaMemcpyAsync(L, st_out, sizeof(double) * m * n, cudaMemcpyDeviceToHost, st));
  }
  if (!u_dev || !L_dev) {
    WT_CUDA(cudaStreamSynchronize(st));
    int status = 0;
    WT_CUDA(cudaMemcpy(&status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) return fail(status, "device reported status %d (non-physical state or NaN)", status);
  }
  return WT_OK;
}

int weno_theta_step(const wt_problem* prob, const wt_grid* grid, double* u, double cfl, double dt_fixed,
                    double t_final, int64_t max_steps, double* t_reached, int64_t* steps, void* ws, size_t ws_bytes,
                    void* stream) {
  int rc;
  if ((rc = check_problem(prob)) != WT_OK) return rc;
  if ((rc = check_grid_1d(prob, grid)) != WT_OK) return rc;
  if (!u) return fail(WT_ERR_ARG, "u must not be NULL");
  if (max_steps < 0) return fail(WT_ERR_ARG, "max_steps must be >= 0");
  if (!(dt_fixed > 0.0) && !(cfl > 0.0 && std::isfinite(cfl))) return fail(WT_ERR_ARG, "need cfl > 0 or dt_fixed > 0");
  if (!(t_final > 0.0) && !(t_final == 0.0)) return fail(WT_ERR_ARG, "t_final must be >= 0");
  if (grid->ndim == 2)
    return step_2d(prob, grid, u, cfl, dt_fixed, t_final, max_steps, t_reached, steps, ws, ws_bytes, stream);
  const int m = prob->m;
  const long long n = grid->n[0];
  const Layout1D lay = layout_1d(m, n);
  int dev;
  if ((rc = check_ws(ws, ws_bytes, lay.total, &dev)) != WT_OK) return rc;
  DeviceGuard guard;
  if ((rc = guard.enter(dev)) != WT_OK) return rc;
  bool u_dev;
  int d_u;
  pointer_info(u, &u_dev, &d_u);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  Ctl* ctl = reinterpret_cast<Ctl*>(w + lay.ctl);
  double* Un = reinterpret_cast<double*>(w + lay.un);
  double* U1 = reinterpret_cast<double*>(w + lay.u1);
  double* U2 = reinterpret_cast<double*>(w + lay.u2);
  double* st_in = reinterpret_cast<double*>(w + lay.st_in);
  const double dx = (grid->hi[0] - grid->lo[0]) / (double)n;
  const int tile = default_tile(prob->flux, n);

  const Ctl h = make_ctl(cfl, dt_fixed, t_final);
  WT_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st));
  if ((rc = stage_in(u, u_dev, st_in, m, n, lay.pitch, Un, prob->bc_lo[0], prob->bc_hi[0], st)) != WT_OK) return rc;
  WT_CUDA(launch_alpha(prob, Un, n, lay.pitch, ctl, 0, st));

  Stage1DArgs a[3];
  for (int s = 0; s < 3; ++s) a[s] = base_args(prob, n, dx, lay.pitch, ctl);
  a[0].uin = Un;
  a[0].uout = U1;
  a[1].uin = U1;
  a[1].un = Un;
  a[1].uout = U2;
  a[2].uin = U2;
  a[2].un = Un;
  a[2].uout = Un;
  Ctl hc;
  const bool bounded_time = std::isfinite(t_final);
  // Launch strategy, by how the grid's tiles fit on the device:
  //   at most one tile per SM: the step-blocked persistent kernel (one cooperative launch per
  //     chunk of steps, halo exchange once per RK step);
  //   all tiles co-resident: the persistent kernel with a halo exchange per stage;
  //   otherwise: CUDA graphs of the three stage kernels of an RK step.
  const bool strict = prob->mode == WT_MODE_STRICT;
  const int tsb = stepblock1d_tile(prob->flux);
  const long long nsb = (n + tsb - 1) / tsb;
  int nsm = 0;
  WT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const long long ntiles = (n + tile - 1) / tile;
  int kind = 0, pgrid = 0;
  if (max_steps > 0 && prob->launch == WT_LAUNCH_AUTO) {
    const int cap_sb = strict ? stepblock1d_capacity_strict(prob->flux) : stepblock1d_capacity_fast(prob->flux);
    if (nsb <= nsm && nsb <= cap_sb && nsb <= lay.amb_ctas) {
      kind = 2;
      pgrid = (int)nsb;
    } else {
      const int cap = strict ? persist1d_capacity_strict(prob->flux, tile) : persist1d_capacity_fast(prob->flux, tile);
      if (cap > 0 && ntiles <= cap) {
        kind = 1;
        pgrid = (int)ntiles;
      }
    }
  }
  if (kind != 0) {
    PersistArgs pa;
    for (int s = 0; s < 3; ++s) pa.a[s] = a[s];
    unsigned long long* amb = reinterpret_cast<unsigned long long*>(w + lay.amb);
    pa.amb = amb;
    pa.hmb_hi = reinterpret_cast<unsigned long long*>(U1);
    pa.hmb_lo = reinterpret_cast<unsigned long long*>(U2);
    constexpr int64_t kChunk = 4096;
    int64_t done = 0;
    while (done < max_steps) {
      int64_t k = max_steps - done;
      if (k > kChunk) k = kChunk;
      pa.n_steps = k;
      WT_CUDA(cudaMemsetAsync(&ctl->gbar, 0, sizeof(unsigned long long) + 4 * sizeof(unsigned int), st));
      if (kind == 2) {
        // the mailboxes start every launch with tag 0 and parity 0
        WT_CUDA(cudaMemsetAsync(amb, 0, (size_t)stepblock_mailbox_words(pgrid) * sizeof(unsigned long long), st));
        WT_CUDA(cudaMemsetAsync(U1, 0, (size_t)m * lay.pitch * sizeof(double), st));
        WT_CUDA(cudaMemsetAsync(U2, 0, (size_t)m * lay.pitch * sizeof(double), st));
        WT_CUDA(strict ? launch_stepblock1d_strict(prob->flux, pa, pgrid, st)
                       : launch_stepblock1d_fast(prob->flux, pa, pgrid, st));
      } else {
        WT_CUDA(strict ? launch_persist1d_strict(prob->flux, tile, pa, pgrid, st)
                       : launch_persist1d_fast(prob->flux, tile, pa, pgrid, st));
      }
      done += k;
      if (done < max_steps) {
        WT_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        WT_CUDA(cudaStreamSynchronize(st));
        if (hc.status != 0 || !(hc.t < hc.t_final)) break;
      }
    }
    return finish_step_1d(ctl, Un, lay, u, u_dev, st_in, m, n, t_reached, steps, st);
  }

  // RK steps replay from graphs of kGraphSteps steps (programmatic edges between their stage
  // launches) plus a one-step graph for the remainder
  constexpr int kGraphSteps = 8;
  cudaGraphExec_t exec1 = nullptr, execK = nullptr;
  if (max_steps > 0 && (rc = get_step_graph(prob, dev, tile, 1, a, &exec1)) != WT_OK) return rc;
  if (max_steps >= kGraphSteps && (rc = get_step_graph(prob, dev, tile, kGraphSteps, a, &execK)) != WT_OK) return rc;

  int64_t launched = 0;
  const int64_t chunk = bounded_time ? 64 : max_steps;
  while (launched < max_steps) {
    int64_t k = max_steps - launched;
    if (k > chunk) k = chunk;
    int64_t i = 0;
    for (; execK && i + kGraphSteps <= k; i += kGraphSteps) WT_CUDA(cudaGraphLaunch(execK, st));
    for (; i < k; ++i) WT_CUDA(cudaGraphLaunch(exec1, st));
    launched += k;
    if (bounded_time) {
      WT_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      WT_CUDA(cudaStreamSynchronize(st));
      if (hc.status != 0 || !(hc.t < hc.t_final)) break;
    }
  }
  return finish_step_1d(ctl, Un, lay, u, u_dev, st_in, m, n, t_reached, steps, st);
}

// Chunks of a pipelined host call (step_batched_pipelined): host arrays the driver has
// page-locked, segments laid out in the order of the problems (so each chunk's part of the
// caller's array is one range) and at least 2^22 cells per chunk; at most four.  1: none.
int pipeline_chunks(const wt_segment* segs, int nprob, long long cells, const double* u) {
  int k = (int)std::min<long long>(4, cells >> 22);
  if (k > nprob) k = nprob;
  if (k < 2) return 1;
  for (int p = 1; p < nprob; ++p)
    if (segs[p].offset < segs[p - 1].offset + segs[p - 1].n) return 1;
  return pinned_host(u) ? k : 1;
}

// Events of one call, destroyed on every way out
struct EventSet {
  std::vector<cudaEvent_t> e;
  cudaError_t make(int n) {
    e.assign(n, nullptr);
    for (auto& x : e) {
      const cudaError_t r = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  }
  ~EventSet() {
    for (auto x : e)
      if (x) cudaEventDestroy(x);
  }
};

// A batched call on host arrays in chunks of problems: per chunk, the copy of its part of the
// caller's array to the device (first copy stream); then, on the call's stream, the boundary
// fill, its alphas, the RK steps (a graph of the three stage launches over the chunk's part of
// the tile table) and the unpacking into the result buffer; then the copy back (second copy
// stream).  One chunk's copies overlap another's steps.  The chunks run the same kernels on
// subsets of problems that share nothing, so every problem's result is bit for bit that of one
// launch over all of them.  The input stays in st_u until the call ends: a failure restores
// it (all of u without a status array, the failed problems' parts with one).
int step_batched_pipelined(const wt_problem* prob, const wt_segment* segs, int nprob, double* u, int64_t total,
                           int64_t n_steps, double* t_out, bool t_dev, int32_t* s_out, bool s_dev,
                           const std::vector<BatchSeg>& hs, const std::vector<Ctl>& hctl, long long pitch, int tile,
                           int nchunk, int dev, Ctl* ctl, BatchSeg* dsegs, int2* dtiles, double* Un, double* U1,
                           double* U2, double* st_u, double* st_o, cudaStream_t st) {
  const int m = prob->m;
  long long cells = 0;
  for (const auto& h : hs) cells += h.n;
  // chunk boundaries: about equal cells, none empty
  std::vector<int> cb(1, 0);
  long long acc = 0;
  for (int p = 0; p + 1 < nprob; ++p) {
    acc += hs[p].n;
    if ((int)cb.size() < nchunk && acc * nchunk >= (long long)cb.size() * cells) cb.push_back(p + 1);
  }
  cb.push_back(nprob);
  const int K = (int)cb.size() - 1;
  // the chunks' tile tables one after another (problem indices local to the chunk)
  std::vector<int2> tl;
  std::vector<long long> tb(K + 1, 0);
  for (int c = 0; c < K; ++c) {
    const std::vector<BatchSeg> sub(hs.begin() + cb[c], hs.begin() + cb[c + 1]);
    const std::vector<int2> t = make_tiles(sub, tile);
    tl.insert(tl.end(), t.begin(), t.end());
    tb[c + 1] = (long long)tl.size();
  }
  WT_CUDA(cudaMemcpyAsync(dtiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, st));
  if (dev < 0 || dev >= 64) return fail(WT_ERR_CUDA, "device index %d out of range", dev);
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (int k = 0; k < 2; ++k)
      if (!g_copy_stream[dev][k]) WT_CUDA(cudaStreamCreateWithFlags(&g_copy_stream[dev][k], cudaStreamNonBlocking));
  }
  cudaStream_t sh = g_copy_stream[dev][0], sd = g_copy_stream[dev][1];
  // every control block at once (pageable memory: a copy per chunk could hold the host thread
  // until the stream reaches it, and with it the next chunk's copies)
  WT_CUDA(cudaMemcpyAsync(ctl, hctl.data(), sizeof(Ctl) * nprob, cudaMemcpyHostToDevice, st));
  EventSet ev;  // [0] start, [1] end, then per chunk: copied in, computed
  WT_CUDA(ev.make(2 + 2 * K));
  WT_CUDA(cudaEventRecord(ev.e[0], st));
  WT_CUDA(cudaStreamWaitEvent(sh, ev.e[0], 0));
  WT_CUDA(cudaStreamWaitEvent(sd, ev.e[0], 0));
  auto span = [&](int c, long long& s0, long long& len) {
    s0 = segs[cb[c]].offset;
    len = segs[cb[c + 1] - 1].offset + segs[cb[c + 1] - 1].n - s0;
  };
  for (int c = 0; c < K; ++c) {
    const int p0 = cb[c], np = cb[c + 1] - cb[c];
    cudaStream_t cs = st;
    long long s0, len;
    span(c, s0, len);
    for (int k = 0; k < m; ++k)
      WT_CUDA(cudaMemcpyAsync(st_u + k * total + s0, u + k * total + s0, sizeof(double) * len, cudaMemcpyHostToDevice,
                              sh));
    WT_CUDA(cudaEventRecord(ev.e[2 + 2 * c], sh));
    WT_CUDA(cudaStreamWaitEvent(cs, ev.e[2 + 2 * c], 0));
    long long maxn = 0;
    for (int p = p0; p < p0 + np; ++p) maxn = hs[p].n > maxn ? hs[p].n : maxn;
    WT_CUDA(launch_pack1d_batched(st_u, total, Un, pitch, dsegs + p0, np, maxn, m, 1, cs));
    WT_CUDA(prob->mode == WT_MODE_STRICT
                ? launch_alpha1d_batched_strict(prob->flux, Un, pitch, dsegs + p0, np, maxn, prob->gamma,
                                                prob->adv_speed, ctl + p0, cs)
                : launch_alpha1d_batched_fast(prob->flux, Un, pitch, dsegs + p0, np, maxn, prob->gamma,
                                              prob->adv_speed, ctl + p0, cs));
    BatchArgs a[3];
    for (int s2 = 0; s2 < 3; ++s2) {
      BatchArgs& b = a[s2];
      memset(&b, 0, sizeof b);
      b.pitch = pitch;
      b.segs = dsegs + p0;
      b.ctl = ctl + p0;
      b.tiles = dtiles + tb[c];
      b.ntiles = (int)(tb[c + 1] - tb[c]);
      b.gamma = prob->gamma;
      b.adv_speed = prob->adv_speed;
      b.eps = prob->eps;
      b.alpha_R = prob->alpha_R;
    }
    a[0].uin = Un;
    a[0].uout = U1;
    a[1].uin = U1;
    a[1].un = Un;
    a[1].uout = U2;
    a[2].uin = U2;
    a[2].un = Un;
    a[2].uout = Un;
    const int grid = batched_grid_size(prob, tile, tb[c + 1] - tb[c], dev);
    cudaGraphExec_t exec;
    int rc;
    if ((rc = get_batched_graph(prob, dev, tile, grid, a, &exec)) != WT_OK) return rc;
    for (int64_t i = 0; i < n_steps; ++i) WT_CUDA(cudaGraphLaunch(exec, cs));
    WT_CUDA(launch_unpack1d_batched(Un, pitch, st_o, total, dsegs + p0, np, maxn, m, cs));
    WT_CUDA(cudaEventRecord(ev.e[3 + 2 * c], cs));
    WT_CUDA(cudaStreamWaitEvent(sd, ev.e[3 + 2 * c], 0));
    for (int k = 0; k < m; ++k)
      WT_CUDA(cudaMemcpyAsync(u + k * total + s0, st_o + k * total + s0, sizeof(double) * len, cudaMemcpyDeviceToHost,
                              sd));
  }
  WT_CUDA(cudaEventRecord(ev.e[1], sd));
  WT_CUDA(cudaStreamWaitEvent(st, ev.e[1], 0));
  std::vector<Ctl> back(nprob);
  WT_CUDA(cudaMemcpyAsync(back.data(), ctl, sizeof(Ctl) * nprob, cudaMemcpyDeviceToHost, st));
  WT_CUDA(cudaStreamSynchronize(st));
  int nfail = 0, first = -1;
  for (int p = 0; p < nprob; ++p)
    if (back[p].status != 0 && nfail++ == 0) first = p;
  if (nfail > 0) {
    // put the input back: every chunk's part without a status array, else the failed problems'
    for (int c = 0; c < K; ++c) {
      long long s0, len;
      span(c, s0, len);
      for (int p = cb[c]; p < cb[c + 1]; ++p) {
        if (s_out && back[p].status == 0) continue;
        const long long o = s_out ? segs[p].offset : s0, n = s_out ? segs[p].n : len;
        for (int k = 0; k < m; ++k)
          WT_CUDA(cudaMemcpyAsync(u + k * total + o, st_u + k * total + o, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                  st));
        if (!s_out) break;
      }
    }
    WT_CUDA(cudaStreamSynchronize(st));
    if (!s_out)
      return fail(back[first].status, "problem %d: device reported status %d after %lld steps (%d problems failed)",
                  first, back[first].status, back[first].steps, nfail);
  }
  if (t_out) {
    if (t_dev) {
      WT_CUDA(launch_gather_t(ctl, nprob, t_out, st));
    } else {
      for (int p = 0; p < nprob; ++p) t_out[p] = back[p].t;
    }
  }
  if (s_out) {
    if (s_dev) {
      WT_CUDA(launch_gather_status(ctl, nprob, s_out, st));
    } else {
      for (int p = 0; p < nprob; ++p) s_out[p] = back[p].status;
    }
  }
  WT_CUDA(cudaStreamSynchronize(st));
  if (nfail > 0) fail(WT_OK, "%d of %d problems failed (first: problem %d, status %d); see status_per_problem", nfail,
                      nprob, first, back[first].status);
  return WT_OK;
}

int weno_theta_step_batched(const wt_problem* prob, const wt_segment* segs, int32_t nprob, double* u_packed,
                            int64_t total, double cfl, int64_t n_steps, double* t_per_problem,
                            int32_t* status_per_problem, void* ws, size_t ws_bytes, void* stream) {
  int rc;
  if ((rc = check_problem(prob)) != WT_OK) return rc;
  if (prob->flux == WT_FLUX_EULER2D) return fail(WT_ERR_UNSUPPORTED, "batched stepping supports the 1D fluxes only");
  if (!segs || !u_packed) return fail(WT_ERR_ARG, "segs and u_packed must not be NULL");
  if (nprob < 1 || nprob > 65535) return fail(WT_ERR_ARG, "nprob = %d outside 1..65535", nprob);
  if (total < 3) return fail(WT_ERR_ARG, "total must be >= 3");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(WT_ERR_ARG, "need cfl > 0");
  if (n_steps < 0) return fail(WT_ERR_ARG, "n_steps must be >= 0");
  const int m = prob->m;
  // segments: validate, order by offset to reject overlaps, lay out the padded planes
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return segs[a].offset < segs[b].offset; });
  for (int k = 0; k < nprob; ++k) {
    const wt_segment& sg = segs[order[k]];
    if (sg.n < G) return fail(WT_ERR_ARG, "segment %d: n = %lld below 3", order[k], (long long)sg.n);
    if (sg.offset < 0 || sg.offset + sg.n > total) return fail(WT_ERR_ARG, "segment %d outside [0, total)", order[k]);
    if (k > 0) {
      const wt_segment& pv = segs[order[k - 1]];
      if (pv.offset + pv.n > sg.offset) return fail(WT_ERR_ARG, "segments %d and %d overlap", order[k - 1], order[k]);
    }
    if (!(sg.hi > sg.lo)) return fail(WT_ERR_ARG, "segment %d: need lo < hi", order[k]);
    if (!bc_ok(sg.bc_lo) || !bc_ok(sg.bc_hi)) return fail(WT_ERR_ARG, "segment %d: unknown boundary", order[k]);
    if ((sg.bc_lo == WT_BC_PERIODIC) != (sg.bc_hi == WT_BC_PERIODIC))
      return fail(WT_ERR_ARG, "segment %d: periodic at one end only", order[k]);
    if (m == 1 && (sg.bc_lo == WT_BC_REFLECTIVE || sg.bc_hi == WT_BC_REFLECTIVE))
      return fail(WT_ERR_UNSUPPORTED, "reflective boundaries are defined for the Euler equations only");
  }
  std::vector<BatchSeg> hs(nprob);
  long long poff = 0, maxn = 0, cells = 0;
  for (int p = 0; p < nprob; ++p) {
    const wt_segment& sg = segs[p];
    hs[p].poff = poff;
    hs[p].uoff = sg.offset;
    hs[p].n = sg.n;
    hs[p].dx = (sg.hi - sg.lo) / (double)sg.n;
    hs[p].inv_dx = 1.0 / hs[p].dx;
    hs[p].bc_lo = sg.bc_lo;
    hs[p].bc_hi = sg.bc_hi;
    poff += ((sg.n + 2 * G + 1) / 2) * 2;  // even: every problem starts 16-byte aligned
    maxn = sg.n > maxn ? sg.n : maxn;
    cells += sg.n;
  }
  const long long pitch = ((poff + 31) / 32) * 32;
  int cand[8];
  const int ncand = tile_candidates(prob->flux, cand);
  long long max_tiles = 0;
  for (int p = 0; p < nprob; ++p) max_tiles += (hs[p].n + cand[0] - 1) / cand[0];
  const BatchLayout lay = layout_batched(m, nprob, pitch, max_tiles, total);
  int dev;
  if ((rc = check_ws(ws, ws_bytes, lay.total, &dev)) != WT_OK) return rc;
  DeviceGuard guard;
  if ((rc = guard.enter(dev)) != WT_OK) return rc;
  bool u_dev, t_dev = false, s_dev = false;
  int d_u, d_t, d_s;
  pointer_info(u_packed, &u_dev, &d_u);
  if (t_per_problem) pointer_info(t_per_problem, &t_dev, &d_t);
  if (status_per_problem) pointer_info(status_per_problem, &s_dev, &d_s);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  Ctl* ctl = reinterpret_cast<Ctl*>(w + lay.ctl);
  BatchSeg* dsegs = reinterpret_cast<BatchSeg*>(w + lay.segs);
  int2* dtiles = reinterpret_cast<int2*>(w + lay.tiles);
  double* Un = reinterpret_cast<double*>(w + lay.un);
  double* U1 = reinterpret_cast<double*>(w + lay.u1);
  double* U2 = reinterpret_cast<double*>(w + lay.u2);
  double* st_u = reinterpret_cast<double*>(w + lay.st_u);

  auto args_for = [&](int ntiles) {
    BatchArgs b;
    memset(&b, 0, sizeof b);
    b.pitch = pitch;
    b.segs = dsegs;
    b.ctl = ctl;
    b.tiles = dtiles;
    b.ntiles = ntiles;
    b.gamma = prob->gamma;
    b.adv_speed = prob->adv_speed;
    b.eps = prob->eps;
    b.alpha_R = prob->alpha_R;
    return b;
  };

  // ---- tile size: autotuned once per batch shape (timed RK stage 1 per candidate)
  int tile = -1;
  const unsigned long long mix = segment_mix(hs);
  // WT_BATCHED_TILE fixes the candidate (tests; callers that tuned offline)
  if (const char* forced = getenv("WT_BATCHED_TILE")) {
    const int code = atoi(forced);
    for (int ci = 0; ci < ncand; ++ci)
      if (cand[ci] == code) tile = code;
    if (tile < 0) return fail(WT_ERR_ARG, "WT_BATCHED_TILE=%s is not a candidate for this flux", forced);
  }
  if (tile < 0) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto& e : g_tuned)
      if (e.flux == prob->flux && e.mode == prob->mode && e.nprob == nprob && e.device == dev && e.total == total &&
          e.pitch == pitch && e.mix == mix)
        tile = e.tile;
  }

  std::vector<Ctl> hctl(nprob, make_ctl(cfl, 0.0, INFINITY));
  WT_CUDA(cudaMemcpyAsync(dsegs, hs.data(), sizeof(BatchSeg) * nprob, cudaMemcpyHostToDevice, st));
  double* st_o = reinterpret_cast<double*>(w + lay.st_o);
  const int nchunk = (!u_dev && tile >= 0 && n_steps > 0) ? pipeline_chunks(segs, nprob, cells, u_packed) : 1;
  if (nchunk > 1)
    return step_batched_pipelined(prob, segs, nprob, u_packed, total, n_steps, t_per_problem, t_dev,
                                  status_per_problem, s_dev, hs, hctl, pitch, tile, nchunk, dev, ctl, dsegs, dtiles,
                                  Un, U1, U2, st_u, st_o, st);
  const double* src = u_packed;
  if (!u_dev) {
    WT_CUDA(cudaMemcpyAsync(st_u, u_packed, sizeof(double) * m * total, cudaMemcpyHostToDevice, st));
    src = st_u;
  }
  WT_CUDA(launch_pack1d_batched(src, total, Un, pitch, dsegs, nprob, maxn, m, 1, st));
  auto init_ctl = [&]() -> int {
    WT_CUDA(cudaMemcpyAsync(ctl, hctl.data(), sizeof(Ctl) * nprob, cudaMemcpyHostToDevice, st));
    WT_CUDA(prob->mode == WT_MODE_STRICT
                ? launch_alpha1d_batched_strict(prob->flux, Un, pitch, dsegs, nprob, maxn, prob->gamma,
                                                prob->adv_speed, ctl, st)
                : launch_alpha1d_batched_fast(prob->flux, Un, pitch, dsegs, nprob, maxn, prob->gamma,
                                              prob->adv_speed, ctl, st));
    return WT_OK;
  };
  if ((rc = init_ctl()) != WT_OK) return rc;

  if (tile < 0 && n_steps > 0) {
    cudaEvent_t e0, e1;
    WT_CUDA(cudaEventCreate(&e0));
    WT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int ci = 0; ci < ncand; ++ci) {
      std::vector<int2> tl = make_tiles(hs, cand[ci]);
      WT_CUDA(cudaMemcpyAsync(dtiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, st));
      BatchArgs b = args_for((int)tl.size());
      b.uin = Un;
      b.uout = U1;
      const int grid = batched_grid_size(prob, cand[ci], (long long)tl.size(), dev);
      WT_CUDA(launch_batched_stage(prob, STAGE_RK1, cand[ci], b, grid, st));
      WT_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < 2; ++r) WT_CUDA(launch_batched_stage(prob, STAGE_RK1, cand[ci], b, grid, st));
      WT_CUDA(cudaEventRecord(e1, st));
      WT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      WT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        tile = cand[ci];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
      std::lock_guard<std::mutex> lk(g_graph_mu);
      if (g_tuned.size() >= 256) g_tuned.erase(g_tuned.begin());
      g_tuned.push_back(TuneEntry{prob->flux, prob->mode, nprob, dev, total, pitch, mix, tile});
    }
    if ((rc = init_ctl()) != WT_OK) return rc;  // the trial launches touched the alpha slots
  }
  if (tile < 0) tile = cand[ncand - 1];

  std::vector<int2> tl = make_tiles(hs, tile);
  WT_CUDA(cudaMemcpyAsync(dtiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, st));
  const int grid = batched_grid_size(prob, tile, (long long)tl.size(), dev);
  BatchArgs a[3];
  for (int s2 = 0; s2 < 3; ++s2) a[s2] = args_for((int)tl.size());
  a[0].uin = Un;
  a[0].uout = U1;
  a[1].uin = U1;
  a[1].un = Un;
  a[1].uout = U2;
  a[2].uin = U2;
  a[2].un = Un;
  a[2].uout = Un;
  if (n_steps > 0) {
    cudaGraphExec_t exec;
    if ((rc = get_batched_graph(prob, dev, tile, grid, a, &exec)) != WT_OK) return rc;
    for (int64_t i = 0; i < n_steps; ++i) WT_CUDA(cudaGraphLaunch(exec, st));
  }
  std::vector<Ctl> back(nprob);
  WT_CUDA(cudaMemcpyAsync(back.data(), ctl, sizeof(Ctl) * nprob, cudaMemcpyDeviceToHost, st));
  WT_CUDA(cudaStreamSynchronize(st));
  int nfail = 0, first = -1;
  for (int p = 0; p < nprob; ++p)
    if (back[p].status != 0 && nfail++ == 0) first = p;
  // Without a status array one failure fails the call (and u is untouched).  With one, each
  // problem's status goes there: the problems that succeeded are written back, the others keep
  // their input state.
  if (nfail > 0 && !status_per_problem)
    return fail(back[first].status, "problem %d: device reported status %d after %lld steps (%d problems failed)",
                first, back[first].status, back[first].steps, nfail);
  const Ctl* skip = nfail > 0 ? ctl : nullptr;
  if (u_dev) {
    WT_CUDA(launch_unpack1d_batched(Un, pitch, u_packed, total, dsegs, nprob, maxn, m, st, skip));
  } else {
    // st_u still holds the caller's input, so skipped problems copy back unchanged
    WT_CUDA(launch_unpack1d_batched(Un, pitch, st_u, total, dsegs, nprob, maxn, m, st, skip));
    WT_CUDA(cudaMemcpyAsync(u_packed, st_u, sizeof(double) * m * total, cudaMemcpyDeviceToHost, st));
  }
  if (t_per_problem) {
    if (t_dev) {
      WT_CUDA(launch_gather_t(ctl, nprob, t_per_problem, st));
    } else {
      for (int p = 0; p < nprob; ++p) t_per_problem[p] = back[p].t;
    }
  }
  if (status_per_problem) {
    if (s_dev) {
      WT_CUDA(launch_gather_status(ctl, nprob, status_per_problem, st));
    } else {
      for (int p = 0; p < nprob; ++p) status_per_problem[p] = back[p].status;
    }
  }
  WT_CUDA(cudaStreamSynchronize(st));
  if (nfail > 0) fail(WT_OK, "%d of %d problems failed (first: problem %d, status %d); see status_per_problem", nfail,
                      nprob, first, back[first].status);
  return WT_OK;
}

size_t wt_adjoint_workspace_bytes(const wt_problem* prob, const wt_grid* grid, int32_t nprob, int64_t n_steps,
                                  int32_t checkpoint_every) {
  AdjLayout L;
  if (adjoint_layout(prob, grid, nprob, n_steps, checkpoint_every, &L) != WT_OK) return 0;
  return L.total;
}

int weno_theta_adjoint(const wt_problem* prob, const wt_grid* grid, int32_t nprob, const double* u0, double cfl,
                       int64_t n_steps, int32_t checkpoint_every, const double* dJ_duT, double* dJ_du0, double* uT,
                       void* ws, size_t ws_bytes, void* stream) {
  int rc;
  AdjLayout lay;
  if ((rc = adjoint_layout(prob, grid, nprob, n_steps, checkpoint_every, &lay)) != WT_OK) return rc;
  if (!u0 || !dJ_duT || !dJ_du0) return fail(WT_ERR_ARG, "u0, dJ_duT and dJ_du0 must not be NULL");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(WT_ERR_ARG, "need cfl > 0");
  int dev;
  if ((rc = check_ws(ws, ws_bytes, lay.total, &dev)) != WT_OK) return rc;
  DeviceGuard guard;
  if ((rc = guard.enter(dev)) != WT_OK) return rc;
  const bool strict = prob->mode == WT_MODE_STRICT;
  WT_CUDA(strict ? prepare_adj_strict() : prepare_adj_fast());
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long n = grid->n[0];
  const long long P = lay.pitch;
  const size_t plane_bytes = sizeof(double) * 3 * (size_t)P;
  const size_t vec_bytes = sizeof(double) * 3 * (size_t)n * nprob;
  char* w = static_cast<char*>(ws);
  Ctl* ctl = reinterpret_cast<Ctl*>(w + lay.ctl);
  BatchSeg* dsegs = reinterpret_cast<BatchSeg*>(w + lay.segs);
  int2* tiles_f = reinterpret_cast<int2*>(w + lay.tiles_f);
  int2* tiles_r = reinterpret_cast<int2*>(w + lay.tiles_r);
  int* tstart = reinterpret_cast<int*>(w + lay.tstart);
  int* tcount = reinterpret_cast<int*>(w + lay.tcount);
  long long* goff = reinterpret_cast<long long*>(w + lay.goff);
  double* Un = reinterpret_cast<double*>(w + lay.un);
  double* U1 = reinterpret_cast<double*>(w + lay.u1);
  double* U2 = reinterpret_cast<double*>(w + lay.u2);
  double* ckpt = reinterpret_cast<double*>(w + lay.ckpt);
  double* segU = reinterpret_cast<double*>(w + lay.segu);
  double* rec_a = reinterpret_cast<double*>(w + lay.rec_a);
  double* rec_dt = reinterpret_cast<double*>(w + lay.rec_dt);
  double* vX = reinterpret_cast<double*>(w + lay.v[0]);
  double* vY = reinterpret_cast<double*>(w + lay.v[1]);
  double* vW = reinterpret_cast<double*>(w + lay.v[2]);
  double* vZ = reinterpret_cast<double*>(w + lay.v[3]);
  double* Gbuf = reinterpret_cast<double*>(w + lay.G);
  double* recbuf = reinterpret_cast<double*>(w + lay.rec);
  const size_t rec_stage = (size_t)kAdjRec * (size_t)(n + 1) * nprob;  // doubles per stage's records
  auto recs = [&](int64_t k, int s) { return recbuf + ((size_t)k * 3 + s) * rec_stage; };
  double* partial = reinterpret_cast<double*>(w + lay.partial);
  int* arg = reinterpret_cast<int*>(w + lay.arg);
  double* dtbar = reinterpret_cast<double*>(w + lay.dtbar);
  double* stage_buf = reinterpret_cast<double*>(w + lay.staging);
  auto segu = [&](int64_t k, int s) { return segU + ((size_t)k * 3 + s) * 3 * (size_t)P; };

  // ---- problems, tiles (forward T = 127, reverse T from the reverse tile code, problem-major)
  const int adj_code = adj_tile_code();
  const int Tr = adj_code % 1000;
  std::vector<BatchSeg> hs(nprob);
  std::vector<long long> hgoff(nprob);
  std::vector<int> hts(nprob), htc(nprob);
  std::vector<int2> tf, tr;
  const long long padded = ((n + 2 * G + 1) / 2) * 2;
  for (int p = 0; p < nprob; ++p) {
    hs[p].poff = p * padded;
    hs[p].uoff = (long long)p * 3 * n;
    hs[p].n = n;
    hs[p].dx = (grid->hi[0] - grid->lo[0]) / (double)n;
    hs[p].inv_dx = 1.0 / hs[p].dx;
    hs[p].bc_lo = prob->bc_lo[0];
    hs[p].bc_hi = prob->bc_hi[0];
    hgoff[p] = (long long)p * (n + 1);
    for (long long k = 0; k < (n + 126) / 127; ++k) tf.push_back(make_int2(p, (int)k));
    hts[p] = (int)tr.size();
    for (long long k = 0; k < (n + Tr - 1) / Tr; ++k) tr.push_back(make_int2(p, (int)k));
    htc[p] = (int)tr.size() - hts[p];
  }
  WT_CUDA(cudaMemcpyAsync(dsegs, hs.data(), sizeof(BatchSeg) * nprob, cudaMemcpyHostToDevice, st));
  WT_CUDA(cudaMemcpyAsync(goff, hgoff.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice, st));
  WT_CUDA(cudaMemcpyAsync(tstart, hts.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, st));
  WT_CUDA(cudaMemcpyAsync(tcount, htc.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, st));
  WT_CUDA(cudaMemcpyAsync(tiles_f, tf.data(), sizeof(int2) * tf.size(), cudaMemcpyHostToDevice, st));
  WT_CUDA(cudaMemcpyAsync(tiles_r, tr.data(), sizeof(int2) * tr.size(), cudaMemcpyHostToDevice, st));
  std::vector<Ctl> hctl(nprob, make_ctl(cfl, 0.0, INFINITY));

  // host <-> device for the caller's arrays
  bool u0_dev, g_dev, o_dev, t_dev = true;
  int dd;
  pointer_info(u0, &u0_dev, &dd);
  pointer_info(dJ_duT, &g_dev, &dd);
  pointer_info(dJ_du0, &o_dev, &dd);
  if (uT) pointer_info(uT, &t_dev, &dd);
  const double* src = u0;
  if (!u0_dev) {
    WT_CUDA(cudaMemcpyAsync(stage_buf, u0, vec_bytes, cudaMemcpyHostToDevice, st));
    src = stage_buf;
  }
  WT_CUDA(launch_pack1d_batched(src, n, Un, P, dsegs, nprob, n, 3, 1, st));
  auto init_ctl = [&](const double* state) -> int {
    WT_CUDA(cudaMemcpyAsync(ctl, hctl.data(), sizeof(Ctl) * nprob, cudaMemcpyHostToDevice, st));
    WT_CUDA(strict ? launch_alpha1d_batched_strict(WT_FLUX_EULER1D, state, P, dsegs, nprob, n, prob->gamma, 0.0, ctl, st)
                   : launch_alpha1d_batched_fast(WT_FLUX_EULER1D, state, P, dsegs, nprob, n, prob->gamma, 0.0, ctl, st));
    return WT_OK;
  };
  if ((rc = init_ctl(Un)) != WT_OK) return rc;
  auto bargs = [&](const double* in, const double* unp, double* out, const int2* tl, int nt, double* rec = nullptr) {
    BatchArgs b;
    memset(&b, 0, sizeof b);
    b.rec = rec;
    b.rec_off = rec ? goff : nullptr;
    b.uin = in;
    b.un = unp;
    b.uout = out;
    b.pitch = P;
    b.segs = dsegs;
    b.ctl = ctl;
    b.tiles = tl;
    b.ntiles = nt;
    b.gamma = prob->gamma;
    b.adv_speed = 0.0;
    b.eps = prob->eps;
    b.alpha_R = prob->alpha_R;
    return b;
  };
  const int nf = (int)tf.size(), nr = (int)tr.size();
  (void)nr;
  // the forward stages: 127-cell tiles with six (interface, field) items per thread, the
  // batched autotuner's pick on large Euler batches (every tile code gives the same bits)
  constexpr int kFwdTile = 5127;
  const int grid_f = batched_grid_size(prob, kFwdTile, nf, dev);
  auto launch_rec_stage = [&](int stage, const BatchArgs& b) {
    return strict ? launch_stage1d_batched_record_strict(stage, b, grid_f, st)
                  : launch_stage1d_batched_record_fast(stage, b, grid_f, st);
  };

  // Steps of one segment from segu(0, 0), keeping u^n, u^(1), u^(2) of every step and the
  // alphas and dt each stage used; the last step's u^{n+1} goes to final_out (if not null).
  auto record_segment = [&](int64_t kseg, double* final_out) -> int {
    for (int64_t k = 0; k < kseg; ++k) {
      double* ra = rec_a + (size_t)k * 3 * 4 * nprob;
      WT_CUDA(launch_adj_record(ctl, 0, ra, nullptr, nprob, st));
      WT_CUDA(launch_rec_stage(STAGE_RK1, bargs(segu(k, 0), nullptr, segu(k, 1), tiles_f, nf, recs(k, 0))));
      WT_CUDA(launch_adj_record(ctl, 1, ra + 4 * nprob, rec_dt + (size_t)k * nprob, nprob, st));
      WT_CUDA(launch_rec_stage(STAGE_RK2, bargs(segu(k, 1), segu(k, 0), segu(k, 2), tiles_f, nf, recs(k, 1))));
      WT_CUDA(launch_adj_record(ctl, 2, ra + 8 * nprob, nullptr, nprob, st));
      double* out = (k + 1 < kseg) ? segu(k + 1, 0) : final_out;
      // stage 3 of a segment's last step runs even where its state is not needed (it is the next
      // checkpoint, already known): the reverse needs its records.  Its state then goes to U1,
      // which nothing reads during the reverse sweep.
      WT_CUDA(launch_rec_stage(STAGE_RK3, bargs(segu(k, 2), segu(k, 0), out ? out : U1, tiles_f, nf, recs(k, 2))));
    }
    return WT_OK;
  };

  // ---- forward pass with checkpoints.  The last segment runs recording: its stage states
  // and alphas are what the reverse sweep starts from, so it is never recomputed.
  const int K = checkpoint_every;
  const int64_t S = (n_steps + K - 1) / K;
  const int64_t last0 = (S > 0) ? (S - 1) * K : 0;  // first step of the last segment
  {
    BatchArgs a3[3] = {bargs(Un, nullptr, U1, tiles_f, nf), bargs(U1, Un, U2, tiles_f, nf), bargs(U2, Un, Un, tiles_f, nf)};
    cudaGraphExec_t exec = nullptr;
    if (last0 > 0 && (rc = get_batched_graph(prob, dev, kFwdTile, grid_f, a3, &exec)) != WT_OK) return rc;
    for (int64_t step = 0; step < last0; ++step) {
      if (step % K == 0) WT_CUDA(cudaMemcpyAsync(ckpt + (size_t)(step / K) * 3 * P, Un, plane_bytes, cudaMemcpyDeviceToDevice, st));
      WT_CUDA(cudaGraphLaunch(exec, st));
    }
    if (n_steps > 0) {
      WT_CUDA(cudaMemcpyAsync(segu(0, 0), Un, plane_bytes, cudaMemcpyDeviceToDevice, st));
      if ((rc = record_segment(n_steps - last0, Un)) != WT_OK) return rc;
    }
  }
  {
    std::vector<Ctl> back(nprob);
    WT_CUDA(cudaMemcpyAsync(back.data(), ctl, sizeof(Ctl) * nprob, cudaMemcpyDeviceToHost, st));
    WT_CUDA(cudaStreamSynchronize(st));
    for (int p = 0; p < nprob; ++p)
      if (back[p].status != 0) return fail(back[p].status, "problem %d: forward pass reported status %d", p, back[p].status);
  }
  if (uT) {
    if (t_dev) {
      WT_CUDA(launch_unpack1d_batched(Un, P, uT, n, dsegs, nprob, n, 3, st));
    } else {
      WT_CUDA(launch_unpack1d_batched(Un, P, stage_buf, n, dsegs, nprob, n, 3, st));
      WT_CUDA(cudaMemcpyAsync(uT, stage_buf, vec_bytes, cudaMemcpyDeviceToHost, st));
    }
  }

  // ---- reverse sweep
  if (g_dev) {
    WT_CUDA(cudaMemcpyAsync(vX, dJ_duT, vec_bytes, cudaMemcpyDeviceToDevice, st));
  } else {
    WT_CUDA(cudaMemcpyAsync(vX, dJ_duT, vec_bytes, cudaMemcpyHostToDevice, st));
  }
  WT_CUDA(cudaMemsetAsync(dtbar, 0, sizeof(double) * nprob, st));
  const int grid_r = 0;  // resident-CTA count from the occupancy calculator
  for (int64_t sg = S - 1; sg >= 0; --sg) {
    const int64_t kseg = std::min<int64_t>(K, n_steps - sg * K);
    // recompute the segment from its checkpoint (the last one was recorded by the forward pass)
    if (sg < S - 1) {
      WT_CUDA(cudaMemcpyAsync(segu(0, 0), ckpt + (size_t)sg * 3 * P, plane_bytes, cudaMemcpyDeviceToDevice, st));
      if ((rc = init_ctl(segu(0, 0))) != WT_OK) return rc;
      if ((rc = record_segment(kseg, nullptr)) != WT_OK) return rc;
    }
    // reverse the steps of the segment
    for (int64_t k = kseg - 1; k >= 0; --k) {
      const double* ra = rec_a + (size_t)k * 3 * 4 * nprob;
      const double* rdt = rec_dt + (size_t)k * nprob;
      const double cLs[3] = {1.0, 0.25, 2.0 / 3.0};
      WT_CUDA(cudaMemsetAsync(vZ, 0, vec_bytes, st));
      for (int s = 2; s >= 0; --s) {
        const double* in = segu(k, s);
        const double* ubo = s == 2 ? vX : (s == 1 ? vY : vW);
        AdjArgs aa;
        memset(&aa, 0, sizeof aa);
        aa.uin = in;
        aa.pitch = P;
        aa.segs = dsegs;
        aa.tiles = tiles_r;
        aa.ntiles = nr;
        aa.ustride = n;
        aa.ubar_out = ubo;
        aa.alpha = ra + (size_t)s * 4 * nprob;
        aa.dt = rdt;
        aa.cL = cLs[s];
        aa.gamma = prob->gamma;
        aa.eps = prob->eps;
        aa.alpha_R = prob->alpha_R;
        aa.goff = goff;
        aa.G = Gbuf;
        aa.partial = partial;
        aa.rec = recs(k, s);
        WT_CUDA(strict ? launch_adj_stage_strict(aa, grid_r, adj_code, st) : launch_adj_stage_fast(aa, grid_r, adj_code, st));
        GatherArgs ga;
        memset(&ga, 0, sizeof ga);
        ga.uin = in;
        ga.pitch = P;
        ga.segs = dsegs;
        ga.goff = goff;
        ga.G = Gbuf;
        ga.ustride = n;
        ga.x = ubo;
        ga.gamma = prob->gamma;
        if (s == 2) {  // ubar(2) = 2/3 ubar(n+1) + J^T w;  ubar(n) = 1/3 ubar(n+1)
          ga.out = vY;
          ga.a_self = 2.0 / 3.0;
          ga.acc = vZ;
          ga.a_acc = 1.0 / 3.0;
        } else if (s == 1) {  // ubar(1) = 1/4 ubar(2) + J^T w;  ubar(n) += 3/4 ubar(2)
          ga.out = vW;
          ga.a_self = 0.25;
          ga.acc = vZ;
          ga.a_acc = 0.75;
        } else {  // ubar(n) += ubar(1) + J^T w
          ga.out = vZ;
          ga.a_self = 1.0;
          ga.accumulate = 1;
        }
        WT_CUDA(launch_adj_gather(ga, nprob, n, st));
        WT_CUDA(cudaMemsetAsync(arg, 0x7f, sizeof(int) * 4 * nprob, st));
        WT_CUDA(strict ? launch_adj_argmax_strict(in, P, dsegs, nprob, n, aa.alpha, prob->gamma, arg, st)
                       : launch_adj_argmax_fast(in, P, dsegs, nprob, n, aa.alpha, prob->gamma, arg, st));
        WT_CUDA(launch_adj_apply(in, P, dsegs, tstart, tcount, partial, aa.alpha, rdt, arg, ga.out, n, dtbar,
                                 s == 0 ? 1 : 0, prob->gamma, nprob, st));
      }
      std::swap(vX, vZ);
    }
  }
  if (o_dev) {
    WT_CUDA(cudaMemcpyAsync(dJ_du0, vX, vec_bytes, cudaMemcpyDeviceToDevice, st));
  } else {
    WT_CUDA(cudaMemcpyAsync(dJ_du0, vX, vec_bytes, cudaMemcpyDeviceToHost, st));
  }
  WT_CUDA(cudaStreamSynchronize(st));
  return WT_OK;
}

int wt_selftest_wait(int32_t which, int64_t limit_cycles, void* ws, size_t ws_bytes, void* stream) {
  if (which < 0 || which > 5) return fail(WT_ERR_ARG, "which = %d outside 0..5", which);
  if (limit_cycles < 1 || limit_cycles > (1LL << 31)) return fail(WT_ERR_ARG, "limit_cycles outside 1..2^31");
  int rc, dev;
  if ((rc = check_ws(ws, ws_bytes, 64, &dev)) != WT_OK) return rc;
  DeviceGuard guard;
  if ((rc = guard.enter(dev)) != WT_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* word = static_cast<unsigned long long*>(ws);
  int* result = reinterpret_cast<int*>(static_cast<char*>(ws) + 16);
  unsigned long long* mbox = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + 32);  // 4 words
  WT_CUDA(cudaMemsetAsync(ws, 0, 64, st));
  WT_CUDA(launch_selftest_wait(which, word, mbox, limit_cycles, result, st));
  int h = 0;
  WT_CUDA(cudaMemcpyAsync(&h, result, sizeof(int), cudaMemcpyDeviceToHost, st));
  WT_CUDA(cudaStreamSynchronize(st));
  if (h == WT_ERR_TIMEOUT) return fail(WT_ERR_TIMEOUT, "the device-side wait gave up after %lld cycles", (long long)limit_cycles);
  return h;
}

}  // extern "C"
