/*
 * weno_theta.h -- C ABI of the GB300 (sm_103a) implementation of the adaptive
 * WENO-theta finite-difference scheme of Jung & Nguyen, arXiv 1504.00731.
 *
 * Problem (Sec. 1, Eq. (mod_con_law); Sec. 2, Eq. (mod_con_scalar)):
 *     u_t + f(u)_x (+ g(u)_y) = 0,  u = (u_1 .. u_m),
 * semi-discretised as du_j/dt = L(u)_j = -(h_{j+1/2} - h_{j-1/2}) / dx (Eq. (mod_semi))
 * with the WENO-theta interface value of Eqs. (fh_nonlinear)-(tau_we6), global
 * Lax-Friedrichs splitting (Eq. (flux_split_lf)), characteristic-wise reconstruction
 * for systems (Sec. 4.2) and the third-order TVD Runge-Kutta method (Eq. (3rd_RK)).
 *
 * Conventions shared by every entry point
 *   - Arrays of doubles are component-major and unpadded: u[c * n + j] in 1D,
 *     u[(c * ny + y) * nx + x] in 2D (x fastest), c = 0 .. m-1.
 *   - Unless stated otherwise a pointer to state data may be DEVICE memory or HOST
 *     memory (pinned or pageable); the library looks at the pointer and copies host
 *     data through the workspace itself.  Device pointers are used in place.
 *   - The caller owns every buffer; the library never allocates device memory and
 *     never frees anything.  The workspace `ws` (device memory, 256-byte aligned,
 *     at least wt_workspace_bytes(...) bytes) holds all scratch state.  Its contents
 *     need no initialisation and are undefined after a call.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Work is queued on it; each entry point states when it synchronises.
 *   - The return value is a wt_status.  On an error the outputs are unspecified, the
 *     input state is untouched (the step entry points integrate in the workspace and
 *     copy back only on success), and wt_last_error() describes the failure.
 *   - Arithmetic is IEEE binary64 throughout (the method's own precision).
 */
#ifndef WENO_THETA_H
#define WENO_THETA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WT_OK = 0,
  WT_ERR_ARG = -1,          /* invalid argument (sizes, pointers, enums, alignment) */
  WT_ERR_UNSUPPORTED = -2,  /* valid but not implemented (e.g. reflective scalar) */
  WT_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  WT_ERR_NONPHYSICAL = -4,  /* the state became non-finite (NaN or Inf); a negative pressure or
                             * density in an intermediate RK stage is not an error: the scheme
                             * has no positivity limiter and integration continues through it */
  WT_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
  WT_ERR_WORKSPACE = -6     /* workspace missing, misaligned or too small */
} wt_status;

typedef enum {
  WT_FLUX_ADVECTION = 0, /* f = a u, m = 1 (Eq. (lin_eq)) */
  WT_FLUX_BURGERS = 1,   /* f = u^2 / 2, m = 1 (Eq. (bur_eq)) */
  WT_FLUX_EULER1D = 2,   /* m = 3, u = (rho, rho u, E) (Eq. (eu_eq)) */
  WT_FLUX_EULER2D = 3    /* m = 4, u = (rho, rho u, rho v, E) (Eq. (eu2D)) */
} wt_flux;

typedef enum {
  WT_BC_PERIODIC = 0,
  WT_BC_OUTFLOW = 1,     /* zero gradient ("transmissive", Sec. 4.2) */
  WT_BC_REFLECTIVE = 2   /* mirror, normal momentum negated (Euler only) */
} wt_bc;

typedef enum {
  /* fused multiply-adds, one division per reconstruction, restricted stencils take the
   * linear weights directly: agrees with the literal arithmetic to rounding */
  WT_MODE_FAST = 0,
  /* every operation in the order the paper prints it, no contraction: reproduces a
   * literal binary64 evaluation bit for bit */
  WT_MODE_STRICT = 1
} wt_mode;

/* How weno_theta_step advances a 1D grid (the 2D and batched entry points ignore it).  The
 * results are the same bit for bit; only the launches differ.  The paper has no counterpart:
 * it lets a caller compare the launch strategies on its own problems. */
typedef enum {
  /* chosen from how the grid's tiles fit the device: the step-blocked persistent kernel when
   * at most one 27-cell (Euler) or 51-cell (scalar) tile per SM is needed, else the
   * persistent kernel when every tile is co-resident, else the next */
  WT_LAUNCH_AUTO = 0,
  /* one launch of the fused RHS + RK stage kernel per stage, replayed from CUDA graphs of
   * eight RK steps */
  WT_LAUNCH_STAGES = 1
} wt_launch;

typedef struct {
  int32_t flux;       /* wt_flux */
  int32_t m;          /* number of components; must match flux (1, 1, 3, 4) */
  double gamma;       /* ratio of specific heats (Euler), e.g. 1.4 */
  double adv_speed;   /* a in f = a u (advection) */
  double eps;         /* epsilon of Eq. (om) and of R(beta) in Eq. (be_res); the paper uses 1e-10 */
  double alpha_R;     /* threshold alpha_R of Eq. (be_res); the paper uses 50, 10 or 1 by test */
  int32_t bc_lo[2];   /* wt_bc at x = lo for direction x (index 0) and y (index 1) */
  int32_t bc_hi[2];   /* wt_bc at x = hi */
  int32_t mode;       /* wt_mode */
  int32_t launch;     /* wt_launch (weno_theta_step, 1D); 0 = WT_LAUNCH_AUTO */
  double gravity;     /* 2D Euler only: g of the source terms -g rho (y momentum) and -g rho v
                         (energy) of the Rayleigh-Taylor test (TEST 6, Sec. 4.3), gravity along
                         -y; 0 for none.  Must be finite; nonzero for another flux is
                         WT_ERR_UNSUPPORTED. */
} wt_problem;

typedef struct {
  int32_t ndim;       /* 1 or 2; must be 2 exactly for WT_FLUX_EULER2D */
  int32_t reserved;   /* must be 0 */
  int64_t n[2];       /* cells per direction (n[1] ignored in 1D); each >= 3 */
  double lo[2];       /* domain [lo, hi] per direction; dx = (hi - lo) / n */
  double hi[2];
} wt_grid;

/* One problem of a batch (weno_theta_step_batched): a 1D grid of n cells on [lo, hi]
 * stored at u_packed[c * total + offset + j]. */
typedef struct {
  int64_t offset;     /* first cell in the packed arrays */
  int64_t n;          /* cells, >= 3 */
  double lo, hi;      /* dx = (hi - lo) / n */
  int32_t bc_lo, bc_hi;
} wt_segment;

/*
 * Workspace size in bytes for the entry points below.  For one grid pass
 * batch_cells = 0 and nprob = 0; for weno_theta_step_batched pass grid = NULL,
 * batch_cells = total cells of the batch and nprob = number of problems.
 * Returns 0 for invalid arguments.
 */
size_t wt_workspace_bytes(const wt_problem* prob, const wt_grid* grid, int64_t batch_cells, int32_t nprob);

/*
 * L(u) of Eq. (mod_semi) for one state: boundary fill of the ghost cells, the global
 * Lax-Friedrichs constants alpha_s = max_j |lambda_s(u_j)| (Eq. (flux_split_lf), one per
 * characteristic field and direction), and the WENO-theta interface fluxes of
 * Eqs. (fh_nonlinear)-(tau_we6) (characteristic-wise for Euler, Sec. 4.2).
 *   u  [m][cells]  input state (host or device)
 *   L  [m][cells]  output, same memory kind as u
 * Asynchronous on `stream` for device arrays; synchronous for host arrays.
 */
int weno_theta_rhs(const wt_problem* prob, const wt_grid* grid, const double* u, double* L, void* ws, size_t ws_bytes,
                   void* stream);

/*
 * Integrates u in place with the third-order TVD Runge-Kutta method (Eq. (3rd_RK)).
 * Each step takes dt = cfl * dx / max_j (|u_j| + c_j) from u^n (2D:
 * cfl / max_j ((|u|+c)/dx + (|v|+c)/dy); advection |a|, Burgers |u_j|), or dt = dt_fixed
 * when dt_fixed > 0, clipped so that t never passes t_final.  It stops after max_steps
 * steps or when t reaches t_final (t_final = +inf: exactly max_steps steps).
 *   u          [m][cells] state, host or device, updated on success
 *   t_reached  out (host, may be NULL): time reached; steps out (host, may be NULL)
 * Synchronises `stream` before returning.
 */
int weno_theta_step(const wt_problem* prob, const wt_grid* grid, double* u, double cfl, double dt_fixed,
                    double t_final, int64_t max_steps, double* t_reached, int64_t* steps, void* ws, size_t ws_bytes,
                    void* stream);

/*
 * Advances nprob independent 1D problems (each its own grid, boundary conditions,
 * Lax-Friedrichs constants and CFL step) by n_steps RK3 steps in one launch per RK
 * stage over all problems.  prob->flux must be 1D (advection, Burgers or Euler 1D).
 * The problems share no data: each is the scheme of Eqs. (mod_semi), (fh_nonlinear),
 * (flux_split_lf) and (3rd_RK) on its own grid, with its own alpha_s and dt.
 *   segs               [nprob] host array of wt_segment; segments must not overlap
 *   u_packed           [m][total] state, host or device, updated on success;
 *                      total = max(offset + n) over the segments
 *   t_per_problem      [nprob] out (host or device, may be NULL): time reached per problem
 *   status_per_problem [nprob] out (host or device, may be NULL): wt_status per problem.
 *                      NULL: the first problem whose state became non-finite (or whose
 *                      device wait gave up) fails the whole call and u_packed is untouched.
 *                      Non-NULL: such a problem stops at the step where it failed, its status
 *                      (WT_ERR_NONPHYSICAL or WT_ERR_TIMEOUT) is stored here, its part of
 *                      u_packed keeps the input state, every other problem is written back
 *                      as without it (bit for bit), and the call returns WT_OK;
 *                      wt_last_error() then names how many failed.
 * The tile of cells each CTA takes and the (interface, field) items each thread carries are
 * chosen by timing the candidates on the first call for a given batch (keyed by flux, mode,
 * device and the segments' lengths and boundaries) and reused afterwards; the results do not
 * depend on the choice.  The environment variable WT_BATCHED_TILE, if set, fixes the choice to
 * one tile code (cells per tile + 1000 x (items per thread - 1); Euler: 31, 63, 127, 1063,
 * 1127, 2127, 3127, 5127; scalar fluxes: 63, 127), for tests and for callers that tuned offline.
 * Host arrays: with u_packed in page-locked host memory, segments laid out in the order of the
 * problems, at least 2^23 cells and the tile already chosen, the call runs in up to four chunks
 * of problems, so that one chunk's copies to and from the device overlap another's steps (the
 * results are the same bit for bit; on failure the input is put back as described above).
 * Synchronises `stream` before returning.
 */
int weno_theta_step_batched(const wt_problem* prob, const wt_segment* segs, int32_t nprob, double* u_packed,
                            int64_t total, double cfl, int64_t n_steps, double* t_per_problem,
                            int32_t* status_per_problem, void* ws, size_t ws_bytes, void* stream);

/*
 * Gradient of J(u(T)) with respect to u(0) through n_steps RK3 steps (CFL step from u^n,
 * t_final = +inf) of nprob independent 1D Euler problems on the same grid, by the discrete
 * adjoint of the exact map the forward pass computes (reverse mode; every branch -- theta,
 * restriction, maxima, absolute values -- frozen where the forward pass took it, and the
 * derivative of a maximum sent to the first cell that attains it).  The forward pass keeps
 * every checkpoint_every-th state; the reverse sweep recomputes each segment from its
 * checkpoint, storing the RK stage states, and reverses it step by step.  The paper has no
 * adjoint; this differentiates its scheme (Eqs. (3rd_RK), (mod_semi), (fh_nonlinear)).
 *   u0      [nprob][3][n] initial states (host or device)
 *   dJ_duT  [nprob][3][n] gradient of J with respect to u(T)
 *   dJ_du0  [nprob][3][n] out: gradient with respect to u(0)
 *   uT      [nprob][3][n] out (may be NULL): u(T)
 * prob->flux must be WT_FLUX_EULER1D.  ws must hold wt_adjoint_workspace_bytes(...) bytes.
 * The environment variable WT_ADJ_TILE (31, 2031, 63, 1063 or 2063: cells per reverse tile +
 * 1000 x (items per thread - 1)) overrides the reverse kernel's tile; the gradients agree to
 * rounding.
 * Synchronises `stream`.
 */
size_t wt_adjoint_workspace_bytes(const wt_problem* prob, const wt_grid* grid, int32_t nprob, int64_t n_steps,
                                  int32_t checkpoint_every);
int weno_theta_adjoint(const wt_problem* prob, const wt_grid* grid, int32_t nprob, const double* u0, double cfl,
                       int64_t n_steps, int32_t checkpoint_every, const double* dJ_duT, double* dJ_du0, double* uT,
                       void* ws, size_t ws_bytes, void* stream);

/*
 * L(u) exactly as weno_theta_rhs computes it, for callers that cannot allocate device
 * memory and so cannot supply a workspace: a host program with no device allocator of
 * its own, a plug-in confined to its host application's fixed memory budget, or a
 * real-time loop in which an allocation would synchronise the device.  The paper has no
 * counterpart; this is a deployment variant of the RHS evaluation.
 *
 * Its scratch (control block and padded state with ghost cells) lives in one array of
 * WT_NOALLOC_SCRATCH_BYTES of device memory built into the library; every GPU that loads
 * the library holds that array until the process exits.  The call allocates and frees
 * nothing.  Sizes whose scratch does not fit (n > 349498 cells for Euler 1D, n > 1048506
 * for a scalar flux) are rejected with WT_ERR_ARG.  1D fluxes only.
 *   u  [m][n]  input, device memory
 *   L  [m][n]  output, device memory on the same GPU
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Every call
 * reuses the same array and each clears what must start at zero; calls whose GPU work
 * overlaps (other streams or host threads) race on it and must be serialised.
 * Asynchronous on `stream`.
 */
#define WT_NOALLOC_SCRATCH_BYTES (8u << 20)
int weno_theta_rhs_noalloc(const wt_problem* prob, const wt_grid* grid, const double* u, double* L, void* stream);

/*
 * Self-test of the bounded device-side waits that guard the kernels (bulk-copy completion
 * on an mbarrier, the grid barrier of the persistent kernels, the mailboxes through which
 * the step-blocked kernel exchanges halos and alphas).  Not part of the method (the paper
 * has no counterpart): it lets a caller check, without faulting or hanging the GPU, that a
 * wait which can never be satisfied gives up and reports WT_ERR_TIMEOUT.
 *   which         0: wait on a grid counter nobody increments; 1: wait on an mbarrier for
 *                 16 bulk-copy bytes that are never sent (no copy is issued); 2: a grid-
 *                 counter wait that is already satisfied; 3: wait for halo mailbox words
 *                 whose step tag never arrives; 4: wait for alpha mailbox words that never
 *                 carry the step's parity; 5: an alpha mailbox wait on words already
 *                 published (and their maxima checked).
 *   limit_cycles  give up after this many SM clock cycles, 1 .. 2^31
 *   ws, ws_bytes  device scratch of at least 64 bytes, 256-byte aligned (caller-owned)
 * Synchronises the stream.  Returns WT_ERR_TIMEOUT when the wait gave up (the expected
 * result for which = 0, 1, 3 and 4), WT_OK when it completed (which = 2 and 5), WT_ERR_ARG
 * for bad arguments; the context stays usable either way.
 */
int wt_selftest_wait(int32_t which, int64_t limit_cycles, void* ws, size_t ws_bytes, void* stream);

/* Message describing the last non-OK status returned on the calling thread. */
const char* wt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WENO_THETA_H */
