/*
 * lbm.h -- C interface of liblbm.so: one explicit time step of the 2-D
 * 16-velocity (Kataoka-Tsutahara) multiple-relaxation-time finite-difference
 * lattice Boltzmann model with flux-limited convection (Chen, Xu, Zhang, Wang,
 * arXiv:1305.4736), on an NVIDIA GB300 (sm_103a).
 *
 * General conventions
 *  - Every call returns LBM_OK (0) or a negative LBM_ERR_* code; no C++
 *    exception crosses this interface.  lbm_last_error() describes the last
 *    failure of a context (or of this thread when the context is NULL).
 *  - Host arrays are caller-owned, row-major [ny][nx] float64 (fields) or
 *    [16][ny][nx] float64 (population / moment sets), copied in or out during
 *    the call and never retained.
 *  - Device memory belongs to the context: two 16-plane buffers (ping-pong) of
 *    (ny + 4) rows by a padded pitch, allocated at create time through the
 *    allocator given to lbm_create_ex (default: cudaMalloc) and released by
 *    lbm_destroy.  All work is enqueued on the context's CUDA stream.
 *  - Grid: cell-centred, dx = dy, two ghost layers on every edge.  R = 1, so
 *    the pressure is P = rho T.  gamma = (b + 2)/b (Sec. II).
 *  - Relaxation rates s[0..15] are s_1 .. s_16 of Eq. (3); s_1..s_4 belong to
 *    conserved moments and are ignored.
 *  - Populations are ordered: i = 0..3 (1,0),(0,1),(-1,0),(0,-1); i = 4..7 the
 *    same times 6; i = 8..11 sqrt2 (1,1),(-1,1),(-1,-1),(1,-1); i = 12..15
 *    (3/sqrt2) (1,1),(-1,1),(-1,-1),(1,-1).  Moment rows k = 0..15 are
 *    m_1 .. m_16 of Appendix A.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,        /* invalid argument (NULL, sizes, rates, BC pairing) */
    LBM_ERR_CFL = -2,        /* max_i,a |v_ia| dt/dx > 1 (Sec. III update would be unstable) */
    LBM_ERR_STABILITY = -3,  /* some s_k dt >= 2 (k >= 5): forward-Euler relaxation unstable */
    LBM_ERR_OOM = -4,        /* device allocation failed */
    LBM_ERR_CUDA = -5,       /* a CUDA runtime call failed (no device, launch error, ...) */
    LBM_ERR_NONFINITE = -6,  /* a moment read-back found a non-finite value or rho <= 0 */
    LBM_ERR_STATE = -7,      /* call out of order (step before init, n <= 0, ...) */
    LBM_ERR_TIMEOUT = -8     /* a bounded device wait (TMA copy) ran out in a step; reported by
                                the next lbm_moments call */
};

/* Convection schemes of Sec. III. */
enum {
    LBM_LIMITER_MC = 0,      /* the paper's flux limiter psi(theta) (monotonised central) */
    LBM_LIMITER_LW = 1,      /* psi = 1: Lax-Wendroff */
    LBM_LIMITER_UPWIND = 2   /* psi = 0: first-order upwind */
};

/* Ghost-cell kinds (Sec. IV.A periodic / fixed equilibrium, Sec. IV.C
   non-equilibrium extrapolation wall, Sec. V inflow / outflow). */
enum {
    LBM_BC_PERIODIC = 0,       /* copy from the opposite edge; must be set on both edges of an axis */
    LBM_BC_ZERO_GRADIENT = 1,  /* copy the nearest interior cell (outflow) */
    LBM_BC_EQUILIBRIUM = 2,    /* f = M^-1 f_hat^eq(rho, u, v, T) of the edge state (inflow) */
    LBM_BC_NEQ_WALL = 3        /* wall on the face with velocity (u, v) and temperature T:
                                  ghost g, mirror m (-1<->0, -2<->1): rho_g = rho_m,
                                  u_g = 2 u_w - u_m, T_g = 2 T_w - T_m,
                                  f_g = f^eq(g) + (f_m - f^eq(m)); rho is unused */
};

/* Storage / arithmetic precision. */
enum {
    LBM_FP64 = 0,      /* f stored and updated in float64 */
    LBM_FP32_DEV = 1   /* g = f - f^eq(rho0, 0, 0, T0) stored and updated in float32;
                          moments recovered in float64 */
};

typedef struct { int kind; double rho, u, v, T; } lbm_edge_bc;
typedef struct { lbm_edge_bc xlo, xhi, ylo, yhi; } lbm_bc;

/* Optional device allocator (e.g. a framework's caching allocator).
   alloc returns a device pointer of at least `bytes` bytes usable on `stream`
   (NULL on failure); free releases it.  Both are called only from
   lbm_create_ex (alloc) and lbm_destroy (free), on the calling thread. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} lbm_allocator;

/* Extended options of lbm_create_ex. */
typedef struct {
    int precision;                 /* LBM_FP64 or LBM_FP32_DEV */
    double rho0, T0;               /* reference state of LBM_FP32_DEV (default 1, 1 when <= 0) */
    void *stream;                  /* cudaStream_t; NULL = the legacy default stream */
    const lbm_allocator *allocator;/* NULL = cudaMalloc / cudaFree */
    int device;                    /* CUDA device ordinal; < 0 = the current device */
    int step_kernel;               /* fused-step kernel: 0 = automatic (float64: the double-float
                                      kernel 8 on grids of at least 32 x 32, 9 on grids of 32
                                      columns or more and 4 to 31 rows; narrower grids:
                                      streaming on grids that give every SM at least 32 rows of a
                                      256-column strip and have at least 4M cells, else plain
                                      64-cell tiles;
                                      float32: TMA-staged where the grid allows, else plain
                                      32 x 8), 1 = plain 32 x 8 tiles (grids narrower than 32
                                      columns: TX x NT/TX tiles of the same NT threads, TX the
                                      smallest power of two >= nx, for options 1, 3, 4, 7)
                                      (global-memory stencil), 2 = TMA-staged 32 x 32 tiles (grids of
                                      at least 32 x 32), 3 = plain 32 x 4, 4 = plain 32 x 16,
                                      5 = streaming (CTAs walk 256-column strips row by row
                                      through a ring of TMA-filled row slots; grids of at least
                                      128 columns), 6 = persistent TMA-staged 32 x 16 tiles with
                                      two tile buffers per CTA (LBM_FP32_DEV only), 7 = plain
                                      64-cell tiles (32 x 2; spreads small float64 grids over
                                      every SM), 8 = LBM_FP64 only: the 32 x 32 TMA-staged tiles
                                      with the step's arithmetic in double-float form (pairs of
                                      float32, about 2^-47 rounding per operation) on the float32
                                      pipe, populations still stored and returned in float64
                                      (grids of at least 32 x 32), 9 = LBM_FP64 only: the same
                                      arithmetic on 32 x 4 tiles, two CTAs per SM (grids of at
                                      least 32 columns and 4 rows); all agree to round-off of
                                      their arithmetic (see lbm_autotune) */
    double dy;                     /* grid spacing along y; <= 0 means dy = dx.  The y projection
                                      of the convection uses the Courant numbers |v_iy| dt / dy and
                                      the y derivatives of the energy-flux correction divide by
                                      2 dy (Sec. III, Sec. II) */
} lbm_options;

typedef struct lbm_ctx lbm_ctx;   /* opaque, owned by the library */

/* Create a problem: grid nx x ny (>= 1), spacing dx > 0 (dy = dx; lbm_create_ex takes
   dy in lbm_options), time step dt > 0, gamma > 1, Prandtl number Pr > 0, rates s[16],
   limiter, boundary kinds.
   s[7] (s_8) <= 0 means s_8 = s_9 = Pr s_5; otherwise |s_8/s_5 - Pr| must be <= 1e-12 Pr.
   Isotropy s_5 = s_6 = s_7 and s_8 = s_9 is required (Sec. II).
   Errors: LBM_ERR_ARG, LBM_ERR_CFL (6 dt > min(dx, dy): a Courant number above 1),
   LBM_ERR_STABILITY, LBM_ERR_OOM, LBM_ERR_CUDA.
   On success *out receives the context (FP64, legacy default stream).  Its device memory
   comes from cudaMalloc: with no allocator given, the library falls back to cudaMalloc /
   cudaFree.  Callers that keep device memory in a framework's pool (the Python binding
   passes PyTorch's caching allocator) use lbm_create_ex with lbm_options.allocator. */
int lbm_create(int nx, int ny, double dx, double dt, double gamma, double Pr,
               const double s[16], int limiter, const lbm_bc *bc, lbm_ctx **out);

/* As lbm_create with precision, stream, allocator and device options (opt may be NULL). */
int lbm_create_ex(int nx, int ny, double dx, double dt, double gamma, double Pr,
                  const double s[16], int limiter, const lbm_bc *bc,
                  const lbm_options *opt, lbm_ctx **out);

/* Initialise every interior cell to f = M^-1 f_hat^eq(rho, u, v, T) (Appendix A;
   the initialisation practice of Sec. IV.A).  Host arrays [ny][nx], caller-owned, not retained.
   When all four lie in page-locked memory allocated or registered through CUDA, the init
   kernel reads them over the host link directly; other host memory is copied through a device
   staging buffer in chunks.  LBM_FP32_DEV evaluates the deviation g = f^eq - f^eq0 in float32
   from float64 deviations of rho, j and P.  rho > 0, T > 0 and finite values, checked on the
   device: LBM_ERR_ARG otherwise, and the context is then left uninitialised.  Synchronous. */
int lbm_init(lbm_ctx *ctx, const double *rho, const double *u, const double *v, const double *T);

/* Enqueue n >= 1 time steps (ghost fill + fused collide/convect per step; Eq. (3) and
   the update of Sec. III).  Asynchronous on the context's stream.  Runs of 16 steps or more
   (outside lbm_profile_begin / lbm_profile_end) replay pairs of steps from a CUDA graph that the
   context captures on a private stream at first use, one per starting buffer (lbm_autotune
   drops them): the same launches, one graph launch per pair.
   LBM_ERR_STATE if n <= 0 or the context was never initialised. */
int lbm_step(lbm_ctx *ctx, int n);

/* Macroscopic fields and non-equilibrium moments Delta_k = (M f)_k - f_hat^eq_k
   (Sec. V).  Outputs [ny][nx] (rho, u, v, T) and [16][ny][nx] (delta); any output
   may be NULL.  When every requested output lies in page-locked memory allocated or
   registered through CUDA, the moments kernel writes them over the host link directly;
   otherwise they come through a device staging buffer.  Synchronous.  LBM_ERR_NONFINITE if
   a cell has a non-finite value or rho <= 0 (outputs are still written). */
int lbm_moments(lbm_ctx *ctx, double *rho, double *u, double *v, double *T, double *delta);

/* Central non-equilibrium moments Delta*_k = (M* (f - f^eq))_k with M* built at each
   cell's own flow velocity (Sec. V, Appendix A).  Output [16][ny][nx].  Synchronous. */
int lbm_moments_central(lbm_ctx *ctx, double *delta_star);

/* Domain totals of rho, j_x, j_y and e (twice the total energy), each times dx dy,
   summed in float64 in a fixed order (deterministic).  Synchronous. */
int lbm_totals(lbm_ctx *ctx, double out[4]);

/* Interior populations f (not g, in LBM_FP32_DEV) as [16][ny][nx] float64: read / write.
   Synchronous.  lbm_set_state also marks the context initialised. */
int lbm_get_state(lbm_ctx *ctx, double *f);
int lbm_set_state(lbm_ctx *ctx, const double *f);

/* Interior populations of rows row0 .. row0+rows-1 only, as [16][rows][nx] float64
   (a window of lbm_get_state, for chunked checkpoints and sampled checks).
   LBM_ERR_ARG if the window leaves [0, ny).  Synchronous. */
int lbm_get_state_rows(lbm_ctx *ctx, int row0, int rows, double *f);

/* Kernel timing for measurement.  lbm_profile_begin(ctx, max_steps) makes the next
   lbm_step calls record a CUDA event pair around each ghost-fill and each fused-step
   launch (up to max_steps steps; the events live on the context's stream).
   lbm_profile_end(ctx, out) waits for them and writes out[0] = total fused-step
   kernel time in ms, out[1] = fused-step launches, out[2] = total ghost-fill time
   in ms, out[3] = ghost-fill launches, then stops recording.
   LBM_ERR_STATE if lbm_profile_end is called without lbm_profile_begin. */
int lbm_profile_begin(lbm_ctx *ctx, int max_steps);
int lbm_profile_end(lbm_ctx *ctx, double out[4]);

/* Measurement helper (not part of the method): sustained float64 FMA throughput of
   device `device` from an FMA-chain kernel, in FLOP/s (FMA = 2), written to *flops.
   The roofline of the float64 mode, which is bound by the float64 pipe, uses it. */
int lbm_peak_fp64(int device, double *flops);

/* Pick the fastest fused-step kernel for this context's grid: times `reps` launches of
   each candidate (plain 32 x 4, 32 x 8, 32 x 16 and 64-cell tiles; TMA-staged tiles, the
   streaming kernel, the double-buffered TMA-staged kernel and the double-float kernels on
   32 x 32 and 32 x 4 tiles when the grid and precision allow) on the context's current state, writing the spare buffer without advancing the
   state, and keeps the fastest for later lbm_step calls.  *choice (may be NULL) receives
   the lbm_options.step_kernel code of the winner.  Synchronous.  Not part of the paper's
   method: a throughput tool. */
int lbm_autotune(lbm_ctx *ctx, int reps, int *choice);

/* Batched stepping of several problems (uneven grids, any mix of precision and limiter).
   Not part of the paper's method: a throughput tool for many small grids, whose single
   steps are launch-bound.  The contexts must be initialised, share one device and one
   stream, and stay alive while the batch exists.  Each step of lbm_batch_step runs, per
   group of contexts with the same precision and limiter, one batched ghost-fill launch and
   fused-step launches over the tiles of the group's grids:
   - contexts whose step kernel is the TMA-staged tile kernel (float32) or a double-float
     kernel (float64), i.e. the automatic choice on grids of at least 32 x 16 (float32) or
     32 x 4 (float64), have their tiles in one launch of that kernel's batched form per 128
     such grids (float64: one for the 32 x 32 tiles, one for the 32 x 4 tiles) (one CTA per tile; the launch's parameters hold each grid's tensor map,
     output buffer and tile count, and the CTA stages its grid's coefficients in shared
     memory), with the arithmetic of the single-grid kernel, bit for bit;
   - the other grids share the packed plain kernel, whose persistent CTAs walk a tile list
     (float32: 256-cell tiles, float64: 64-cell tiles, which spread small float64 grids over
     more SMs; 32 columns wide, or TX = the smallest power of two >= nx for narrower grids)
     with the arithmetic of the plain step kernel, to round-off (the compiler may contract
     multiply-adds differently);
   - a context on the streaming or the double-buffered kernel with at least 512 cells per SM
     takes part in its group's ghost launch only and steps with its own kernel, launched on
     one of eight forked streams so that such grids overlap, bit for bit.
   Pairs of steps are replayed from a CUDA graph captured on the first call with n >= 2
   (recaptured when a context was stepped alone an odd number of times since).  Tiles are independent, so a grid's result does not depend on the other members
   of its batch (bit for bit).
   Contexts may also be stepped alone between batch steps.  Errors: LBM_ERR_ARG (NULL, empty, mixed device or stream, a
   context listed twice), LBM_ERR_STATE (uninitialised context, n <= 0), LBM_ERR_OOM,
   LBM_ERR_CUDA. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_ctx *const *ctxs, int n, lbm_batch **out);
int lbm_batch_step(lbm_batch *batch, int n);        /* asynchronous on the shared stream */
void lbm_batch_destroy(lbm_batch *batch);           /* waits for the stream; NULL-safe */

/* Failure-path check of the bounded device waits of the TMA-fed step kernels, with no GPU
   fault: one warp waits on an mbarrier phase that nothing completes, using the kernels' own
   bounded wait (global-timer limit 2 s); the wait gives up, the kernel records it and returns,
   and the device stays usable.  Returns LBM_ERR_TIMEOUT when the wait ran out (the expected
   outcome), LBM_OK if the phase completed, LBM_ERR_CUDA on a CUDA error.  *elapsed_ms (may be
   NULL) receives the kernel's duration.  Not part of the paper's method. */
int lbm_wait_selftest(int device, double *elapsed_ms);

/* Largest ny accepted by lbm_totals_noalloc (its scratch holds one partial per grid row). */
#define LBM_TOTALS_NOALLOC_MAX_ROWS 16384

/* Conserved totals of a population field without allocating any device memory.
   The paper has no counterpart: this is a service for callers that cannot
   allocate -- their device memory belongs to another allocator (a framework's
   caching pool, a serving engine with a fixed memory plan), or they must not call
   cudaMalloc / cudaFree, which can synchronise the whole device.
   f: device pointer to caller-owned float64 populations, dense [16][ny][nx] (the
   layout lbm_get_state writes), on the current device.  dx, dy: grid spacings.
   out: host array that receives sum rho, sum j_x, sum j_y, sum e, each times the
   cell area dx dy (the scaling of lbm_totals).
   stream: cudaStream_t (NULL = legacy default stream); the call waits for it.
   Scratch: a fixed file-scope device array of (LBM_TOTALS_NOALLOC_MAX_ROWS + 1) x 4
   doubles (512 KB), held by every GPU that loads the library until the process
   exits.  The first call on a device looks up that array's address on the device
   and keeps it (make that first call before any stream capture); after a
   cudaDeviceReset of the device the kept address is stale, so do not call this on a
   device that was reset.  All calls share the array; each overwrites what it uses,
   so nothing needs clearing, but calls that overlap on the GPU race on it and must
   be serialised by the caller.
   Errors: LBM_ERR_ARG (NULL pointer, nx or ny < 1, dx or dy <= 0, ny above
   LBM_TOTALS_NOALLOC_MAX_ROWS), LBM_ERR_CUDA.  No cudaMalloc or cudaFree is called. */
int lbm_totals_noalloc(const double *f, int nx, int ny, double dx, double dy, void *stream, double out[4]);

/* Steps taken since the last lbm_init / lbm_set_state. */
long long lbm_step_count(const lbm_ctx *ctx);

/* The lbm_options.step_kernel code (1 .. 9) of the fused-step kernel this context runs
   (after automatic selection or lbm_autotune); -1 for a NULL context. */
int lbm_step_kernel(const lbm_ctx *ctx);

/* Device footprint in bytes of a problem of this size and precision (both buffers). */
size_t lbm_footprint(int nx, int ny, int precision);

/* Text of the last error (never NULL). */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Release the context and its device memory (waits for its stream).  NULL-safe. */
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
