/*
 * sparkling.h -- C ABI of the GB300 (sm_103a) library for the hot path of
 * full-3D SPARKLING (arxiv 2108.02991): the gradient and energy of the
 * attraction-repulsion cost with kernel H(x) = |x|_2, and the per-shot
 * projection onto the gradient-amplitude and slew-rate constraints.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Samples K are N = Nc * Ns points in [-1/2,1/2]^3 (the paper's Omega =
 *   [-1,1]^3 of Sec. II-A scaled by 1/2), stored shot after shot as an
 *   array-of-structs [N][3] of float (SPARKLING_F32) or double (SPARKLING_F64).
 * - The target density is sampled on a cell-centred grid: along an axis of n
 *   cells over [lo, hi] the points are lo + (q + 1/2)(hi - lo)/n, q = 0..n-1.
 *   rho is float32, C order [nz][ny][nx] (x fastest), rho >= 0; the sum is
 *   expected to be 1 (eq. discritize with the integral replaced by a sum) but
 *   is not enforced.
 * - Array arguments are DEVICE pointers (cudaMalloc or managed memory) owned
 *   by the caller unless the name ends in _host.  The library never frees them.
 *   A pointer the CUDA runtime does not report as device or managed memory is
 *   rejected with SPARKLING_E_INVAL before anything is launched.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls are asynchronous on it unless they return a host value (those block
 *   on `stream` before returning).
 * - Each context owns its device workspace.  It grows on demand: the library
 *   synchronises the device, frees the old buffer and cudaMallocs a larger
 *   one (SPARKLING_E_NOMEM if that fails).  Call once at the largest size
 *   before capturing a CUDA graph.  A context is not thread-safe; use one per
 *   host thread.
 * - Arguments are validated before any launch; a failing check returns
 *   SPARKLING_E_INVAL and sparkling_last_error() says which.  No C++ exception
 *   crosses the ABI.
 * - Errors found on the device (non-finite input, a bounded wait that ran out)
 *   are recorded in a device status word of the context.  Blocking calls
 *   return them; after asynchronous calls, sparkling_status() reports them.
 *
 * Notation (paper Sec. II-B/II-C, eqs. attraction_term, repulsion_term,
 * attraction_derivative_basic, Fr_grad with H = |.|_2, H' = 1):
 *   A_i = sum_q rho_q (K_i - x_q) / |K_i - x_q|           attraction force
 *   R_i = (1/N) sum_{j != i} (K_i - K_j) / |K_i - K_j|    repulsion force
 *   G_i = A_i - R_i = N * dF/dK_i                         the "gradient"
 *   F   = F^a - F^r,  F^a = (1/N) sum_i sum_q rho_q |K_i - x_q|,
 *                     F^r = (1/(2 N^2)) sum_{i != j} |K_i - K_j|
 * A pair whose distance is (numerically) zero contributes nothing.
 */
#ifndef SPARKLING_H
#define SPARKLING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(_WIN32)
#define SPARKLING_API
#else
#define SPARKLING_API __attribute__((visibility("default")))
#endif

/* Status codes returned by every int-valued entry point. */
#define SPARKLING_OK 0
#define SPARKLING_E_INVAL 1     /* bad argument; nothing was launched */
#define SPARKLING_E_NOMEM 2     /* workspace allocation failed */
#define SPARKLING_E_CUDA 3      /* a CUDA runtime call failed (no device, launch error...) */
#define SPARKLING_E_NONFINITE 4 /* NaN/Inf in K or rho, or negative rho */
#define SPARKLING_E_TIMEOUT 5   /* a bounded device wait gave up (the kernel returned early) */
#define SPARKLING_E_NOTCONV 6   /* converged-mode projection did not certify within n_iter */
#define SPARKLING_E_IO 7        /* a checkpoint file could not be written */
#define SPARKLING_E_RANGE 8     /* a sample lies outside the fast-repulsion mesh */

/* Element types of K, G, A, R. */
#define SPARKLING_F32 0
#define SPARKLING_F64 1

/* Per-target accumulation of the FP32 pair sums.
 * KAHAN32:   every grid row / source block is summed in FP32 and folded into
 *            a compensated (TwoSum) FP32 accumulator.
 * FP64:      the same FP32 partial sums are folded into FP64 accumulators.
 * FP64_PAIR: the plain FP64-accumulate form, kept to compare against: every
 *            attraction pair term is converted to FP64 and added to FP64
 *            sums one by one (GB300's FP64 pipe bounds it; about 30 times
 *            slower).  The repulsion then folds its FP32 block sums in FP64.
 *            Accepted by sparkling_grad, sparkling_energy,
 *            sparkling_energy_backward, sparkling_step and the driver; the
 *            batched step and sparkling_grad_noalloc reject it. */
#define SPARKLING_ACC_KAHAN32 0
#define SPARKLING_ACC_FP64 1
#define SPARKLING_ACC_FP64_PAIR 2

typedef struct sparkling_ctx sparkling_ctx;

/* Density grid (eq. discritize): device pointer rho [nz][ny][nx] float32 on
 * the cell-centred grid over [lo, hi]^3 described above.  1 <= n[a] and
 * n[0] (= nx) <= 4096. */
typedef struct sparkling_grid {
    const float *rho;
    double lo;
    double hi;
    int32_t n[3]; /* nx, ny, nz */
    int32_t reserved;
} sparkling_grid;

/* Constraint set of one shot (eq. constraints): |s|_inf <= box,
 * |s[n+1]-s[n]|_2 <= alpha, |s[n+2]-2s[n+1]+s[n]|_2 <= beta for every n, and
 * s[pin_index] = pin (the linear constraint A k = v; pin_index < 0: none).
 * alpha or beta = +inf switches that constraint off.
 * tol <= 0: exactly n_iter dual-FISTA iterations.  tol > 0 ("converged
 * mode"): aim at the set with alpha, beta shrunk by (1 - margin) and stop at
 * the first check (every check_every iterations) where all violations of that
 * set and the duality gap are <= tol. */
typedef struct sparkling_proj {
    double alpha;
    double beta;
    double box;
    double tol;
    double margin;
    double pin[3];
    int32_t pin_index;
    int32_t n_iter;
    int32_t check_every;
    int32_t reserved;
} sparkling_proj;

/* Kernel kinds reported by sparkling_kernel_times(). */
#define SPARKLING_KERNEL_PACK 0
#define SPARKLING_KERNEL_ATTRACTION 1
#define SPARKLING_KERNEL_REPULSION 2
#define SPARKLING_KERNEL_COMBINE 3
#define SPARKLING_KERNEL_PROJECT 4
#define SPARKLING_KERNEL_ENGINE 5   /* a whole batched step (packs + persistent engine) */
#define SPARKLING_KERNEL_DRIVER 6   /* up-sampling and step-size reductions of the driver */
#define SPARKLING_KERNEL_STEP 7     /* the whole device work of one sparkling_step call */
#define SPARKLING_KERNEL_COUNT 8

/* Arithmetic of the projection (sparkling_set_projection). */
#define SPARKLING_PROJECTION_FP64 0    /* duals, primal and step in FP64 for every K dtype (default) */
#define SPARKLING_PROJECTION_MIXED 1   /* FP32 K, fixed n_iter: FP32 iteration on s - k and the duals */

/* How sparkling_step runs its device work (sparkling_set_step_path). */
#define SPARKLING_STEP_AUTO 0      /* the persistent engine from 2^22 samples on, else the kernels (default) */
#define SPARKLING_STEP_KERNELS 1   /* attraction, repulsion, combine and projection kernels in turn */
#define SPARKLING_STEP_ENGINE 2    /* the one-launch persistent engine wherever it applies */

/* How the attraction term is evaluated (sparkling_set_attraction). */
#define SPARKLING_ATTRACTION_DIRECT 0   /* direct sum over the grid: O(N P) */
#define SPARKLING_ATTRACTION_FIELD 1    /* interpolated node field: O(N), approximate */

/* How the repulsion term is evaluated (sparkling_set_repulsion). */
#define SPARKLING_REPULSION_DIRECT 0    /* every pair: O(N^2), exact */
#define SPARKLING_REPULSION_MESH 1      /* particle-particle particle-mesh: ~O(N), approximate */

/* Mesh of the fast repulsion.  The mesh covers [lo, hi]^3 with n_cells
 * cells of side h = (hi - lo) / n_cells per axis plus g guard cells on each
 * side (g >= 4, the smallest making n_cells + 2g a product of 2, 3, 5, 7);
 * samples may lie up to g - 2 cells outside [lo, hi]. */
typedef struct sparkling_mesh {
    double lo, hi;         /* the samples' box */
    double sigma_cells;    /* split width sigma in cells, > 0 (2.5: long-range error ~1e-6) */
    double rc_sigmas;      /* short-range cut-off in units of sigma, >= 2 (4: erfc(4) = 1.5e-8) */
    int32_t n_cells;       /* mesh cells across [lo, hi], 8 .. 1024 */
    int32_t reserved;
} sparkling_mesh;

/* Flags of sparkling_step_batched. */
#define SPARKLING_BATCH_GRAPH 1     /* replay the step from a cached CUDA graph */
#define SPARKLING_BATCH_TWO_LAUNCHES 2 /* the symmetric repulsion in its own kernel first */

/* Step schedule of the multi-resolution driver (Algorithm 1 and Sec. II-C,
 * choice of step size). */
typedef struct sparkling_schedule {
    double eta;            /* fixed step, in units of G (K <- Pi(K - eta G)); > 0 */
    double eta_min;        /* Barzilai-Borwein steps are clamped to [eta_min, eta_max], */
    double eta_max;        /*   0 < eta_min <= eta_max */
    double alpha_factor;   /* level l runs under alpha * alpha_factor^l and beta * beta_factor^l */
    double beta_factor;    /*   (per-step bounds: 2 and 4 when the raster step doubles) */
    int32_t n_git;         /* projected-gradient iterations per level, >= 0 */
    int32_t n_fixed;       /* iterations on the fixed step before Barzilai-Borwein (the paper: 20) */
    int32_t reserved[2];
} sparkling_schedule;

/* Create a context bound to CUDA device `device`.  Nothing is allocated on
 * the device and no CUDA call is made until the first compute call.
 * Returns SPARKLING_E_INVAL if out is NULL or device < 0. */
SPARKLING_API int sparkling_create(sparkling_ctx **out, int device);

/* Release the context and its workspace (synchronises the device first).
 * NULL is ignored. */
SPARKLING_API void sparkling_destroy(sparkling_ctx *ctx);

/* Message of the last failure on this context (ctx == NULL: of the last
 * failure with no context on this thread).  Never NULL; owned by the library,
 * valid until the next call on the same context/thread. */
SPARKLING_API const char *sparkling_last_error(const sparkling_ctx *ctx);

/* Attraction-repulsion gradient (Sec. II-C, eqs. attraction_derivative_basic
 * and Fr_grad; the attraction is the direct sum over the density grid).
 *   K       [N][3] of K_dtype, N >= 2 (read only)
 *   grid    density grid (struct in host memory, rho on the device)
 *   acc     SPARKLING_ACC_KAHAN32 or SPARKLING_ACC_FP64
 *   G       [N][3] of G_dtype, receives A - R
 *   A, R    optional [N][3] of G_dtype (NULL: not written), receive A and R
 * Asynchronous on `stream`. */
SPARKLING_API int sparkling_grad(sparkling_ctx *ctx, const void *K, int K_dtype, int64_t N,
                                 const sparkling_grid *grid, int acc, void *G, int G_dtype,
                                 void *A, void *R, void *stream);

/* Energy F = F^a - F^r (eqs. global_minimization, attraction_term,
 * repulsion_term).  Same K, grid, acc as sparkling_grad.  Writes the three
 * host doubles (any may be NULL) and blocks on `stream`.  The per-target sums
 * are reduced in a fixed order, so repeated calls give identical results. */
SPARKLING_API int sparkling_energy(sparkling_ctx *ctx, const void *K, int K_dtype, int64_t N,
                                   const sparkling_grid *grid, int acc, double *F_host,
                                   double *Fa_host, double *Fr_host, void *stream);

/* Backward of sparkling_energy for automatic differentiation: writes
 *   dK = g * dF/dK = g * (A - R) / N,   g = scale * (*g_dev)  (g_dev NULL: 1)
 * where g_dev is a device pointer to one double (the upstream gradient of
 * the energy).  dK is [N][3] of dK_dtype on the device.  The per-pair
 * distances are recomputed, never stored.  Asynchronous on `stream`. */
SPARKLING_API int sparkling_energy_backward(sparkling_ctx *ctx, const void *K, int K_dtype,
                                            int64_t N, const sparkling_grid *grid, int acc,
                                            const double *g_dev, double scale, void *dK,
                                            int dK_dtype, void *stream);

/* Projection of each of Nc shots of Ns samples onto the constraint set
 * (Sec. II-D, Suppl. Sec. I), in place on K ([Nc*Ns][3], K_dtype), with the
 * dual FISTA iteration in FP64 (sparkling_set_projection: the opt-in mixed
 * form for FP32 K):
 *   D1 s[n] = s[n+1]-s[n], D2 s[n] = s[n+2]-2s[n+1]+s[n];
 *   s(q) = pin(clip_box(k - D1^T q1 - D2^T q2)); step tau = 1/20;
 *   z = y + tau D s(y); q+ = z - P_ball(tau*alpha or tau*beta)(z) per row;
 *   t+ = (1 + sqrt(1 + 4t^2))/2; y = q+ + ((t-1)/t+)(q+ - q);
 *   output s(q) (q = y = 0, t = 1 at the start of every call).
 * Nc >= 1, 1 <= Ns <= 65536.  viol_host (optional, [4]) receives the largest
 * amplitude, slew, box and pin violation of the result; when it is given, or
 * in converged mode, the call blocks on `stream`. */
SPARKLING_API int sparkling_project(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc,
                                    int64_t Ns, const sparkling_proj *proj, double *viol_host,
                                    void *stream);

/* One projected-gradient step (eq. proj_grad_descent, Algorithm 1 inner
 * loop): K <- Pi(K - eta * G(K)) in place, G = A - R as in sparkling_grad
 * (so eta = 1/N is a unit step on dF/dK).  The gradient is kept in FP64 in
 * the workspace; the step and the projection run in FP64 (unless the
 * context chose SPARKLING_PROJECTION_MIXED) and the result is rounded to
 * K_dtype.  With timing on, the device work of the call is also timed as one
 * SPARKLING_KERNEL_STEP scope.  The device work runs either as the separate
 * kernels or as one launch of the persistent engine (sparkling_step_batched
 * with B = 1: the same arithmetic, attraction and symmetric repulsion items
 * sharing the SMs), as sparkling_set_step_path chooses; the engine applies
 * with direct sums, ACC_KAHAN32 or ACC_FP64 and a fixed n_iter.
 * Asynchronous on the kernels path unless converged mode is requested; the
 * engine path first waits for the stream's earlier work. */
SPARKLING_API int sparkling_step(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc, int64_t Ns,
                                 const sparkling_grid *grid, int acc, double eta,
                                 const sparkling_proj *proj, void *stream);

/* One projected-gradient step K_b <- Pi(K_b - eta_b G(K_b)) for B
 * independent trajectories of uneven size in one persistent launch (plus
 * the packing of samples and densities): a work list of attraction items (a
 * tile of 1024 targets against a run of grid rows) and symmetric repulsion
 * items (a tile of targets against a run of source tiles, each unordered
 * pair once, exact fixed-point totals per sample), followed by one
 * projection item per shot that waits (bounded) for its trajectory's pair
 * items.  With SPARKLING_BATCH_TWO_LAUNCHES (and wherever the one-launch
 * kernel shape cannot be resident) the symmetric repulsion of every
 * trajectory runs first in its own kernel -- the same totals bit for bit --
 * and the persistent kernel's list holds only the attraction and projection
 * items.  (Where the symmetric kernel cannot be resident either, the
 * repulsion runs as directed items of the work list.)  Same arithmetic as
 * sparkling_step: FP32 pairs,
 * acc per-target folds, FP64 gradient, step and projection (fixed n_iter;
 * converged mode is not available here); the context's regularisation
 * applies, its attraction and repulsion modes do not (direct sums).
 *   traj_off  host [B+1]: trajectory b is samples [traj_off[b], traj_off[b+1])
 *             of K; traj_off[0] = 0; every trajectory holds >= 2 samples and
 *             a whole number of shots of Ns samples
 *   K         device [traj_off[B]][3] of K_dtype, updated in place
 *   grids     host [B] density grids (rho on the device); eta host [B];
 *   proj      host [B] constraint sets (tol must be <= 0)
 *   flags     SPARKLING_BATCH_GRAPH: from the second call with the same
 *             shapes, K, densities and workspace on, the device work of the
 *             step is captured once into a CUDA graph and replayed (calls on
 *             a stream the caller is itself capturing are never captured);
 *             SPARKLING_BATCH_TWO_LAUNCHES: the repulsion kernel ahead of
 *             the persistent kernel, as above.
 * The work list is planned and uploaded when the shapes change; make the
 * first call of a shape outside any caller-side stream capture.  The item
 * granularity comes from the context's autotuned setting.  Asynchronous. */
SPARKLING_API int sparkling_step_batched(sparkling_ctx *ctx, int32_t B, const int64_t *traj_off,
                                         void *K, int K_dtype, int32_t Ns,
                                         const sparkling_grid *grids, const double *eta,
                                         const sparkling_proj *proj, int acc, int flags,
                                         void *stream);

/* sparkling_step on HOST buffers: K_host [Nc*Ns][3] (K_dtype) is copied to
 * the device, stepped, and copied back; rho_host [nz][ny][nx] float32 is
 * copied to the device (grid->rho is ignored).  Blocks until K_host holds
 * the result.  Pinned host memory makes the copies asynchronous DMA. */
SPARKLING_API int sparkling_step_host(sparkling_ctx *ctx, void *K_host, int K_dtype, int64_t Nc,
                                      int64_t Ns, const sparkling_grid *grid,
                                      const float *rho_host, int acc, double eta,
                                      const sparkling_proj *proj, void *stream);

/* The gradient of sparkling_grad without any device allocation, for callers
 * that must not (or cannot) let a library call cudaMalloc: processes whose
 * device memory belongs to their own pool or arena, code that must not
 * trigger the synchronisation or failure modes of a new allocation, and
 * deployments that need every byte a library holds known in advance.  The
 * paper has no counterpart; this is an engineering variant of the gradient.
 *
 * No context: scratch space is one fixed array compiled into the library,
 * 32 MiB, held on every GPU that loads the library until the process exits.
 * A problem needs about 16 N + 4 ny nz ceil4(nx) bytes plus at least 128 KiB
 * per 1024 samples of partial sums (more when the GPU has CTAs to spare); sizes that
 * do not fit are rejected with SPARKLING_E_INVAL and a message giving the
 * bytes needed (e.g. N up to ~2e5 with a 64^3 grid fits).  K, G and
 * grid->rho are device memory as in sparkling_grad; G = A - R in G_dtype.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it: make that
 * first call before capturing any CUDA stream.  All calls share the array;
 * each call clears its status word and overwrites every other byte it reads,
 * but calls whose kernels overlap on the GPU race on it and must be
 * serialised by the caller.  Blocks on `stream` and returns device-side
 * errors (SPARKLING_E_NONFINITE, SPARKLING_E_TIMEOUT) directly; messages go
 * to sparkling_last_error(NULL). */
SPARKLING_API int sparkling_grad_noalloc(const void *K, int K_dtype, int64_t N,
                                         const sparkling_grid *grid, int acc, void *G, int G_dtype,
                                         void *stream);

/* Synchronise `stream`, then return and clear the device status word of the
 * context (SPARKLING_OK, SPARKLING_E_NONFINITE or SPARKLING_E_TIMEOUT). */
SPARKLING_API int sparkling_status(sparkling_ctx *ctx, void *stream);

/* Kernel timing: when enabled, every kernel launch of the context is
 * bracketed by CUDA events on its stream.  sparkling_kernel_times()
 * synchronises the pending events and writes, for the first n kinds
 * (SPARKLING_KERNEL_*), the total milliseconds and the number of timed
 * scopes since the last reset (one per launch, except PACK -- samples and
 * density packed together -- COMBINE in energy mode -- two reduction kernels
 * -- ENGINE -- a whole batched step -- and STEP -- the whole device work of a
 * sparkling_step or sparkling_step_host call, between the host copies);
 * reset != 0 clears the totals afterwards. */
SPARKLING_API int sparkling_set_timing(sparkling_ctx *ctx, int enable);
SPARKLING_API int sparkling_kernel_times(sparkling_ctx *ctx, double *ms_out, int64_t *launches_out,
                                         int n, int reset);

/* Autotuner of the tile shapes of the pair kernels (threads per CTA, i.e.
 * targets held in registers per thread, and the unroll of the repulsion's
 * source loop).  When enabled (the default), the first sparkling_grad /
 * sparkling_energy / sparkling_step call of a new key -- accumulation mode and
 * padded grid-row length for the attraction, accumulation mode for the
 * repulsion -- times every shape on a prefix of the caller's own problem
 * (about 1e11 pairs each; this synchronises the stream) and keeps the fastest
 * for the context.  enable = 0 uses the default shapes for keys not tuned yet,
 * 1 tunes, -1 forgets every choice and tunes again.  Nothing is tuned on a
 * stream that is being captured. */
SPARKLING_API int sparkling_set_autotune(sparkling_ctx *ctx, int enable);

/* Pin the tile shape of one pair kernel for the context's later calls
 * (reproducible timing; the tests run every shape through it), instead of
 * the autotuner's choice.  kernel = SPARKLING_KERNEL_ATTRACTION: variant 0,
 * 1, 2 = 128, 256, 512 threads per CTA (8, 4, 2 targets per thread).
 * kernel = SPARKLING_KERNEL_REPULSION (the symmetric kernel of
 * sparkling_grad, sparkling_energy, sparkling_step and the batched step):
 * variant 0 = 256 threads per CTA (4 targets per lane), 2 sources per lane,
 * targets paired in the 64-bit registers; 1 = 256 threads, 4 sources per
 * lane, targets paired; 2 = 256 threads, 2 sources per lane, the two sources
 * paired; 3 = 128 threads per CTA (8 targets per lane), 2 sources paired
 * (the shape used where nothing is tuned or pinned, e.g. by the batched
 * step).  variant = -1 unpins (the next call of a new key tunes
 * again when the autotuner is on).  sparkling_set_autotune(ctx, -1) unpins
 * both.  Returns SPARKLING_E_INVAL for another kernel or variant. */
SPARKLING_API int sparkling_set_shape(sparkling_ctx *ctx, int kernel, int variant);

/* Text of the tuning trials (pairs/s per shape) and of the choices, NUL
 * terminated, truncated to len bytes. */
SPARKLING_API int sparkling_tuning_report(const sparkling_ctx *ctx, char *buf, int64_t len);

/* Kernel of the energy: H(r) = sqrt(r^2 + eps^2), the regularised norm of
 * Sec. II-C (choice of step size), whose gradient is Lipschitz (constant
 * 1/eps), so that a fixed step proportional to eps converges.  eps = 0 (the
 * default) is the plain norm H(r) = r of the rest of the paper.  Applies to
 * every later sparkling_grad, sparkling_energy, sparkling_energy_backward,
 * sparkling_step, sparkling_step_host and sparkling_step_batched call of the
 * context and to the attraction field (not to sparkling_grad_noalloc, which
 * has no context and always takes eps = 0).  The pair kernels add eps^2,
 * rounded to float, to every squared distance; the energy leaves out the N
 * self pairs (i = j), as F^r does.  Returns SPARKLING_E_INVAL unless
 * 0 <= eps <= 1e3. */
SPARKLING_API int sparkling_set_regularisation(sparkling_ctx *ctx, double eps);

/* Arithmetic of the context's projections (sparkling_project, sparkling_step,
 * sparkling_step_host, sparkling_step_batched, the driver).
 *   SPARKLING_PROJECTION_FP64 (default): the dual FISTA iteration, the primal
 *     map and the step in FP64 for every K dtype; the result is rounded to
 *     K_dtype once.
 *   SPARKLING_PROJECTION_MIXED: for FP32 K with a fixed n_iter, the iteration
 *     runs in FP32 on the displacement e = s - k and the duals (D1 k, D2 k and
 *     the box and pin offsets formed once per shot in FP64, the output
 *     k + e in FP64); FP64 K and converged mode keep the FP64 iteration.
 * Returns SPARKLING_E_INVAL for another mode. */
SPARKLING_API int sparkling_set_projection(sparkling_ctx *ctx, int mode);

/* Device path of the context's sparkling_step and sparkling_step_host calls
 * (SPARKLING_STEP_*).  AUTO (default) takes the one-launch persistent engine
 * for steps of 2^22 samples or more (on the 1e7-sample workload it is ~8 %
 * faster than the kernels in turn, since SFU-bound attraction items and
 * FP32-bound repulsion items share each SM) and the kernels below that;
 * ENGINE takes the engine at every size; KERNELS never.  Steps the engine
 * does not cover (fast summation modes, ACC_FP64_PAIR, converged mode) run
 * on the kernels whatever the setting.  Returns SPARKLING_E_INVAL for
 * another value. */
SPARKLING_API int sparkling_set_step_path(sparkling_ctx *ctx, int path);

/* Budget of the context's bounded device waits (a TMA copy's mbarrier, and,
 * with a multiple of the budget -- four, or more where one pair item of the
 * work list may take longer -- the persistent engine's wait for a
 * trajectory's pair items, which other CTAs may have only just started), in
 * SM clock cycles; cycles < 0 restores the default 4e9 (about 2 s).  A wait that runs past it
 * sets the status bit that makes the call (or the next sparkling_status)
 * return SPARKLING_E_TIMEOUT, and its kernel returns early, leaving its
 * outputs incomplete; the context stays usable.  After a timeout a CTA still
 * waits, with the default budget, for its own copies in flight before it
 * exits.  A small budget is a way to exercise that path; 0 makes every wait
 * that does not succeed at once time out.  Synchronises the device when the
 * context is already in use.  Returns SPARKLING_E_INVAL above 2^40 cycles. */
SPARKLING_API int sparkling_set_wait_budget(sparkling_ctx *ctx, int64_t cycles);

/* Cap on the device memory the context allocates for itself (its workspace,
 * the device copies of sparkling_step_host and the attraction field; the
 * fast-repulsion mesh allocates outside it), in bytes; 0 (the default)
 * removes the cap.  A call whose allocation would take the context past the
 * cap returns SPARKLING_E_NOMEM before anything is launched and leaves the
 * context usable.  Returns SPARKLING_E_INVAL for bytes < 0. */
SPARKLING_API int sparkling_set_memory_limit(sparkling_ctx *ctx, int64_t bytes);

/* Attraction mode of the context's sparkling_grad, sparkling_energy,
 * sparkling_energy_backward and sparkling_step calls (the batched step and
 * sparkling_grad_noalloc always take the direct sum).
 *   SPARKLING_ATTRACTION_DIRECT (default): the direct sum over the grid.
 *   SPARKLING_ATTRACTION_FIELD: the fast summation of Sec. II-C.1 (eq.
 *     attraction_derivative_basic).  The attraction force
 *     E(y) = sum_q rho_q (y - x_q) / |y - x_q| and the attraction potential
 *     phi(y) = sum_q rho_q |y - x_q| of the density are computed exactly (an
 *     FP64 FFT convolution, stored as float) on the cell-centre nodes of the
 *     grid extended by one node per side, (nx+2)(ny+2)(nz+2) nodes, and the
 *     samples take their trilinear interpolation: O(N) work per evaluation
 *     instead of O(N P).  It is an approximation; its error against the
 *     direct sum is measured by the caller, not bounded here.  Samples
 *     outside [lo, hi] take the value of the nearest boundary cell.
 * Returns SPARKLING_E_INVAL for another mode. */
SPARKLING_API int sparkling_set_attraction(sparkling_ctx *ctx, int mode);

/* Repulsion mode of the context's sparkling_grad, sparkling_energy,
 * sparkling_energy_backward, sparkling_step, sparkling_step_host and driver
 * calls (the batched step and sparkling_grad_noalloc always sum every pair).
 *   SPARKLING_REPULSION_DIRECT (default; mesh may be NULL): every pair.
 *   SPARKLING_REPULSION_MESH: the fast summation that replaces the paper's
 *     fast multipole method (Sec. II-C.2), a particle-particle particle-mesh
 *     split of the kernel d/|d|_eps = d/r erfc(r/sigma) + d/r erf(r/sigma):
 *     the first part is summed directly over the pairs closer than
 *     rc = rc_sigmas * sigma (a cell list), the second on the mesh (cubic
 *     B-spline charges, FP32 FFT convolution with a deconvolved, tapered
 *     kernel, interpolation back); the energy the same way with the matching
 *     potential.  Approximate: its error against the direct sum is measured
 *     by the caller.  The kernel spectra are built at the first call that
 *     needs them (blocking; about 384 M^3 bytes of temporary device memory,
 *     M = n_cells + 2g), again when the mesh or the regularisation changes;
 *     the context then keeps about 330 M^3 bytes (spectra, FFT and charge
 *     buffers) plus 80 bytes per sample.  A sample outside the mesh gives
 *     SPARKLING_E_RANGE.  The first evaluation of a sample count sizes the
 *     buffers and waits once for the length of its short-range work list;
 *     later evaluations of that count are asynchronous (the list's length is
 *     read on the device), so after one such call outside any stream
 *     capture they can be captured into a CUDA graph.  A captured call that
 *     would have to size buffers returns SPARKLING_E_INVAL; a graph captured
 *     before a call with another sample count (which resizes them) must be
 *     captured again.
 * Returns SPARKLING_E_INVAL for a bad mode or mesh. */
SPARKLING_API int sparkling_set_repulsion(sparkling_ctx *ctx, int mode, const sparkling_mesh *mesh);

/* Build the node field of `grid`'s density for SPARKLING_ATTRACTION_FIELD
 * and keep it in the context (one field at a time, (n+2)^3 float4 on the
 * device).  Calls in field mode build it themselves when the grid (rho
 * pointer, n, lo, hi) differs from the one kept; call this again after
 * changing the density values in place (or after placing another density
 * of the same shape at the same address).  Allocates temporary FFT buffers of
 * about 40 L^3 bytes, L = the smallest 2,3,5,7-smooth size >= 2n+1 per
 * axis, and blocks until the field is ready.  Must not be called while
 * `stream` is being captured.  Errors: SPARKLING_E_INVAL (bad grid),
 * SPARKLING_E_NOMEM, SPARKLING_E_CUDA (CUDA or cuFFT failure). */
SPARKLING_API int sparkling_attraction_field(sparkling_ctx *ctx, const sparkling_grid *grid,
                                             void *stream);

/* The linear interpolator between resolution levels of Algorithm 1
 * (L_{2d}, Sec. II-E): every shot of d samples becomes 2d samples -- sample
 * n goes to 2n, sample 2n+1 is the midpoint of samples n and n+1, and the
 * last one continues the last segment (a one-sample shot is repeated).
 *   Kc  device [Nc*d][3] of dtype (read only); Kf device [Nc*2d][3] of dtype
 *   (must not overlap Kc).  Arithmetic in double, one rounding to dtype.
 * Asynchronous on `stream`. */
SPARKLING_API int sparkling_upsample(sparkling_ctx *ctx, const void *Kc, void *Kf, int dtype,
                                     int64_t Nc, int64_t d, void *stream);

/* n_git projected-gradient iterations at one resolution (the inner loop of
 * Algorithm 1, eq. proj_grad_descent): K <- Pi_Q(K - eta_t G(K)), where
 * eta_t = sched->eta for the first sched->n_fixed iterations and then the
 * Barzilai-Borwein step eta_t = <s, s> / <s, y>, s = K_t - K_{t-1},
 * y = G(K_t) - G(K_{t-1}) (FP64 reductions on the device), clamped to
 * [eta_min, eta_max]; when <s, y> <= 0 the previous step is kept.
 *   K      device [Nc*Ns][3] of K_dtype, updated in place
 *   proj   constraint set of this resolution (tol <= 0: n_iter FISTA steps)
 *   trace  optional host [n_git]: the step of every iteration
 * Uses the context's attraction mode and regularisation.  Blocks on
 * `stream` (the step is read back after each gradient once Barzilai-Borwein
 * is on); device errors are returned. */
SPARKLING_API int sparkling_optimize(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc,
                                     int64_t Ns, const sparkling_grid *grid,
                                     const sparkling_proj *proj, int acc,
                                     const sparkling_schedule *sched, double *trace, void *stream);

/* Algorithm 1, the multi-resolution SPARKLING: levels l = start_level, ..., 0,
 * level l with Ns / 2^l samples per shot, constraints
 * alpha * alpha_factor^l, beta * beta_factor^l and the pinned sample
 * pin_index / 2^l (floor), n_git iterations of sparkling_optimize, then
 * sparkling_upsample to the next level.  Level 0 is optimised as well
 * (the printed loop stops after the last up-sampling).
 *   K      device buffer of Nc*Ns*3 elements of K_dtype; holds
 *          Nc * (Ns >> start_level) samples on entry, Nc * Ns on exit
 *   proj   the full-resolution constraint set
 *   checkpoint_prefix  NULL, or a path prefix: after each level the result
 *          (before up-sampling) is written to "<prefix>_level<l>.bin" -- a
 *          64-byte header ("SPKLCKPT", int64 version 1, Nc, samples per
 *          shot, level, K_dtype, 16 reserved bytes) and the raw [Nc*Ns_l][3]
 *          array; resume with sparkling_upsample of a checkpoint and
 *          start_level = l - 1
 *   trace  optional host [(start_level + 1) * n_git] steps, level by level
 * Ns must be a multiple of 2^start_level and Ns >> start_level >= 1.
 * Blocks; errors as sparkling_optimize, SPARKLING_E_IO for a checkpoint
 * that cannot be written. */
SPARKLING_API int sparkling_multires(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc,
                                     int64_t Ns, const sparkling_grid *grid,
                                     const sparkling_proj *proj, int acc,
                                     const sparkling_schedule *sched, int32_t start_level,
                                     const char *checkpoint_prefix, double *trace, void *stream);

/* Number of kernels this context has launched since it was created. */
SPARKLING_API int64_t sparkling_launch_count(const sparkling_ctx *ctx);

/* Library version string, e.g. "sparkling-gb300 0.1 sm_103a". */
SPARKLING_API const char *sparkling_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPARKLING_H */
