/*
 * vlasov.h -- C ABI of the GB300 phase-space-conserving Vlasov step.
 *
 * Method (Edelen & Webb, "A Vlasov Algorithm Derived from Phase Space
 * Conservation"): the density is a set of weights w on a tensor-product mesh
 * of basis functions (Sec. III, the basis expansion). Each step every mesh node
 * is pushed as a particle over the step h (Sec. II), and the shifted basis
 * functions are projected back onto the mesh (Sec. III, the Galerkin equation
 * Lambda w_fin = Delta^T w_in and its update w_fin = Lambda^{-1} Delta^T w_in).
 * For the 1-D FEL model the bunching <exp(-i theta)> of the weights drives
 * the field amplitude A (Sec. IV.B, dA/dz = <exp(-i Phi)>).
 *
 * Conventions shared by every call:
 *   - the mesh is row-major [np][nx], x (the coordinate) fastest;
 *     x_i = x0 + i (x1 - x0) / nx is periodic (Sec. IV: periodic coordinates),
 *     p_j = p0 + j (p1 - p0) / (np - 1) is open, end nodes included (Sec. IV:
 *     open momenta; weight pushed beyond p0 or p1 is lost and counted);
 *   - all device memory is owned by the caller: vp_workspace_size() says how
 *     much, vp_create() receives it. The library allocates no device memory.
 *   - every call returns a vp_status; no call throws. vp_last_error() gives a
 *     human-readable reason for the last failure on that simulation.
 *   - calls on one vp_sim are not thread-safe; use one host thread per sim.
 *   - work is enqueued on the stream given in vp_opts.stream (a cudaStream_t,
 *     NULL = legacy default stream); calls that return host data synchronise
 *     that stream.
 */
#ifndef VLASOV_H
#define VLASOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vp_status {
    VP_OK = 0,
    VP_ERR_ARG = 1,         /* invalid argument (NULL pointer, bad size or enum) */
    VP_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
    VP_ERR_WORKSPACE = 3,   /* workspace NULL, misaligned or smaller than required */
    VP_ERR_NONFINITE = 4,   /* a step produced a NaN or infinity (device flag) */
    VP_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (device flag) */
    VP_ERR_STATE = 6,       /* call out of order (e.g. vp_step before vp_set_f) */
    VP_ERR_UNSUPPORTED = 7, /* valid request this build cannot serve (size limits) */
    VP_ERR_CANCELLED = 8    /* a served request was cancelled (vp_server_cancel) */
} vp_status;

/* Deposition kernel = autoconvolution of the basis (Sec. III, Delta). */
enum {
    VP_BASIS_TENT = 0,           /* top-hat basis: tent deposit, Lambda = h I (orthogonal) */
    VP_BASIS_CUBIC_BSPLINE = 1,  /* tent basis: cubic B-spline deposit, Lambda = h tridiag(1/6,2/3,1/6) */
    VP_BASIS_SEPTIC_BSPLINE = 2  /* cubic B-spline basis (smoother basis, Sec. V): septic B-spline
                                    deposit, Lambda = h B7(j - k), 7 bands; scatter kernel */
};

/* Particle pusher for the node flow (Sec. II; examples of Sec. IV). */
enum {
    VP_PUSH_LEAPFROG_KDK = 0,    /* kick-drift-kick, H = p^2/2 + V(x) */
    VP_PUSH_EXACT_ROTATION = 1,  /* linear oscillator advanced analytically (Sec. IV.A) */
    VP_PUSH_FEL_DKD = 2,         /* 1-D FEL, drift-kick-drift with A^{n+1/2} (Sec. IV.B) */
    VP_PUSH_FEL_RK4 = 3          /* 1-D FEL, classical RK4 with the bunching of every stage
                                    (the integrator of Sec. IV.B); runs on the scatter kernel,
                                    not in batches or the server */
};

enum {
    VP_POT_FREE = 0,       /* V = 0 */
    VP_POT_PENDULUM = 1,   /* V = -v_sign cos x (v_sign = -1: the paper's H = p^2/2 + cos x) */
    VP_POT_HARMONIC = 2    /* V = omega^2 x^2 / 2 */
};

enum { VP_FP32 = 0, VP_FP64 = 1 };

/* Treatment of Lambda for the cubic B-spline deposit (Sec. III update equation). */
enum {
    VP_PROJ_GALERKIN = 0,  /* solve Lambda w_fin = Delta^T w_in exactly */
    VP_PROJ_LUMPED = 1     /* Lambda replaced by its row sum h I (no solve) */
};

/* Step-kernel choice. */
enum {
    VP_KERNEL_AUTO = 0,     /* planner's choice (fused when the mesh allows, else tiled) */
    VP_KERNEL_TILED = 1,    /* deposit into shared-memory tiles; Lambda^{-1} in two more passes */
    VP_KERNEL_SCATTER = 2,  /* one thread per source node, global atomics (reference path) */
    VP_KERNEL_FUSED = 3,    /* one pass: p solve + push + deposit + x solve per tile */
    /* the one-pass tile without the x solve (no x halo: fewer source columns per tile), then
     * Lambda_x^{-1} as an exact cyclic pass over whole rows (one more launch, 8 B/node more
     * traffic). Cubic B-spline Galerkin (the FEL's bunching is summed from the deposit and
     * divided by the eigenvalue 2/3 + cos(h_theta)/3 of Lambda_x at exp(-i theta)); not the RK4
     * FEL; FP32 rows up to 32768 nodes, FP64 up to 16384; else VP_ERR_UNSUPPORTED. Not accepted
     * by batches or the server. */
    VP_KERNEL_FUSED_XPASS = 4
};

typedef struct vp_grid {
    int32_t nx, np;        /* nodes along x (>= 4) and p (>= 4) */
    double x0, x1;         /* periodic coordinate range [x0, x1) */
    double p0, p1;         /* open momentum range [p0, p1], end nodes included */
} vp_grid;

typedef struct vp_pusher {
    int32_t kind;          /* VP_PUSH_* */
    int32_t potential;     /* VP_POT_* (leapfrog / rotation) */
    double v_sign;         /* pendulum amplitude and sign, V = -v_sign cos x */
    double omega;          /* harmonic frequency */
    double dt;             /* step h */
    double a0_re, a0_im;   /* FEL: field amplitude A at tau = 0 */
    /* FEL model of Sec. IV.B in full: d theta/dz = delta + eta and the kick
     * amplitude A + i sigma2 <exp(-i theta)> (space charge), taken at the
     * half-drifted phases of each step. 0, 0: the universal-scaling model.
     * Batches and the server take sigma2 = 0 only (VP_ERR_UNSUPPORTED). */
    double delta;
    double sigma2;
} vp_pusher;

typedef struct vp_opts {
    int32_t precision;     /* VP_FP32 or VP_FP64: type of w, the push and the deposit */
    int32_t projection;    /* VP_PROJ_* (cubic B-spline only) */
    int32_t kernel;        /* VP_KERNEL_* */
    int32_t tile_x;        /* tiled kernel: destination tile width (0 = planner) */
    int32_t tile_p;        /* tiled kernel: destination tile height (0 = planner) */
    int32_t history_cap;   /* FEL field-history ring capacity in steps (0 = 4096) */
    void *stream;          /* cudaStream_t for all work of this sim (NULL = default stream) */
} vp_opts;

/* FP64 diagnostics (Sec. IV: sum of weights, entropy; Sec. IV.B: field). */
typedef struct vp_moments_t {
    double sum_w;          /* sum of weights */
    double mass;           /* sum_w * hx * hp */
    double mean_x, mean_p;
    double var_x, var_p, cov_xp;
    double energy;         /* <H> for Hamiltonian pushers; <p> + |A|^2 for the FEL */
    double trapped;        /* mass with H < max V (pendulum), else 0 */
    double entropy;        /* -sum_{w>0} w ln w * hx * hp */
    double neg_mass;       /* sum_{w<0} w * hx * hp */
    double b_re, b_im;     /* <exp(-i x)> of the weights */
    double max_abs_w;
    double lost_mass;      /* deposit pushed beyond the momentum range, times hx hp, cumulative */
    double a_re, a_im;     /* FEL field A at the current step */
    double tau;            /* step * dt */
    int64_t step;
} vp_moments_t;

typedef struct vp_sim vp_sim;

/* Bytes of device workspace vp_create() needs for this configuration. */
vp_status vp_workspace_size(const vp_grid *grid, int32_t basis, const vp_pusher *pusher,
                            const vp_opts *opts, size_t *bytes);

/*
 * Create a simulation. workspace: caller-owned device memory, 256-byte aligned,
 * at least vp_workspace_size() bytes, kept alive until vp_destroy(). The
 * geometry tables of the push are built on the device here (Sec. II flow).
 */
vp_status vp_create(const vp_grid *grid, int32_t basis, const vp_pusher *pusher,
                    const vp_opts *opts, void *workspace, size_t workspace_bytes, vp_sim **out);

/* Set the weights from host memory ([np][nx], dtype VP_FP32 / VP_FP64, n = nx*np).
 * Converts to the sim's precision. Returns once the weights have been read: the
 * caller owns the buffer again. When the stored state is s = Lambda_p w (fused
 * Galerkin plan), dtype equals the sim precision and the buffer is pinned or
 * registered host memory aligned to dtype, the Lambda_p multiply reads it in place
 * (no staging copy); otherwise it is copied to the device first.
 * Resets step, tau, lost mass and A = A0. */
vp_status vp_set_f(vp_sim *sim, const void *host, int32_t dtype, size_t n);
/* Same from device memory (device-to-device on the sim's stream; ordered on that stream only:
 * whatever produced dev on another stream must have finished). */
vp_status vp_set_f_device(vp_sim *sim, const void *dev, int32_t dtype, size_t n);
/* vp_set_f without waiting: the weights (dtype = the sim's precision, else VP_ERR_ARG) are
 * copied to the device by the copy engine on the sim's stream, then Lambda_p is applied; the
 * call returns at once. The host buffer must stay valid and unchanged until the stream has
 * passed the copy (vp_sync, or any later synchronising call). Pinned memory makes the copy
 * truly asynchronous, and lets simulations on other streams overlap their transfers with it. */
vp_status vp_set_f_async(vp_sim *sim, const void *host, int32_t dtype, size_t n);

/* Advance n steps: push + deposit (+ Lambda^{-1}) (+ FEL bunching and field). Asynchronous. */
vp_status vp_step(vp_sim *sim, int32_t n);

/* vp_step, with CUDA events recorded between the phases of every step on the
 * sim's stream. phase_ms[k] (k < nphases <= VP_NPHASES) receives the summed
 * device time of phase k over the n steps: 0 push + deposit (Delta^T w),
 * 1 Lambda^{-1} along x, 2 Lambda^{-1} along p, 3 FEL bunching + field update
 * (or the step counter). Phases a configuration does not run read 0.
 * Synchronises the stream. n <= 4096. */
#define VP_NPHASES 4
vp_status vp_step_profiled(vp_sim *sim, int32_t n, double *phase_ms, int32_t nphases);

/* Copy the weights out ([np][nx] in dtype). vp_get_f synchronises the stream. When
 * the stored state is s = Lambda_p w, dtype equals the sim precision and the buffer
 * is pinned or registered host memory aligned to dtype, the p solve writes the
 * weights into it in place; otherwise they are staged on the device and copied. */
vp_status vp_get_f(vp_sim *sim, void *host, int32_t dtype, size_t n);
vp_status vp_get_f_device(vp_sim *sim, void *dev, int32_t dtype, size_t n);
/* vp_get_f without waiting: the weights (dtype = the sim's precision, else VP_ERR_ARG) are
 * formed on the device and copied to host by the copy engine on the sim's stream; the call
 * returns at once, and the host buffer holds them once the stream has passed the copy
 * (vp_sync). Device-side errors (non-finite weights) are reported by that vp_sync. */
vp_status vp_get_f_async(vp_sim *sim, void *host, int32_t dtype, size_t n);

/* FP64 reductions over the current weights; synchronises. */
vp_status vp_moments(vp_sim *sim, vp_moments_t *out);

/* FEL: A after each step (re, im pairs), oldest first, up to max_entries of the
 * most recent history_cap steps; *count receives the number written. */
vp_status vp_field_history(vp_sim *sim, double *re_im, size_t max_entries, size_t *count);

/* Synchronise the sim's stream and report device-side error flags. */
vp_status vp_sync(vp_sim *sim);

/* Moments of a weight array the caller already holds on the device, with no
 * device allocation. The paper has no counterpart. It serves callers that cannot
 * allocate device memory when they want the diagnostics: an application whose
 * framework allocator already holds the device's memory (a cudaMalloc would fail
 * or make that allocator give its cache back), or a latency-critical loop that
 * must not take the device synchronisation a cudaMalloc or cudaFree can bring.
 * It gives the FP64 moments vp_moments gives (plain FP64 sums in another
 * summation order, so the two agree to rounding). w: device pointer, [np][nx]
 * of dtype VP_FP32 or VP_FP64; lost_mass and a_re_im (host, may be NULL) are
 * copied into the result; stream: cudaStream_t (NULL = default); the call reads
 * the result back to the host and synchronises that stream.
 * The partial sums live in one static device array of this library (about
 * 427 KB per GPU, held until exit); meshes above 2^26 nodes are rejected with
 * VP_ERR_UNSUPPORTED. The first call on a device looks up that array's device
 * address (kept for the process; not valid across a cudaDeviceReset). Calls
 * share the array: calls that overlap on the GPU race. */
vp_status vp_moments_static(const void *w, int32_t dtype, const vp_grid *grid,
                            const vp_pusher *pusher, double lost_mass, const double *a_re_im,
                            vp_moments_t *out, void *stream);

/* What the planner chose for a simulation (read-only; no device work). */
typedef struct vp_plan_info {
    int32_t kernel;           /* VP_KERNEL_FUSED, _FUSED_XPASS, _TILED or _SCATTER */
    int32_t tile_x, tile_p;   /* destination tile (fused, tiled); whole mesh for scatter */
    int32_t ntiles_x, ntiles_p;
    int32_t threads;          /* threads per CTA of the fused step kernel, else 0 */
    int32_t full_row;         /* fused: tiles span the whole x period */
    int32_t state_is_s;       /* 1: the stored state is s = Lambda_p w (fused Galerkin) */
    int32_t launches_per_step;/* kernels one vp_step(1) launches */
    int32_t pad;
    int64_t workspace_bytes;
    int64_t smem_bytes;       /* dynamic shared memory per CTA of the step kernel */
} vp_plan_info;
vp_status vp_plan(const vp_sim *sim, vp_plan_info *out);

/* Redirect later work to another stream (no synchronisation is implied). */
vp_status vp_set_stream(vp_sim *sim, void *stream);

/* Device pointer of the current weights (valid until the next vp_step or vp_set_f), for
 * reading: change the state only through vp_set_f / vp_set_f_device. With the stored state
 * s = Lambda_p w the weights are computed into the buffer the next step writes. */
vp_status vp_state_device(vp_sim *sim, void **dev);

void vp_destroy(vp_sim *sim);
const char *vp_last_error(const vp_sim *sim);
const char *vp_status_string(vp_status status);

/* ---------------------------------------------------------------- batching
 * Many independent simulations (different meshes and pushers, same precision,
 * basis and projection, all on the one-pass kernel) advance together: one
 * launch per step runs one CTA per (simulation, tile) item of a device work
 * list (largest tiles first), then one launch finishes every simulation's step
 * (FEL field update or step counter). Steady-state steps replay a captured CUDA graph. Each
 * simulation's weights, field and moments stay readable through the vp_sim
 * calls; a simulation must not be stepped on its own while a batch step of it
 * is in flight. The batch keeps its tables in caller-owned device memory. */
typedef struct vp_batch vp_batch;

vp_status vp_batch_workspace_size(vp_sim *const *sims, int32_t count, size_t *bytes);
/* sims: count simulations (kept by the caller, alive while the batch exists). */
vp_status vp_batch_create(vp_sim *const *sims, int32_t count, void *stream, void *workspace,
                          size_t workspace_bytes, vp_batch **out);
/* Advance every simulation of the batch n steps (asynchronous). use_graph = 1
 * replays one captured step graph per step (captured on the first call); on the
 * legacy default stream (stream NULL), which cannot be captured, the steps are
 * launched directly instead. */
vp_status vp_batch_step(vp_batch *batch, int32_t n, int32_t use_graph);
/* As vp_batch_step, but simulation k advances min(n, max_steps[k]) steps (0 or less:
 * none): the launches of the n steps skip a simulation's tiles once it has taken its
 * steps, so uneven runs share the launches without splitting the call. max_steps: host
 * array of the batch's count entries, read before the call returns. */
vp_status vp_batch_step_each(vp_batch *batch, int32_t n, const int32_t *max_steps, int32_t use_graph);
vp_status vp_batch_sync(vp_batch *batch);
void vp_batch_destroy(vp_batch *batch);
const char *vp_batch_last_error(const vp_batch *batch);

/* ----------------------------------------------------------------- serving
 * A request loop with continuous batching: requests (mesh, pusher, initial
 * weights, step count) arrive at any time; each scheduling round admits queued
 * requests first-in first-out while their device memory fits the budget (a
 * first-fit allocator over a caller-owned arena), advances all admitted
 * requests together as one batch for a slice of steps, and retires those that
 * are done (moments and, on request, the final weights are kept for the
 * caller; the memory returns to the arena). Requests that cannot join a batch
 * (FP64, or meshes the one-pass kernel does not take) are stepped on their own
 * in the same round. Single host thread; times are host steady-clock seconds. */
typedef struct vp_server vp_server;

typedef struct vp_server_opts {
    size_t budget_bytes;   /* device memory the server may hold (<= arena bytes) */
    int32_t slice_steps;   /* steps per round at most (0 = 50) */
    int32_t max_active;    /* admitted requests at most (0 = 4096) */
    void *stream;          /* cudaStream_t of all server work */
} vp_server_opts;

typedef struct vp_request {
    uint64_t id;           /* caller's identifier, reported back */
    vp_grid grid;
    int32_t basis;
    vp_pusher pusher;
    int32_t precision, projection;
    int32_t steps;         /* steps to advance */
    int32_t keep_f;        /* 1: keep the final weights for vp_server_take_f */
    const void *f0;        /* host initial weights [np][nx], copied by vp_server_submit */
    int32_t f0_dtype;      /* VP_FP32 or VP_FP64 */
} vp_request;

typedef struct vp_result {
    uint64_t id;
    int32_t status;        /* vp_status of the request */
    int32_t batched;       /* advanced inside a batch */
    double t_submit, t_admit, t_finish;
    vp_moments_t moments;  /* at completion */
} vp_result;

vp_status vp_server_create(const vp_server_opts *opts, void *arena, size_t arena_bytes,
                           vp_server **out);
vp_status vp_server_submit(vp_server *srv, const vp_request *req);
/* Run up to rounds scheduling rounds (stops early when nothing is queued or active).
 * *queued and *active (may be NULL) receive the counts after the last round. */
vp_status vp_server_run(vp_server *srv, int32_t rounds, int32_t *queued, int32_t *active);
/* Move up to max finished results into out; *count receives how many. */
vp_status vp_server_poll(vp_server *srv, vp_result *out, int32_t max, int32_t *count);
/* Cancel request id (the first queued or running request with that id). A queued
 * request leaves the queue at once; a running one is retired at the start of the
 * next scheduling round, before any further step, and its device memory returns to
 * the arena. Either way its result arrives through vp_server_poll with status
 * VP_ERR_CANCELLED and the moments of its state when it was retired (a queued
 * request has none); no final weights are kept. The other requests are not
 * affected: each simulation's arithmetic does not depend on the batch it runs in.
 * Returns VP_ERR_STATE if no queued or running request has that id (e.g. it has
 * finished already). Host-side only: no device work, no wait. */
vp_status vp_server_cancel(vp_server *srv, uint64_t id);
/* Final weights of a finished request submitted with keep_f (then released). */
vp_status vp_server_take_f(vp_server *srv, uint64_t id, void *host, int32_t dtype, size_t n);
/* Host steady-clock seconds, the clock of vp_result. */
double vp_server_clock(void);
void vp_server_destroy(vp_server *srv);
const char *vp_server_last_error(const vp_server *srv);

/* ---------------------------------------------------------------- autotuning
 * Chooses the destination tile shape of the step kernel (vp_opts.tile_x,
 * tile_p) by timing candidate shapes on the device: the planner's default and a
 * fixed list of widths and heights (shapes the planner rejects, or plans onto
 * another kernel, are dropped; shapes that plan to the same tiles are timed
 * once). Every
 * candidate is created in the caller's workspace, filled with a constant
 * density, warmed up and timed with CUDA events on opts->stream over at least
 * min_steps steps and min_ms of device time (the better of two runs). The
 * tile shape has no effect on the arithmetic of a node: every candidate
 * computes the same step. batched = 1 times the `count` configurations
 * together, each candidate shape applied to all of them as one vp_batch
 * (FP32, one-pass kernel); batched = 0 tunes count = 1 configuration alone.
 * With batched = 0 and opts->kernel = VP_KERNEL_AUTO, when the planner takes
 * the one-pass kernel, the separate-x-pass plan (VP_KERNEL_FUSED_XPASS) is
 * timed over its own shape list too, and the result's kernel says which won:
 * create the simulation with that kernel and shape.
 * FEL configurations are timed at their A0; the windows grow with |A|.
 * Results are kept in a process-wide cache keyed by the configurations (all
 * grid and pusher fields except A0) and the options, so a second call with
 * the same key times nothing (from_cache = 1). Synchronises opts->stream. */
typedef struct vp_tune_config {
    vp_grid grid;
    int32_t basis;
    int32_t pad;
    vp_pusher pusher;
} vp_tune_config;

typedef struct vp_tune_opts {
    int32_t min_steps;     /* timed steps per candidate, at least (0 = 3) */
    int32_t batched;       /* 1: time the configurations together as one batch */
    int32_t use_cache;     /* 1: read and fill the process-wide cache */
    int32_t pad;
    double min_ms;         /* device time per candidate, at least (0 = 2 ms) */
} vp_tune_opts;

typedef struct vp_tune_result {
    int32_t tile_x, tile_p;      /* chosen shape, as vp_opts.tile_x and tile_p reproduce it */
    int32_t kernel;              /* kernel of that plan (VP_KERNEL_*) */
    int32_t candidates;          /* distinct shapes timed */
    int32_t from_cache;
    int32_t pad;
    double ms_per_step;          /* one step with the chosen shape (batched: the whole batch) */
    double default_ms_per_step;  /* the same with the planner's default shape */
} vp_tune_result;

/* Bytes of device workspace vp_autotune() needs (the largest candidate, all
 * configurations at once when batched, plus a density buffer). */
vp_status vp_autotune_workspace_size(const vp_tune_config *cfgs, int32_t count, const vp_opts *opts,
                                     const vp_tune_opts *topts, size_t *bytes);
/* cfgs: count configurations; opts: precision, projection, kernel, history
 * capacity and stream shared by all (its tile fields are ignored); out: count
 * results (batched: one shape for all, as each configuration plans it). */
vp_status vp_autotune(const vp_tune_config *cfgs, int32_t count, const vp_opts *opts,
                      const vp_tune_opts *topts, void *workspace, size_t workspace_bytes,
                      vp_tune_result *out);
/* Forget every cached tuning result. */
void vp_autotune_clear_cache(void);

#ifdef __cplusplus
}
#endif

#endif /* VLASOV_H */
