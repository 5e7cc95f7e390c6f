/*
 * sipf.h -- C ABI of the GB300 SIPF-W step library (libsipf.so).
 *
 * The library advances the 3D u/v/m/w haptotaxis system
 *     u_t + chi div(u grad v) = Du lap u - u + rho(w) u
 *     v_t = -alpha m v
 *     m_t = Dm lap m - beta m + u
 *     w_t = Dw lap w - eta(u) w + gamma v - w,   rho(w) = 2w/(1+w), eta(u) = 2u/(1+u)
 * (paper Eq. haptotaxis-system) with the stochastic interacting
 * particle-field scheme with weighted particles, SIPF-W (paper Alg. 3):
 * u is an empirical measure of P weighted particles, v, m, w live on an
 * H^3 periodic grid (equivalently H^3 Fourier modes, Eq. vmw_hat), and each
 * step does particle-to-grid deposit (Alg. 1), grid-to-particle gather
 * (Alg. 2), the Euler-Maruyama push and mass update (Eq. u_hat_update), the
 * explicit reaction and the spectral diffusion solve (Eq. g_hat_phy,
 * k_q_update).  All arithmetic runs in CUDA kernels on the device the
 * context was created on; there is no CPU fallback.
 *
 * Conventions shared by every call
 *   - Return value: SIPF_OK (0) or a negative SIPF_E* code; the context's
 *     last error message (sipf_last_error) says more.
 *   - `where` selects the memory space of a caller buffer: SIPF_HOST
 *     (pageable or pinned host memory) or SIPF_DEVICE (device memory on the
 *     context's GPU).  Caller buffers are only read/written during the call
 *     (plus the copy it enqueues, completed before the call returns); the
 *     library never keeps a pointer to them.
 *   - Positions cross the ABI as physical coordinates in the box
 *     [origin, origin + L)^3, structure of arrays: x[0..N) then y[0..N) then
 *     z[0..N) (3*N floats).  Fields cross as H^3 float32 arrays indexed
 *     [z][y][x] (x fastest), node (i, j, k) at origin + (i, j, k) h, h = L/H.
 *   - Work is enqueued on the CUDA stream given at creation; calls that
 *     return data synchronise that stream.  A context must be used from one
 *     host thread at a time; distinct contexts are independent.
 *   - Noise: the Brownian increment of particle `id` in step n (n = 1, 2, ...)
 *     is sqrt(2 Du dt) z with z from Box-Muller on the Philox4x32-10 words of
 *     counter (n, 0, id, 0) and key (seed mod 2^32, seed >> 32).  Results
 *     therefore depend only on (initial state, parameters, seed, dt
 *     sequence), not on launch configuration.
 */
#ifndef SIPF_H
#define SIPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIPF_OK            0
#define SIPF_EINVAL       -1   /* invalid argument (value, size, pointer, order of calls) */
#define SIPF_ENOMEM       -2   /* device or host allocation failed                       */
#define SIPF_ECUDA        -3   /* a CUDA runtime call or kernel launch failed            */
#define SIPF_EUNSUPPORTED -4   /* valid request this build does not implement            */
#define SIPF_ENONFINITE   -6   /* a particle position became non-finite (reset to 0)      */
#define SIPF_EINTERNAL    -7   /* a device-side consistency check failed                 */

#define SIPF_HOST   0
#define SIPF_DEVICE 1

/* field selection bits for sipf_fields; fields are written in this order */
#define SIPF_FIELD_U  1u    /* deposited density u_bar of the current particles (Alg. 1) */
#define SIPF_FIELD_V  2u
#define SIPF_FIELD_M  4u
#define SIPF_FIELD_W  8u
#define SIPF_FIELD_GX 16u   /* spectral d v / dx on the nodes (Eq. gradv) */
#define SIPF_FIELD_GY 32u
#define SIPF_FIELD_GZ 64u

#define SIPF_DIFFUSION_IMPLICIT 0  /* 1/(1 + tau R + tau D|k|^2), convergence analysis Sec. 4 */
#define SIPF_DIFFUSION_EXP      1  /* exp(-tau D|k|^2 - tau R), Eq. k_q_update              */
#define SIPF_V_IMPLICIT 0          /* v/(1 + alpha tau m), Sec. 2.3.3                         */
#define SIPF_V_EXPLICIT 1          /* v (1 - alpha tau m), source S of Eq. g_t                */

typedef struct sipf_ctx sipf_ctx;

/* Periodic box [origin, origin + L)^3 with H nodes per axis (paper Sec. 2.1;
 * Omega = [-L/2, L/2]^3 there, origin = -L/2).  H must be a multiple of 8
 * of the form 2^a 3^b up to 512: 8, 16, 24, 32, 48, 64, 72, 96, 128, 144,
 * 192, 216, 256, 288, 384, 432 or 512. */
typedef struct {
    int32_t H;
    double L;
    double origin[3];
} sipf_grid;

/* Model and scheme parameters (paper Eq. haptotaxis-system; all >= 0 and
 * finite).  H0: low-pass cut-off exp(-2 pi^2 |q|^2 / H0^2) of Alg. 3 applied
 * to the m, w spectra and to the v spectrum used for grad v; 0 or >= H is
 * off (the paper's experiments run with it off; the Theorem-overall
 * configuration takes H0 = H^(8/13)).  p2g_order: assignment function of the
 * particle-to-grid transfer, 2 (or 0) the trilinear R_h, 4 the fourth-order
 * star stencil R_h^(4) of Sec. 2.2.1 (32 nodes; negative weights, so u_bar
 * may be negative); the grid-to-particle interpolation is trilinear either
 * way.  reserved must be 0.  sigma >= 0: variance (units of L^2) of the
 * Gaussian kernel K_sigma = N(0, sigma I_3) of Eq. m_reg, which replaces the
 * m source u by K_sigma * u (applied spectrally, exp(-sigma |k|^2 / 2)); the
 * w source keeps u; 0 (the default, as in the paper's experiments) is off. */
typedef struct {
    double chi, Du, Dm, Dw, alpha, beta, gamma;
    int32_t diffusion;   /* SIPF_DIFFUSION_*  */
    int32_t v_update;    /* SIPF_V_*          */
    double H0;
    uint64_t seed;       /* Philox key        */
    int32_t p2g_order;   /* 0 or 2: trilinear, 4: R^(4) */
    int32_t reserved;
    double sigma;        /* K_sigma regularisation of the m source; 0 = off */
} sipf_params;

/* FP64 diagnostics of the current state (Lemma mass, Corollary mass and the
 * positivity lemma of the paper): total particle mass sum a_p, grid mass
 * h^3 sum u_bar, minima of u_bar, v, m, w, and the count of non-finite
 * values in v, m, w and the positions. */
typedef struct {
    double mass_particles, mass_grid, min_u, min_v, min_m, min_w;
    int64_t step;
    double time;
    int64_t nonfinite;
} sipf_diag;

/* Create a context on the current CUDA device for N particles on `grid`.
 * `stream` is a cudaStream_t (NULL = legacy default stream) on which all
 * later work of the context is enqueued.  Allocates all device state
 * (about 110 N + 110 H^3 bytes: two particle buffers with tile buckets and
 * an overflow region of N slots each, fields, spectra).  Errors: SIPF_EINVAL (N < 1 or N >= 2^31,
 * H not supported, L <= 0, a parameter negative or non-finite, diffusion,
 * v_update or p2g_order unknown), SIPF_ENOMEM. */
int sipf_create(const sipf_grid* grid, int64_t N, const sipf_params* params,
                void* stream, sipf_ctx** out);

/* Set the state at t = 0 (paper Alg. 3, initialisation): particle
 * positions x (3*N physical coordinates, SoA; wrapped into the box),
 * masses `mass` (N doubles, > 0, or 0 for a massless tracer), persistent
 * ids `id` (N uint32; NULL means 0..N-1) and the node values of v, m, w
 * (H^3 floats each).  grad v is computed from v by the spectral derivative
 * (Eq. gradv) and the particles are binned by cell.  Resets the step counter
 * and the time to 0.  Errors: SIPF_EINVAL (NULL pointer, bad `where`, a
 * negative or non-finite mass), SIPF_ECUDA. */
int sipf_set_state(sipf_ctx* ctx, const float* x, const double* mass, const uint32_t* id,
                   const float* v, const float* m, const float* w, int where);

/* Enqueue k steps of size dt (paper Alg. 3 loop body, Jacobi ordering:
 * deposit, gather, push and field update all read the state at step n-1).
 * Asynchronous: returns after enqueueing; device-side failures are reported
 * by the next synchronising call.  With k >= 2 on a stream other than the
 * legacy default one and tracing off, pairs of steps are launched as a CUDA
 * graph captured from the context's own launches on the first such call for
 * this dt (kept per context, at most four); the kernels and their arguments
 * are the same, so the results are identical to k single steps.  Errors:
 * SIPF_EINVAL (state not set, dt <= 0, dt > 0.5 -- the positivity lemma's
 * bound -- or k < 0), SIPF_ECUDA. */
int sipf_step(sipf_ctx* ctx, double dt, int64_t k);

/* Copy the fields selected by `mask` (SIPF_FIELD_* bits) into dst, one H^3
 * float array after another in bit order.  SIPF_FIELD_U deposits the
 * current particles (Alg. 1).  Synchronises the context stream and reports
 * any deferred device error.  Errors: SIPF_EINVAL, SIPF_ECUDA, deferred
 * codes. */
int sipf_fields(sipf_ctx* ctx, uint32_t mask, float* dst, int where);

/* Copy the particles in the library's storage order (bucketed by tile of
 * 8^3 cells, tiles in tile-index order, order within a tile unspecified;
 * particles that overflowed their tile's bucket in the last step follow at
 * the end):
 * physical positions x (3*N floats, SoA; may be NULL), masses a = exp(log a)
 * (N doubles; may be NULL) and ids (N uint32; may be NULL).  Synchronises. */
int sipf_particles(sipf_ctx* ctx, float* x, double* mass, uint32_t* id, int where);

/* Raw particle state in storage order: positions in grid units
 * s = (x - origin)/h in [0, H) (3*N floats, SoA), log-masses (N doubles) and
 * ids; any pointer may be NULL.  Synchronises. */
int sipf_particle_state(sipf_ctx* ctx, float* s, double* loga, uint32_t* id, int where);

/* Exclusive prefix sum of the number of particles per cell (H^3 + 1 int32):
 * the offsets of each cell's run if the particles were sorted by cell key.
 * Cells are numbered tile-major: key = tile * 512 + local, tiles of 8^3
 * cells, tile = ((cz/8) T + cy/8) T + cx/8 with T = H/8, local =
 * ((cz%8) 8 + cy%8) 8 + cx%8, cell (cx, cy, cz) = floor(s).  Synchronises. */
int sipf_cell_start(sipf_ctx* ctx, int32_t* cell_start, int where);

/* The canonical particle order: cell_start as sipf_cell_start (may be NULL)
 * and ids (N uint32; may be NULL) = the particles' ids sorted by (cell key,
 * id), a deterministic order for the particle loops of Alg. 1
 * (particle-to-grid) and Alg. 2 (grid-to-particle), which the paper leaves
 * unordered; the run of cell key k is ids[cell_start[k] .. cell_start[k+1]).
 * The step itself never needs this order: its deposit sums integers, so no
 * order of the particles changes u_bar by a bit; this call makes the order a
 * checkable output.  Computed on the device (counting sort by key, then rank
 * by id inside each cell's run); uses the context's free particle buffer as
 * work space, allocates nothing.  Synchronises.  Errors: SIPF_EINVAL (both
 * pointers NULL, bad `where`, no state), SIPF_ECUDA. */
int sipf_canonical_order(sipf_ctx* ctx, int32_t* cell_start, uint32_t* ids, int where);

/* Tuning.  Launch choices that change speed, never results beyond float32
 * rounding: radix_plan selects how the spectral step transforms: 0 or 1,
 * two Stockham plans of each transform length in the plane passes (e.g.
 * 96 = 8 x 4 x 3 or 12 x 8); 2, the per-axis pipeline of transforms held by
 * groups of lanes (H = 64, 128, 256; other sizes take plan 0 instead); the
 * plans' results differ only by float32 rounding;
 * step_blocks_per_sm (0 = the occupancy limit, else at
 * most that many particle-step blocks per SM); bucket capacity = count +
 * count / bucket_slack_div + bucket_slack_add per tile, 8 <= div <= 1024,
 * 0 <= add <= 32 (smaller slack sends more particles to the overflow region;
 * the particle results are bit for bit the same).  The autotuner
 * (paper_2605_20140_gb300/autotune.py) times the candidates on the GPU and
 * writes a table the library reads: sipf_create applies the first line of
 * the table matching its (H, N); the table is the file named by the
 * SIPF_TUNING environment variable, else sipf_tuning.txt next to
 * libsipf.so, read at the first sipf_create (or sipf_tuning_lookup), or one
 * loaded with sipf_tuning_load (NULL: empty table).
 * sipf_set_tuning applies a choice to a context (dropping its captured step
 * graphs; synchronises); sipf_get_tuning reads it back.  sipf_tuning_lookup
 * returns 1 and fills *out when the table has a line for (H, N), else 0.
 * Errors: SIPF_EINVAL (NULL, out of range, unreadable or malformed file). */
typedef struct {
    int32_t radix_plan;
    int32_t step_blocks_per_sm;
    int32_t bucket_slack_div;
    int32_t bucket_slack_add;
} sipf_tuning;
int sipf_set_tuning(sipf_ctx* ctx, const sipf_tuning* tuning);
int sipf_get_tuning(const sipf_ctx* ctx, sipf_tuning* tuning);
int sipf_tuning_load(const char* path);
int sipf_tuning_lookup(int32_t H, int64_t N, sipf_tuning* out);

/* FP64 diagnostics of the current state; synchronises. */
int sipf_diagnostics(sipf_ctx* ctx, sipf_diag* out);

/* Wait for the context's stream and return any deferred device error. */
int sipf_sync(sipf_ctx* ctx);

/* Residual resampling (paper Alg. 4): the particles are replaced by N
 * equal-weight particles.  Particle p (in id order) is copied k_p =
 * floor(a_p / a_0) times, a_0 = (sum a_p) / N, and the remaining
 * N - sum k_p particles are drawn independently with probabilities
 * proportional to the residuals a_p - k_p a_0 (Philox4x32-10, key = seed,
 * counter (step, 1, draw, 0)).  The integer decisions use the masses in
 * 31-bit fixed point relative to the largest, so they are exact; the new
 * particles carry the ids 0..N-1 in the order (copies in order of p, then
 * draws) and the mass a_0 of the exact fixed-point total.  Resamples only when
 * max a_p > ratio * min a_p (ratio <= 0: always); *resampled (may be NULL)
 * receives 1 if it did.  Requires the ids to be a permutation of 0..N-1
 * (true for ids assigned by sipf_set_state with id = NULL and after a
 * resampling).  Synchronises.  Uses about 40 N bytes of work space, allocated
 * on the first call and kept by the context.  Errors: SIPF_EINVAL (no state,
 * ratio not finite, ids not a permutation, all masses zero), SIPF_ENONFINITE
 * (a mass is not finite), SIPF_ENOMEM, SIPF_ECUDA. */
int sipf_resample(sipf_ctx* ctx, double ratio, int32_t* resampled);

/* Ensembles: many independent runs (different grids, particle counts,
 * parameters and seeds) advanced together.  The paper's method is one run;
 * an ensemble is replicas of it with no shared state: each member is an
 * ordinary context on a stream of its own, so the kernels of small members
 * run concurrently on the GPU, and each member's results are bit for bit
 * those of the same run alone.
 *
 * sipf_ensemble_create: count members, member i created as
 * sipf_create(&grids[i], N[i], &params[i]) on a new non-blocking stream owned
 * by the ensemble.  Errors: those of sipf_create (nothing is kept on error).
 * sipf_ensemble_member: member i (for sipf_set_state, sipf_fields, ...;
 * owned by the ensemble; NULL if i is out of range).
 * sipf_ensemble_step: k steps of every member, dt[i] for member i (host
 * array of count doubles); enqueues only.  Errors: SIPF_EINVAL (a member
 * without state, a dt outside (0, 0.5]).
 * Batched steps (mode SIPF_ENSEMBLE_BATCHED, the default): when every member
 * uses the trilinear assignment without the filter or the K_sigma source, has
 * H <= 128, and all members are at the same buffer parity (true for members
 * whose states were set and that were stepped together; at most 256 members),
 * a step of the whole ensemble is one persistent particle-step launch over
 * the concatenated (run, tile-item) work list of all members, one launch
 * planning every member's next step, and each of the three spectral passes
 * once per (grid size, radix plan) group (the members of a group batched, 64
 * per launch; members on radix plan 2 run its passes one after another); pairs
 * of steps are captured once per (dt vector, parity) as a CUDA graph (at most
 * four kept) and replayed.  Otherwise, or in mode SIPF_ENSEMBLE_STREAMS, each
 * member advances on its own stream with its own two-step graph.  Either way
 * each member ends bit for bit where the same run alone ends.
 * sipf_ensemble_set_mode selects the mode (SIPF_EINVAL for anything else);
 * sipf_ensemble_last_path returns the mode the last sipf_ensemble_step used
 * (-1 before the first).
 * sipf_ensemble_sync: waits for all members; returns the first deferred
 * device error.  sipf_ensemble_last_error: message of the last failed call
 * ("" if none).  sipf_ensemble_destroy frees everything (NULL: no-op). */
typedef struct sipf_ensemble sipf_ensemble;
#define SIPF_ENSEMBLE_BATCHED 0
#define SIPF_ENSEMBLE_STREAMS 1
int sipf_ensemble_create(int32_t count, const sipf_grid* grids, const int64_t* N,
                         const sipf_params* params, sipf_ensemble** out);
int sipf_ensemble_set_mode(sipf_ensemble* ens, int mode);
int sipf_ensemble_last_path(const sipf_ensemble* ens);
sipf_ctx* sipf_ensemble_member(sipf_ensemble* ens, int32_t i);
int sipf_ensemble_step(sipf_ensemble* ens, const double* dt, int64_t k);
int sipf_ensemble_sync(sipf_ensemble* ens);
const char* sipf_ensemble_last_error(const sipf_ensemble* ens);
void sipf_ensemble_destroy(sipf_ensemble* ens);

/* Device memory of a context: sipf_context_bytes gives the bytes
 * sipf_create(grid, N, params) will allocate (a negative SIPF_E* code for
 * arguments sipf_create would reject), without touching the GPU;
 * sipf_device_bytes the bytes a context did allocate (the two agree).  Not
 * included: the work space of sipf_resample, allocated on its first call. */
int64_t sipf_context_bytes(const sipf_grid* grid, int64_t N, const sipf_params* params);
int64_t sipf_device_bytes(const sipf_ctx* ctx);

/* Serving with continuous batching: independent runs (requests) submitted at
 * any time, admitted first come first served while their device memory
 * (sipf_context_bytes) fits the budget, advanced together a few steps per
 * scheduling round (each on a stream of its own, pairs of steps replayed as
 * graphs), and released as soon as their results are collected.  A
 * request's results are bit for bit those of the same run alone.  All calls
 * are host calls of one thread.
 *
 * sipf_server_create: budget_bytes > 0.  sipf_server_submit: the run's grid,
 * N, parameters, initial state (host buffers, copied during the call: x
 * 3*N physical coordinates SoA, mass N, v, m, w H^3 each; ids 0..N-1) and its
 * length (steps of dt); *id receives the request id.  Errors: SIPF_EINVAL
 * (NULL, bad dt or steps, arguments sipf_create would reject, a request
 * larger than the whole budget).  sipf_server_advance: admits what fits,
 * enqueues up to `quantum` steps of every running request, marks finished
 * the requests whose last step has completed on the device; *pending (may
 * be NULL) = queued + unfinished requests.  sipf_server_poll: up to
 * `capacity` ids of newly finished requests into ids[]; *count = how many.
 * sipf_server_collect: copies the fields of a finished request (mask and
 * layout as sipf_fields, host buffer) and releases its device memory; mask
 * 0 only releases.  sipf_server_stats: device bytes in use and at most in
 * use so far, queued and admitted-but-uncollected requests.
 *
 * Failures: submit rejects what sipf_create or sipf_set_state would reject
 * (SIPF_EINVAL, including a negative or non-finite mass).  A request whose
 * admission or steps fail later (a CUDA error; device memory short of the
 * budget) is marked failed and stops; it never blocks the queue.  It is
 * reported by sipf_server_poll like a finished one, and sipf_server_collect
 * returns its error code (with sipf_server_last_error saying what failed)
 * and releases it.
 *
 * Device memory: a request's context takes its arrays from a stream-ordered
 * memory pool owned by the server (cudaMallocFromPoolAsync), whose release
 * threshold is the budget, and its stream and event from a free list, so
 * admission and collection call neither cudaMalloc nor cudaFree (which can
 * synchronise the device and stall the requests in flight).
 *
 * sipf_server_set_limit: admit at most max_live requests at a time (0, the
 * default: only the budget limits); 1 serves the requests one at a time.
 * sipf_server_fail_next_admission: fault injection for tests -- the next
 * admission attempt fails with `code` (< 0) before touching the GPU.
 * Errors of both: SIPF_EINVAL. */
typedef struct sipf_server sipf_server;
int sipf_server_create(int64_t budget_bytes, sipf_server** out);
int sipf_server_submit(sipf_server* srv, const sipf_grid* grid, int64_t N,
                       const sipf_params* params, const float* x, const double* mass,
                       const float* v, const float* m, const float* w, double dt,
                       int64_t steps, int64_t* id);
int sipf_server_advance(sipf_server* srv, int64_t quantum, int32_t* pending);
int sipf_server_poll(sipf_server* srv, int64_t* ids, int32_t capacity, int32_t* count);
int sipf_server_collect(sipf_server* srv, int64_t id, uint32_t mask, float* dst);
int sipf_server_stats(const sipf_server* srv, int64_t* in_use, int64_t* peak, int32_t* queued,
                      int32_t* live);
const char* sipf_server_last_error(const sipf_server* srv);
void sipf_server_destroy(sipf_server* srv);
int sipf_server_set_limit(sipf_server* srv, int32_t max_live);
int sipf_server_fail_next_admission(sipf_server* srv, int code);

/* Checkpoint / resume.  The paper has no checkpoint; what is saved is the
 * state of the scheme after step n of Alg. 3: the particles X^n (grid units)
 * with log a^n and ids, the grids v^n, m^n, w^n and the gather array
 * (grad v^n, w^n), plus the step count, time, seed and the deposit's
 * fixed-point reference (which fixes how u_bar is rounded).  A context
 * loaded from the file and advanced k steps gives bit for bit the state of
 * the saved context advanced k steps with the same dt sequence.
 *
 * sipf_save writes the file `path` (overwritten), native byte order, about
 * 20 N + 28 H^3 bytes plus a header; synchronises.  Errors: SIPF_EINVAL
 * (no state set, NULL path, file not writable), SIPF_ENOMEM (host buffer),
 * SIPF_ECUDA, and any deferred device error.
 *
 * sipf_load creates a new context on the current device from the file, with
 * all later work on `stream` (a cudaStream_t, NULL = legacy default), and
 * stores it in *out (the caller destroys it).  Errors: SIPF_EINVAL (NULL
 * argument, unreadable file, wrong magic/version, sizes that do not match
 * the header, payload checksum mismatch, unsupported H), SIPF_ENOMEM,
 * SIPF_ECUDA. */
int sipf_save(sipf_ctx* ctx, const char* path);
int sipf_load(const char* path, void* stream, sipf_ctx** out);

/* The context's grid, particle count, parameters, steps taken and time
 * (host scalars; any output pointer may be NULL).  Does not synchronise.
 * Errors: SIPF_EINVAL (NULL ctx). */
int sipf_describe(const sipf_ctx* ctx, sipf_grid* grid, int64_t* N, sipf_params* params,
                  int64_t* step, double* time);

/* Free all device state of the context (synchronising first); NULL is a
 * no-op. */
void sipf_destroy(sipf_ctx* ctx);

/* Static description of a return code. */
const char* sipf_strerror(int code);

/* Message of the last failed call on the context ("" if none). */
const char* sipf_last_error(const sipf_ctx* ctx);

/* Brownian normals used by the push, for checking the generator: for each
 * i < N, z[i], z[N+i], z[2N+i] are the three standard normals of particle
 * ids[i] in step n with key `seed` (Box-Muller on Philox4x32-10, counter
 * (n, 0, id, 0)); `bits` (4*N uint32, SoA, may be NULL) receives the raw
 * Philox words.  ids, z and bits are device pointers; runs on `stream` and
 * synchronises it.  Errors: SIPF_EINVAL, SIPF_ECUDA. */
int sipf_brownian_normals(const uint32_t* ids, int64_t N, uint32_t n, uint64_t seed,
                          float* z, uint32_t* bits, void* stream);

/* Tracing.  sipf_profile(ctx, 1) starts recording CUDA events (on the
 * context's stream) between the kernel groups of each subsequent step, for
 * at most 4096 steps; sipf_profile(ctx, 0) stops; enabling again clears the
 * record.  Groups, in launch order: 0 particle_step (deposit, gather, push,
 * mass update and binning of all particles), 1 forward_xy, 2 z_multiply,
 * 3 inverse_xy (names from sipf_profile_name); the plan of the next step's
 * bucket layout runs concurrently on a second stream and is not timed.  sipf_profile_read synchronises the stream and writes,
 * for k < n, the summed device time ms[k] (milliseconds) and the number of
 * kernel launches launches[k] over the recorded steps.  Errors: SIPF_EINVAL,
 * SIPF_ECUDA. */
int sipf_profile(sipf_ctx* ctx, int enable);
int sipf_profile_read(sipf_ctx* ctx, double* ms, int64_t* launches, int n);
const char* sipf_profile_name(int k);

/* Allocation-free deposit.  The paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory when they need a
 * density -- code running under another framework's memory budget (whose
 * caching allocator must not see foreign cudaMalloc/cudaFree calls, which
 * also synchronise the device), real-time loops that may not block or fail
 * on allocation, or plug-ins that are handed only pre-allocated buffers.
 * It computes the same particle-to-grid deposit u_bar as sipf_fields with
 * SIPF_FIELD_U, for N particles with physical positions x (3*N floats, SoA,
 * wrapped into the box) and masses `mass` (N doubles, >= 0), into u (H^3
 * floats, [z][y][x]); x, mass and u are device pointers owned by the caller.
 * A particle whose mass is not finite (inf, NaN) or not positive contributes
 * nothing (the context path rejects such masses in sipf_set_state instead).
 * It calls no cudaMalloc, cudaFree or other allocating routine: its integer
 * accumulator is a fixed array in the library's device memory, sized for at
 * most 64^3 nodes, which every GPU that loads the library keeps until the
 * process exits.  Grids with H > 64 are rejected with SIPF_EINVAL, as are
 * NULL pointers, N < 1 or N >= 2^31, and a non-positive or non-finite L.
 * Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without waiting; launch failures return
 * SIPF_ECUDA.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture;
 * the address is kept for the life of the process, so the call must not be
 * used on a device after a cudaDeviceReset of it in the same process.
 * Every call on a device shares the one array and clears it before use, so
 * calls whose work overlaps on the GPU (different streams, or threads
 * without ordering) race and corrupt each other's results; order them on
 * one stream. */
int sipf_deposit_noalloc(const sipf_grid* grid, const float* x, const double* mass, int64_t N,
                         float* u, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SIPF_H */
