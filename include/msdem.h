/*
 * msdem.h -- C-ABI of libmsdem.so, the GB300 (sm_103a) hot path of the
 * particle-continuum sea-ice model "msDEM" of Deng, Stechmann & Chen
 * (arXiv 2303.07819).
 *
 * The model: one doubly periodic discrete-element model (DEM) of disk floes
 * per coarse cell (Sec. 3.1), whose per-cell moments drive a Lax-Friedrichs
 * solution of the moment equations (Eq. 2.26 with the Oseen form Eq. 3.3,
 * Sec. 3.2), fed back gradually into the floes (Sec. 3.3, Eqs. 3.4-3.7) on
 * the schedule of Algorithm 1; beside it the un-localised full-domain DEM the
 * paper compares against (Sec. 4).
 *
 * Conventions for every entry point
 *  - Units are SI (m, s, kg) unless the caller picks consistent non-dimensional
 *    values, as the paper's Sec. 4 scenarios do.
 *  - Pointers marked "host" are ordinary CPU memory owned by the caller; the
 *    library copies from or into them before returning.  The library never
 *    keeps a caller pointer.
 *  - Device memory is allocated by the library (cudaMalloc) in ms_init and
 *    released by ms_free.  One model handle belongs to one host thread at a
 *    time; calls on different handles are independent.
 *  - Every call is synchronous: when it returns, its work on the model's
 *    stream has finished and its outputs are valid.
 *  - Return value: MS_OK (0) or a negative MS_ERR_* code; ms_last_error()
 *    gives a message for the calling thread's last failure.
 */
#ifndef MSDEM_H
#define MSDEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MS_NMOM 12   /* moment columns per cell, see ms_moments */
#define MS_NWIN 5    /* accumulated-window columns, see ms_coupling */
#define MS_MAX_MODES 16

enum {
    MS_OK = 0,
    MS_ERR_ARG = -1,       /* invalid argument: sizes, NaN, overlap, call order of dt */
    MS_ERR_CUDA = -2,      /* a CUDA call failed (message says which) */
    MS_ERR_UNSTABLE = -3,  /* non-finite floe state, or an overlap deeper than r_min / 2 */
    MS_ERR_TIMEOUT = -4,   /* a bounded device-side wait ran out */
    MS_ERR_STATE = -5      /* call not valid in the model's current state */
};

enum { MS_FP32 = 0, MS_FP64 = 1 };

/* Coarse grid over the doubly periodic domain [0, Lx) x [0, Ly): nx x ny
 * cells of side (Lx/nx, Ly/ny); cell c = iy * nx + ix.  Each cell carries its
 * own periodic DEM (Sec. 3.1).
 * nens > 1: an ensemble of nens independent realizations of that domain
 * (same forcing, own floes), batched in one model.  Realization e occupies
 * y in [e Ly, (e + 1) Ly) (floe y coordinates, ms_get_floes and cell indices
 * c = (e ny + iy) nx + ix follow this stacking); each realization is periodic
 * on its own, in the coarse step as in the ocean forcing, and takes its own
 * number of Lax-Friedrichs substeps, so the result is that of nens separate
 * models.  An ensemble has no truth DEM (ms_truth_* return MS_ERR_STATE).
 * 0 or 1: one realization. */
typedef struct ms_grid {
    int32_t nx, ny;
    double Lx, Ly;
    int32_t nens;
    /* Boundary in x: 0 periodic (above); 1 or 2 rigid walls at x = 0 and
     * x = Lx, periodic in y (Sec. 4.4).  With walls the floes must start
     * inside [0, Lx); the truth DEM is not periodic in x and a floe touching a
     * wall gets the contact law of Eq. (2.2) against it (the wall taken as a
     * floe at rest of unbounded radius and at least the floe's thickness:
     * overlap d - r with d the centre's distance to the wall, chord
     * 2 sqrt(r^2 - d^2)); a centre that would pass a wall stays on it.  The
     * coarse Lax-Friedrichs step has ghost cells beyond the walls: walls = 1
     * holds them at zero (zero Dirichlet on concentration, momentum and
     * angular momentum, as Sec. 4.4 states it); walls = 2 mirrors the
     * boundary cell (normal momentum and velocity reversed), an impermeable
     * wall that keeps the coarse mass.  Each cell's own DEM stays doubly
     * periodic (Sec. 3.1).  Any other value is MS_ERR_ARG. */
    int32_t walls;
} ms_grid;

/* Floe state (Sec. 2.1): centre (x, y) in domain coordinates, angle theta,
 * velocity (u, v), spin omega, radius r, thickness h.  Host arrays of n
 * doubles each.  A floe belongs to the cell holding its centre (half-open
 * cells) for the whole msDEM run. */
typedef struct ms_floes {
    int64_t n;
    const double *x, *y, *theta, *u, *v, *omega, *r, *h;
} ms_floes;

/* Forcing, material constants and coupling parameters.
 *  ocean:  u_o = (uo_x, uo_y) + curl of psi, psi = sum_m A_m sin(2 pi (kx_m X/Lx
 *          + ky_m Y/Ly) + phi_m); modes = host [n_modes][4] = (A, kx, ky, phi),
 *          kx, ky integers; plus velocity modes for compressible currents
 *          (the currents of Secs. 4.2-4.3): u_o += sum_m (Au_m, Av_m)
 *          cos(kx_m X + ky_m Y + phi_m), vmodes = host [n_vmodes][5] = (Au,
 *          Av, kx, ky, phi), kx, ky real (rad per unit length; the current need
 *          not be periodic), curl -(Av kx - Au ky) sin(.) per mode;
 *          n_modes + n_vmodes <= MS_MAX_MODES.  Drag Eq. (2.1c-d):
 *          Cd rho_o pi r^2 (u_o - v)|u_o - v| and Cd rho_o pi r^4 (curl/2 - w)|.|.
 *  wind:   (wind_x, wind_y) rotated by 2 pi t / wind_period (0: constant);
 *          drag Ca rho_a pi r^2 (u_a - v)|u_a - v|, no wind torque.
 *  ice:    mass rho_ice pi r^2 h; inertia m r^2 (inertia_half = 1: m r^2 / 2).
 *  contact (Eq. 2.2): normal c (h_min/h_ref) (E delta + eta v_n), never
 *          attractive; tangential c (h_min/h_ref) G v_t capped at mu |normal|.
 *  coupling (Algorithm 1): couple = 1 runs the coarse Lax-Friedrichs step every
 *          N0 fine steps and n_t-step gradual updates; 0 runs the cells'
 *          DEMs alone.  N0 % n_t == 0.
 *  precision: MS_FP32 (floe state and forces in FP32, positions as 32-bit
 *          fixed point of the periodic cell; moments and coarse solve in FP64)
 *          or MS_FP64 (everything in FP64). */
typedef struct ms_forcing {
    double uo_x, uo_y;
    int32_t n_modes;
    const double *modes;
    double rho_o, Cd, rho_a, Ca;
    double wind_x, wind_y, wind_period;
    double rho_ice, E, G, eta, mu, h_ref;
    int32_t inertia_half;
    int32_t couple, N0, n_t;
    int32_t precision;
    int32_t n_vmodes;
    const double *vmodes;
} ms_forcing;

typedef struct ms_model ms_model;

/* Create a model on the current CUDA device: validates the inputs, uploads
 * them, assigns floes to cells and builds the per-cell floe layout by a
 * counting sort on the device (floes of a cell contiguous, in the caller's
 * order), and keeps a second copy of the state for the truth DEM.
 * Rejects (MS_ERR_ARG): nx, ny < 1; non-positive or non-finite sizes; n < 0;
 * non-finite floe values; r <= 0 or h <= 0; 2 r_max >= half the smaller cell
 * side (the periodic minimum image would be ambiguous); a cell with more than
 * 4096 floes (FP32) or 2048 (FP64); non-integer wave numbers.
 * *out receives the handle (NULL on failure). */
int ms_init(ms_model **out, const ms_grid *grid, const ms_floes *floes,
            const ms_forcing *forcing);

/* Advance the msDEM model by nsteps fine steps of dt (forward Euler,
 * Sec. 3.1), running the coarse step and the gradual updates of Algorithm 1
 * when couple = 1.  The first call fixes dt; a later call with another dt
 * returns MS_ERR_ARG.  nsteps = 0 is a no-op.  Full coarse intervals replay a
 * captured CUDA graph.  MS_ERR_UNSTABLE if the state became non-finite or the
 * coarse step needed more Lax-Friedrichs substeps than it holds; overlaps
 * deeper than half the smaller radius are counted (ms_info entry 13). */
int ms_step(ms_model *m, double dt, int64_t nsteps);

/* As ms_step, but only enqueues the work on the model's stream and returns;
 * errors raised by the kernels surface at the next synchronous call (ms_sync,
 * ms_moments, ...).  For callers that time or overlap the step themselves. */
int ms_step_async(ms_model *m, double dt, int64_t nsteps);

/* Wait for the model's stream and report errors raised by its kernels. */
int ms_sync(ms_model *m);

/* Moments of the current msDEM state per cell, host out[ncell][MS_NMOM]
 * (FP64): 0 n, 1 sum m, 2 sum m u, 3 sum m v, 4 sum I, 5 sum I omega,
 * 6 sum pi r^2, 7 sum m u^2, 8 sum m v^2, 9 sum Fdrag_x, 10 sum Fdrag_y,
 * 11 sum Tdrag (drag of the last step; zero before the first).
 * Mass density rho = col1 / A_c, concentration = col6 / A_c (Sec. 2.3, 4.1). */
int ms_moments(ms_model *m, double *out);

/* Floe state of the msDEM model, host out[8][n] in the caller's original
 * floe order, domain coordinates: x, y, theta, u, v, omega, r, h. */
int ms_get_floes(ms_model *m, double *out);

/* Replace the msDEM floe state (same n, every floe in the cell it started
 * in; MS_ERR_ARG otherwise) from host arrays.  The coupling state is kept.
 * The arrays go to the device (64 bytes per floe) -- straight from the
 * caller's memory when all eight are page-locked (cudaHostAlloc,
 * cudaHostRegister), else copied (all host cores) into pinned memory array by
 * array, each array's transfer overlapping the next one's copy -- and are
 * checked and converted to the cell layout there: a non-finite value, r <= 0 or h <= 0, or a floe
 * outside its cell fails with MS_ERR_ARG naming the smallest such index (the
 * value checks first), and the model's state is then left as it was.  The
 * caller's arrays are only read, and not used after the call returns. */
int ms_set_floes(ms_model *m, const ms_floes *floes);

/* Coupling state, host arrays (any may be NULL): q[4][ncell] coarse solution
 * (rho, rho u, rho v, P_omega per unit area), targets[4][ncell] of the
 * gradual update (radius scale, du, dv, domega), window[MS_NWIN][ncell]
 * sums over the current coarse step of (mean u, mean v, sum Fdrag_x,
 * sum Fdrag_y, sum Tdrag), flags[3] = (coarse state set, targets set, steps). */
int ms_coupling(ms_model *m, double *q, double *targets, double *window,
                int64_t *flags);

/* The un-localised truth DEM (Sec. 4): the same floes on the whole periodic
 * domain, advanced on the library's own copy (rebinned every step by a GPU
 * counting sort).  Same dt rule as ms_step. */
int ms_truth_step(ms_model *m, double dt, int64_t nsteps);

/* Truth floes binned by the coarse cell holding their centre; same columns
 * as ms_moments. */
int ms_truth_moments(ms_model *m, double *out);

/* Truth floe state, host out[8][n], original order, domain coordinates. */
int ms_truth_get_floes(ms_model *m, double *out);

/* Use this CUDA stream (a cudaStream_t passed as void*) for all later work;
 * NULL selects the library's own stream.  The caller keeps the stream alive
 * while the model uses it. */
int ms_set_stream(ms_model *m, void *stream);

/* Autotune the msDEM cell kernel on the model's current state: times each
 * launch variant (pair search, threads per block, bin width) out of place
 * (the state is not changed) and keeps the fastest.  FP32 candidates are
 * timed over `reps` whole coarse intervals (ms_time_kernel which = 2), FP64
 * ones over `reps` single steps.  best_ms (host, may be NULL) receives the
 * fastest mean time per fine step. */
int ms_autotune(ms_model *m, double dt, int32_t reps, double *best_ms);

/* Choose the cell-kernel launch by hand: variant 0 = brute-force pairs within
 * the cell, 1 = binned pair search (FP32 only); threads per block 64, 128 or
 * 256 (variant 0 and FP64; the size classes of variants 1-4 set their own);
 * persistent = 1 runs a grid of resident blocks that take cells from a work
 * queue (largest cells first); bin_beta = bin side in units of the cell's
 * mean floe spacing (variants 1-4); variant 2 = binned, one warp per cell of
 * 33 to 256 floes, a block per larger cell, and cells of at most 32 floes
 * packed several to a warp (a lane per floe, the floe kept in registers for a
 * whole coarse interval), the size classes on concurrent streams; variant 3 =
 * variant 2 with each warp cell also kept in shared memory for a whole
 * coarse interval (one launch per interval instead of one per fine step; the
 * per-step arithmetic of variant 2); variant 4 (the default) = variant 2
 * with per-floe contact candidate lists kept across steps (pairs within
 * r_l + r_j + skin, rebuilt by the binned search at the start of every
 * gradual-update period, whenever a floe has moved half the skin, and
 * after a list overflowed), cells of up to 640 floes warp-per-cell and
 * larger ones block-per-cell; variant 5 (the default) keeps every cell of up
 * to 1024 floes resident in registers for a whole run of steps (one launch
 * per coarse interval on the graph path): a floe per thread of a 256-thread
 * block that several small cells share, 2 or 4 floes per thread for cells of
 * 257-512 or 513-1024 floes, blocks taking groups of cells from a work queue
 * largest first; contact candidates from per-floe skins, summed in
 * ascending partner order; larger cells run the block list kernel step by
 * step (see ms_set_resident for its tunables).  Variants 2-5 give the same
 * results whether an interval runs in one launch or step by step.  With a
 * closure attached, the cells that take the closure for an interval hold no
 * floes in their group for that interval (variants 2-5 skip them).
 * MS_ERR_ARG for an unsupported choice. */
int ms_set_launch(ms_model *m, int32_t variant, int32_t threads, int32_t persistent, double bin_beta);

/* Mean device time (ms, CUDA events on the model's stream) of `reps`
 * out-of-place runs on the current state, which the runs do not change:
 * which = 0, one fine step of the msDEM cell kernels; 1, one truth step;
 * 2, the cell kernels of one whole coarse interval (N0 fine steps from the
 * interval's first step, no coarse step). */
int ms_time_kernel(ms_model *m, int32_t which, double dt, int32_t reps, double *mean_ms);

/* Tunables of launch variant 5 (the default for FP32): each floe's skin --
 * how far it may move before its cell group searches for contact candidates
 * again -- is its speed (plus what the coming gradual updates add) times
 * skin_steps fine steps (1 .. 1000); cells of at most 256 floes share a
 * block of 256 threads, a floe per thread, up to block_floes (32 .. 256)
 * floes in all; a larger cell has a block of its own.  Floes do not depend
 * on skin_steps, block_floes or the other cells of the model, and
 * neither do the moments: the per-cell sums are exact fixed-point integer
 * sums (each value relative to the largest binary exponent of its cell and
 * column), whichever cells share a block.  ms_autotune chooses both;
 * ms_info entries 16 and 17 report them.  MS_ERR_ARG outside the ranges. */
int ms_set_resident(ms_model *m, double skin_steps, int32_t block_floes);

/* Model facts, host out[21] (int64): 0 n, 1 ncell, 2 largest cell, 3 precision,
 * 4 kernel variant, 5 threads per block, 6 bin width (per mille of the mean
 * floe spacing), 7 cell-kernel launches per coarse interval (msDEM, whole
 * intervals, no coarse step),
 * 8 kernels per coarse step, 9 kernels per truth step, 10 steps done,
 * 11 truth steps done, 12 graph replays so far, 13 contacts seen deeper than
 * half the smaller radius, 14 persistent launch, 15 LF substeps of the last
 * coarse step, 16 skin horizon of variant 5 in thousandths of a fine step,
 * 17 floes per block of small cells of variant 5, 18 ranks of a sharded
 * grid (0: not sharded), 19 this model's rank, 20 cells it owns. */
int ms_info(ms_model *m, int64_t *out);

/* ---- sharded grids (Sec. 3.1's processor grid of cell blocks, one rank per
 * GPU).  Between coarse steps a cell's DEM touches only its own floes
 * (Algorithm 1), so a rank's model holds the floes of its own cells and the
 * ranks meet once per coarse interval: each packs the coarse inputs of its
 * cells (MS_SHARD_NCOL doubles per cell: moment columns 1-5, then the five
 * window sums, the only DEM data the coarse step reads), every rank gathers
 * all ranks' rows and takes the whole grid's coarse step itself.  That step
 * is the same computation on the same inputs on every rank, so the floes
 * and moments of a rank's cells equal those of the unsharded model bit for
 * bit, in FP64 and in FP32 with launch variant 5 (whose results do not
 * depend on which cells share a block, see ms_set_resident). */
#define MS_SHARD_NCOL 10

/* The cell (j * nx + i, rows j of every realization stacked in y) that
 * ms_init assigns each floe to: each coordinate wrapped into the periodic
 * domain, then the half-open cell holding it -- computed by ms_init's own
 * kernel on the current CUDA device (temporary device memory, freed before
 * returning).  floes: host arrays (only x and y are read); cell_out: host,
 * floes->n int32.  MS_ERR_ARG for a bad grid, NULL arrays or a non-finite
 * position; MS_ERR_CUDA if the device work fails. */
int ms_floe_cells(const ms_grid *grid, const ms_floes *floes, int32_t *cell_out);

/* The model's floe layout: off (host, ncell + 1 int32) the first stored
 * floe of each cell (off[ncell] = n), orig (host, n int32) the caller's
 * index of each stored floe -- the cells' floes in the caller's order.
 * Either may be NULL. */
int ms_layout(ms_model *m, int32_t *off, int32_t *orig);

/* Exchange of a sharded model's coarse inputs, called by ms_step and
 * ms_step_async on the calling thread at each coarse step, after the rank's
 * rows have been packed into its send buffer on `stream` (the model's
 * cudaStream_t).  It must leave every rank's send buffer in recv, rank r's
 * rows at r * max_cells .. (see ms_shard_buffers), ordered before later work
 * on `stream`: an all-gather enqueued on that stream (NCCL), or a
 * synchronous copy after synchronizing it.  Returns 0, non-zero on failure. */
typedef int (*ms_exchange_fn)(void *ctx, void *stream);

/* Make m rank `rank` of `nranks` ranks: rank r owns the cells
 * cells[rank_off[r] .. rank_off[r + 1]) (host arrays, caller-owned, copied:
 * rank_off [nranks + 1] from 0, non-decreasing, up to the number of cells;
 * cells a permutation of all cells).  m must hold floes of its own cells only
 * (build it from the floes that ms_floe_cells places there; its cells may
 * be empty).  fn(ctx, stream) is the exchange (ms_exchange_fn), called once
 * per coarse step of a coupled model.  After a failed exchange the model
 * stands at the end of an interval without its coarse step and ms_step
 * returns MS_ERR_STATE from then on.  ms_moments of a sharded model: its own
 * cells' rows; other cells hold zeros but in columns 1-5, which hold the
 * last exchange's values.  A sharded model runs no closure
 * (ms_closure_attach and ms_closure_collect return MS_ERR_STATE).
 * MS_ERR_ARG: bad layout, fn NULL, a floe in a cell of another rank;
 * MS_ERR_STATE: already sharded, or a closure attached. */
int ms_set_shard(ms_model *m, int32_t nranks, int32_t rank, const int32_t *rank_off, const int32_t *cells,
                 ms_exchange_fn fn, void *ctx);

/* The exchange buffers of a sharded model, device memory owned by the model
 * (valid until ms_free): send [max_cells][MS_SHARD_NCOL] FP64, rows past the
 * rank's own cells zero; recv [nranks * max_cells][MS_SHARD_NCOL] FP64;
 * max_cells the largest number of cells a rank owns.  Outputs may be NULL.
 * MS_ERR_STATE if m is not sharded. */
int ms_shard_buffers(ms_model *m, double **send, double **recv, int32_t *max_cells);

/* Per-cell moments of a floe set held in the caller's device memory, computed
 * without allocating any memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc while they run, such as
 * a host code that reserves all its device memory up front and forbids
 * allocation inside its time loop, or a framework whose allocator already owns
 * the device memory.  It bins the floes by the coarse cell holding their
 * centre and writes out[ncell][MS_NMOM] with the columns of ms_moments, in
 * ascending floe order within each cell.  Cells are assigned as ms_init
 * assigns them: each coordinate is first wrapped into the periodic domain
 * (X - Lx floor(X / Lx); y over the nens stacked realizations), then falls in
 * the half-open cell [i dX, (i + 1) dX); so x = Lx lands in cell 0 and
 * x = -dX in the last column.
 * Inputs (device, FP64, n each, caller-owned): x, y in domain coordinates,
 * u, v, omega, r, h, and fd = [3][n] per-floe drag (Fx, Fy, torque; zeros if
 * there is none); mass rho_ice pi r^2 h, inertia m r^2 (inertia_half = 1:
 * m r^2 / 2).  out is device memory for ncell * MS_NMOM doubles.
 * Working memory is one fixed device array compiled into the library (about
 * 2.2 MB on every device that loads it, held until exit): at most 262144
 * floes and 16384 cells; larger inputs return MS_ERR_ARG.  Every call looks
 * the array's device address up on the current device
 * (cudaGetSymbolAddress), so the call works on whichever device is current
 * and after a context was torn down and created again.  All calls on a device
 * share that array and each call clears what must start at zero, so calls
 * whose work overlaps on the GPU (from different host threads or streams)
 * corrupt each other's results.
 * The work runs on `stream` (NULL: the legacy default stream) and the call
 * waits for it before returning. */
int ms_cell_moments_noalloc(const ms_grid *grid, double rho_ice, int32_t inertia_half, int64_t n,
                            const double *x, const double *y, const double *u, const double *v,
                            const double *omega, const double *r, const double *h, const double *fd,
                            double *out, void *stream);

/* ---- learned closure (not in the paper: a learned model of the bulk feedback)
 * A 16 -> 128 -> 128 -> 128 -> 4 MLP, tanh hidden units:
 *   xh = (x - mu_x)/sd_x, h1 = tanh(W1 xh + b1), h2 = tanh(W2 h1 + b2),
 *   h3 = tanh(W3 h2 + b3), yh = W4 h3 + b4, y = mu_y + sd_y yh,
 * trained on the mean-squared error of yh against (y_target - mu_y)/sd_y with
 * Adam (beta 0.9, 0.999, eps 1e-8).  Products run on BF16 tensor cores with
 * FP32 accumulation; master weights, biases and Adam state are FP32.
 * Packed parameter layout (35,716 floats): W1[128][16], b1[128], W2[128][128],
 * b2[128], W3[128][128], b3[128], W4[4][128], b4[4] (W[out][in]).
 * Features x (16 per sample) and targets y (4) are FP32, sample-major. */
typedef struct ms_mlp ms_mlp;

/* Create a network from host params (packed) and norm = host
 * [mu_x(16), sd_x(16), mu_y(4), sd_y(4)] (sd > 0); max_batch = largest batch
 * of any later call (1 .. 2^22). */
int ms_mlp_create(ms_mlp **out, const float *params, const float *norm, int32_t max_batch);

/* Input and output normalisation of a training set, computed on the
 * device: host X[n][16] and Y[n][4] (FP32, sample-major, only read) ->
 * host norm[40] = [mu_x(16), sd_x(16), mu_y(4), sd_y(4)], the per-column
 * mean and population standard deviation (sums in FP64, fixed order, so the
 * same inputs give the same result), each sd at least 1e-12: the z-scoring
 * of the loss above, in the layout ms_mlp_create takes.  MS_ERR_ARG for a
 * NULL pointer or n outside [1, 2^31]; MS_ERR_CUDA if a CUDA call fails (the
 * call allocates 80 n bytes of device memory for its duration). */
int ms_mlp_fit_norm(const float *X, const float *Y, int64_t n, float *norm);

/* Forward pass: host X[n][16] -> host Y[n][4] in physical units. */
int ms_mlp_predict(ms_mlp *m, const float *X, int64_t n, float *Y);

/* Gradient of the loss of one batch (n <= max_batch) without updating:
 * host grads in the packed layout, *loss (host, may be NULL). */
int ms_mlp_grad(ms_mlp *m, const float *X, const float *Y, int64_t n, float *grads, double *loss);

/* One Adam step of learning rate lr on one batch (n <= max_batch). */
int ms_mlp_step(ms_mlp *m, const float *X, const float *Y, int64_t n, float lr);

/* Train for `epochs` passes over host data (n <= 2^30 samples) in batches of
 * `batch` (8 .. max_batch; a last batch below 8 samples is left out of the
 * epoch).  The data go to the device once; every epoch gathers them there in
 * a new order -- a keyed permutation of [0, n) (four-round Feistel network
 * with cycle walking, keys drawn from `seed` by SplitMix64) -- and replays one
 * captured CUDA graph of the epoch's batches; the host waits only at the
 * end.  loss_per_epoch (host [epochs], may be NULL) gets each epoch's mean
 * loss.  The call allocates 80 n bytes of device memory for its duration. */
int ms_mlp_train(ms_mlp *m, const float *X, const float *Y, int64_t n, int32_t epochs, int32_t batch, float lr,
                 uint64_t seed, double *loss_per_epoch);

/* Current FP32 parameters, host, packed layout. */
int ms_mlp_get_params(ms_mlp *m, float *params);

/* Forward pass on device buffers X[n][16] -> Y[n][4] on `stream`, without
 * waiting. */
int ms_mlp_forward_device(ms_mlp *m, const float *X, int64_t n, float *Y, void *stream);

/* Engine of every later call on m: 1 (the default) the tcgen05 tensor
 * cores -- inference is one persistent kernel whose CTAs keep the BF16
 * weights in shared memory and run 128 cells per tile through all four
 * layers, each layer a chain of tcgen05.mma with the FP32 accumulator in
 * tensor memory (about 107 KB of shared memory and 128 tensor-memory columns
 * per CTA); a training batch is three kernels: forward, loss and backward per
 * 128-sample tile (210 KB of shared memory and all 512 tensor-memory columns
 * of its SM), the weight and bias gradients as tcgen05 tiles over slices of
 * the batch, and Adam.  0: the tiled mma.sync GEMMs.  Both round the
 * activations to BF16 between layers; their results differ by the order of
 * the FP32 accumulation and by tanh (tanh.approx.f32 on engine 1, tanhf on
 * engine 0, about 2^-11 apart).  Waits for m's work; MS_ERR_ARG for another
 * value. */
int ms_mlp_set_engine(ms_mlp *m, int32_t engine);

/* MS_ERR_TIMEOUT if a bounded wait of a tcgen05 kernel on its tensor-core
 * work ran out since the last check (the affected outputs are not written;
 * the flag is cleared), else MS_OK.  ms_mlp_predict, ms_mlp_grad,
 * ms_mlp_step, ms_mlp_train and the model's step check it. */
int ms_mlp_check(ms_mlp *m);

void ms_mlp_free(ms_mlp *m);

/* Closure plus particle fallback on a coupled FP32 model (not in the paper).
 * mode 0: at the start of each coarse interval every cell's features
 * (rho, mean u, v, omega, variances of u and v, ocean u, v, divergence and
 * curl at the cell centre, wind u, v, the cell's drag per unit mass (x, y)
 * and drag torque per unit inertia at the interval's start -- moment columns
 * 9-11, measured by its DEM or predicted -- and the rate of change of its
 * velocity variance over the interval before) go through `mlp`, which
 * predicts the interval-mean drag force per unit mass (x, y), drag torque per
 * unit inertia and the rate of change of the velocity variance.  A cell runs
 * the closure only when the interval before computed tendencies, its
 * features lie inside box (host [2][16] min, max; NULL: no bound), and the
 * particle path has checked the network on it: after each interval a cell
 * runs its DEM, the network's prediction for that interval is compared with
 * the measured drag, and the cell may take the closure for at most 3
 * intervals after a check whose relative error was at most tol (floor: the
 * drag of 1 cm/s on 1 m ice).  So the first interval after attaching runs
 * every cell's DEM.  Every other cell runs the particle step (the fallback).  A closure cell skips its DEM for
 * the interval: it takes its pending coarse increments at once, its velocity
 * spread follows the predicted variance rate, and the coarse step sees the
 * predicted tendencies.  mode 2: as mode 0, but `mlp` predicts the
 * tendencies less features 12-15 (the drag at the interval's start and the
 * variance rate before), which the closure adds back (train it on
 * Y - X[:, 12:16]).  mode 1: the
 * mean-field drag for every cell (no network).  mode -1: off.  Attach between coarse intervals; `mlp` must
 * outlive the attachment.  Each closure cell counts as N0 cell-steps. */
int ms_closure_attach(ms_model *m, ms_mlp *mlp, int32_t mode, double tol, const float *box);

/* Training data from the particle path: runs nint coarse intervals (from an
 * interval boundary, after the first ms_step call fixed dt) and writes host
 * X[nint][ncell][16] (features at each interval's start; when the interval
 * before the first computed no tendencies, one unrecorded interval runs
 * first) and
 * Y[nint][ncell][4] (the window means of the drag force per unit mass, drag
 * torque per unit inertia, and (variance at the end - at the start) / dT). */
int ms_closure_collect(ms_model *m, int32_t nint, float *X, float *Y);

/* host out[4]: closure cell-intervals so far, cells, mode, coarse intervals done. */
int ms_closure_stats(ms_model *m, int64_t *out);

/* Checkpoint ("save data", Algorithm 1): write the model's whole state to
 * the file at host path `path`: the floes in the model's cell layout, the
 * per-cell moments, window sums, coarse state and gradual-update targets, the
 * device control block (step counters, flags), dt, the launch choice, the
 * FP32 candidate lists, and the truth DEM's state and last drag.  The file
 * holds device-order raw values of this library, each item followed by a
 * hash of its bytes, and is read back only by ms_load.  MS_ERR_STATE while a closure is attached; MS_ERR_ARG if the file
 * cannot be written; MS_ERR_CUDA if reading the device state fails. */
int ms_save(ms_model *m, const char *path);

/* Resume from a checkpoint written by ms_save, into a model made by ms_init
 * with the same grid, boundary, precision, number of floes and floes per
 * cell (and, for an exact resume, the same floes, forcing and laws as the
 * saved model): it then continues as the saved model would have, bit for
 * bit, and restores the saved launch choice.  Every item of the file
 * carries a 64-bit FNV-1a hash of its bytes, and the whole file is read and
 * checked before the model changes: MS_ERR_ARG for a file that is not such a
 * checkpoint, is truncated, has an item whose bytes do not match its hash
 * (the message says "checksum"), or belongs to another model, and the model
 * is then left as it was; MS_ERR_STATE while a closure is attached;
 * MS_ERR_CUDA if writing the device state fails (the model's state is then
 * undefined: load again or call ms_set_floes). */
int ms_load(ms_model *m, const char *path);

/* Release the model's device memory, graphs, events and stream. */
void ms_free(ms_model *m);

/* FP32 FMA throughput of the current device in TFLOP/s (host *tflops; an FMA
 * counts as 2 flops): `reps` timed launches (>= 1) of a kernel whose every
 * thread runs 8 independent FMA chains on all SMs, after one warm-up launch,
 * on a stream of its own (about 2 ms per launch on a GB300).  The
 * denominator of the FP32-pipe fraction of the cell step.  MS_ERR_ARG for
 * reps < 1 or a NULL pointer; MS_ERR_CUDA if a CUDA call fails. */
int ms_probe_fp32(int32_t reps, double *tflops);

/* Message of the calling thread's last failed call ("" if none). */
const char *ms_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
