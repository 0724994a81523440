/*
 * nemd.h -- C ABI of the GB300 cell-list force evaluation for homogeneous
 * linear flows under Kraynik-Reinelt periodic boundary conditions.
 *
 * Paper: M. Dobson, I. Fox, A. Saracino, "Cell List Algorithms for
 * Nonequilibrium Molecular Dynamics", arXiv:1412.3784.
 *
 * One force evaluation is the call sequence
 *     nemd_set_state(q, t)  ->  nemd_build_cells(variant, rc)  ->  nemd_compute_forces(F, U, W)
 * after a one-time nemd_set_flow(A, L0, M, T) and nemd_set_potential(...);
 * nemd_integrate steps positions and momenta through many such evaluations,
 * and nemd_batch_* evaluates many independent systems at once.
 * Every step runs as CUDA kernels on the context's stream:
 *   set_state      lattice L(t) = exp(A (t mod T)) L0, its inverse, heights, QR  (Sec. 2.1, 2.2)
 *   build_cells    cell grid and neighbour stencil from the deformed metric,
 *                  fractional wrap and counting-sort binning in cell order       (Sec. 4.1, 4.2)
 *   compute_forces cell-pair LJ/WCA force, energy and virial                     (Sec. 3, 5)
 *
 * Conventions
 *   - Matrices are 3x3 row-major.  The COLUMNS of L0 (and of L) are the lattice
 *     vectors v1, v2, v3 (Sec. 2: L = [v1 v2 v3]).
 *   - Positions q are N x 3 float64, Cartesian, any periodic image.
 *   - Pointers may be host or device memory; the library inspects each pointer
 *     (cudaPointerGetAttributes).  Device pointers are used in place and are
 *     read/written asynchronously on the stream.  Host pointers are copied
 *     through library-owned device buffers; a call that writes host outputs
 *     synchronises the stream before it returns.
 *   - The library owns all scratch memory and grows it on demand.  The caller
 *     owns every pointer it passes in; the library never frees them.
 *   - Errors are returned as a nemd_status value (0 = OK).  Errors detected on
 *     the device (a box too small for the cut-off, non-finite coordinates, a
 *     wait that timed out) are deferred: they are returned by nemd_sync() and by
 *     the next call that synchronises.  nemd_last_error() gives a message.
 *   - A context is used by one host thread at a time.
 */
#ifndef NEMD_H
#define NEMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nemd_ctx nemd_ctx;

typedef enum nemd_status {
    NEMD_OK = 0,
    NEMD_ERR_ARG = 1,            /* null pointer, N < 0, bad enum value, rc <= 0 ...      */
    NEMD_ERR_NOT_SL3Z = 2,       /* M is not an integer matrix with det M = 1 (Sec. 2.2) */
    NEMD_ERR_NOT_KR = 3,         /* |exp(T A) L0 - L0 M| > 1e-9 |L0| (Eq. kr)           */
    NEMD_ERR_TRACE = 4,          /* |tr A| > 1e-12 |A|: the flow must be incompressible  */
    NEMD_ERR_BOX_TOO_SMALL = 5,  /* a cell count c_i or l_i is 0: face width < rc        */
    NEMD_ERR_ORDER = 6,          /* calls out of order (e.g. forces before build_cells)  */
    NEMD_ERR_CUDA = 7,           /* a CUDA runtime call failed                           */
    NEMD_ERR_NONFINITE = 8,      /* NaN or Inf in the positions                          */
    NEMD_ERR_TIMEOUT = 9,        /* a bounded device wait ran out                        */
    NEMD_ERR_CAPACITY = 10,      /* a device table outgrew its bound                     */
    NEMD_ERR_NOMEM = 11,         /* device or host allocation failed                     */
    NEMD_ERR_UNSUPPORTED = 12    /* option or mode not available                         */
} nemd_status;

typedef enum nemd_variant {
    NEMD_DS = 0,              /* dynamic size cell list, Sec. 4.1                          */
    NEMD_DO = 1,              /* dynamic offset cell list, Sec. 4.2                        */
    NEMD_AUTO_HEURISTIC = 2,  /* per step, the variant with the smaller neighbourhood
                                 volume V_DS = 27 V / (c1 c2 c3) versus
                                 V_DO = avg r11 r22 r33 / (l1 l2 l3)  (Sec. 5.1, 5.2)     */
    NEMD_AUTO_LEARNED = 3     /* per step, the variant and cell factor of the learned
                                 selector (nemd_model_train / nemd_model_load); the
                                 heuristic when no model is set                         */
} nemd_variant;

typedef enum nemd_potential {
    NEMD_LJ = 0,   /* 4 eps [(sigma/r)^12 - (sigma/r)^6], optionally shifted to 0 at rc   */
    NEMD_WCA = 1   /* the same with rc = 2^(1/6) sigma and the shift on (Sec. 5 runtime)   */
} nemd_potential;

typedef enum nemd_option {
    NEMD_OPT_PRECISE = 1,       /* 1: accepted pairs are re-evaluated in float64 (energy
                                   and virial to ~1e-13); 0 (default): float32 pair math */
    NEMD_OPT_RECORD_PAIRS = 2,  /* > 0: capacity of the pair record (verification mode)   */
    NEMD_OPT_KERNEL = 3,        /* force kernel: 0 plain (one thread per particle),
                                   1 grouped (a group of lanes per chunk of a cell row,
                                   queued force evaluation; N <= 2^21), 2 warp (one chunk
                                   of 32 per warp, neighbour rows staged in shared
                                   memory), 3 warp with half neighbourhoods (each
                                   unordered pair evaluated once, partner forces added
                                   with atomics: F is not bitwise reproducible from run
                                   to run; pair records use kernel 2), 4 row (one chunk of
                                   32 per warp, each lane testing only its own window
                                   along the row, coarse test in half precision).  1-4
                                   need k <= 2, otherwise the plain kernel runs            */
    NEMD_OPT_CELL_FACTOR = 4,   /* k >= 1: cells at least rc/k wide, stencil reach k    */
    NEMD_OPT_BLOCK = 5,         /* threads per block of the force kernel (multiple of 32) */
    NEMD_OPT_TIMING = 6,        /* 1: record CUDA events around every force-kernel launch
                                   (read with nemd_get_kernel_time)                       */
    NEMD_OPT_GROUP = 7,         /* lanes per group of the grouped kernel: 4, 8, 16 or 32 */
    NEMD_OPT_AUTOTUNED = 8,     /* 1: nemd_build_cells applies the autotuner's choice for
                                   the current shape class (when it has one)              */
    NEMD_OPT_ASYNC_HOST = 10,   /* 1: host inputs and outputs do not synchronise.  A host
                                   q is copied on the context's copy stream into one of
                                   two device buffers (so the copy of the next state
                                   overlaps the current evaluation) and must stay valid
                                   and unchanged until the next nemd_sync; host F, U, W
                                   are written by that copy stream and are valid after
                                   the next nemd_sync.  0 (default): a call that writes
                                   host outputs synchronises before it returns.          */
    NEMD_OPT_INT_GRAPH = 11,    /* nemd_integrate: 1 (default) captures one step in a
                                   CUDA graph and replays it for the remaining steps
                                   (same results bit for bit); 0 launches every step.
                                   Steps are launched eagerly anyway with
                                   NEMD_OPT_ASYNC_HOST or NEMD_OPT_TIMING on.            */
    NEMD_OPT_REMAP = 9          /* remap instant within a period: 0 (default) at its end,
                                   tau = t - T floor(t/T) in [0, T); 1 half way,
                                   tau = t - T floor(t/T + 1/2) in [-T/2, T/2) -- the
                                   shear flow remapped at half a lattice spacing keeps
                                   the box within 26.57 degrees of upright (Sec. 2.2).
                                   Applies from the next nemd_set_state.                  */
} nemd_option;

/* Statistics of the last force evaluation (read with nemd_get_stats). */
typedef struct nemd_stats {
    int64_t n;              /* particles                                              */
    int64_t pairs;          /* interacting unordered pairs (r < rc)                   */
    int64_t candidates;     /* ordered candidate pairs tested (full neighbourhoods)   */
    int64_t ncells;         /* cells in the grid                                      */
    int32_t counts[3];      /* c_i (dynamic size) or l_i (dynamic offset)             */
    int32_t variant;        /* variant actually used (NEMD_DS or NEMD_DO)             */
    int32_t cell_factor;    /* k                                                      */
    int32_t max_rows;       /* row stride of the stencil table                        */
    int64_t stencil_cells;  /* sum over home cells of neighbourhood cells             */
    int64_t rechecks;       /* candidates decided by the float64 guard-band test      */
    double tau;             /* t mod T                                                */
    double band;            /* float32 guard band on r^2 (absolute)                   */
    int64_t launches;       /* kernels this context has launched since creation       */
} nemd_stats;

/* Create a context on CUDA device `device`, issuing all work on `stream`
 * (a cudaStream_t; NULL means the legacy default stream).  *ctx receives the
 * handle.  Returns NEMD_ERR_CUDA if the device cannot be used.  Contexts are
 * independent: several contexts on several streams may evaluate independent
 * states at the same time (one context's setup kernels then run beside
 * another's force kernel), with results equal bit for bit to evaluating the
 * states one after another. */
int nemd_create(nemd_ctx **ctx, int device, void *stream);

/* Release all library-owned memory.  Safe on NULL. */
int nemd_destroy(nemd_ctx *ctx);

/* Set the flow (Sec. 2.1: u(x) = A x, dL/dt = A L) and the Kraynik-Reinelt
 * remap (Sec. 2.2, Eq. kr: exp(A T) L0 = L0 M, M in SL(3,Z)).  A, L0: 9
 * float64 each; M: 9 int64; T > 0 the period (ignored, and M must be the
 * identity, when A = 0).  Validated on the device before returning (this call
 * synchronises): NEMD_ERR_NOT_SL3Z, NEMD_ERR_TRACE, NEMD_ERR_NOT_KR. */
int nemd_set_flow(nemd_ctx *ctx, const double A[9], const double L0[9], const int64_t M[9], double T);

/* Pair potential (Sec. 5: WCA in the paper's runtime test; LJ otherwise).
 * kind: nemd_potential; eps, sigma > 0; shift != 0 subtracts u(rc).  For
 * NEMD_WCA the cut-off passed to nemd_build_cells must be 2^(1/6) sigma. */
int nemd_set_potential(nemd_ctx *ctx, int kind, double eps, double sigma, int shift);

/* Positions and time.  q: N x 3 float64 (host or device), any image; t: time.
 * Launches the lattice evolution L(t) = exp(A (t mod T)) L0, i.e. the remap
 * L <- L M^-1 applied at every period (Sec. 2.2).  A device q must stay valid
 * and unchanged until the next nemd_compute_forces has completed. */
int nemd_set_state(nemd_ctx *ctx, const double *q, int64_t n, double t);

/* Cell grid, stencil and binning for cut-off rc > 0 (Sec. 3, 4).
 *   NEMD_DS: c_i = floor(h_i / rc) cells congruent to the box, 27 cells (Sec. 4.1);
 *   NEMD_DO: rectangular cells l_i = floor(r_ii / rc) in the QR frame of the box,
 *            with neighbourhoods expanded across offset faces (Sec. 4.2);
 *   NEMD_AUTO_*: chosen per step on the device (see nemd_variant).
 * The counts carry a relative safety margin of 1e-12 (floor((1-1e-12) h/rc)).
 * A zero count is reported (deferred) as NEMD_ERR_BOX_TOO_SMALL. */
int nemd_build_cells(nemd_ctx *ctx, int variant, double rc);

/* Forces, energy and virial of the current state (Sec. 3, 5).
 *   F: N x 3 float32 in input order, F_i = sum_j -u'(r_ij) (q_i - q_j - L n)/r_ij;
 *   U: 1 float64, sum over unordered pairs of u(r);
 *   W: 9 float64 row-major, sum over unordered pairs of r_ij (x) f_ij with
 *      r_ij = q_i - (q_j + L n) and f_ij the force on i from j.
 * Any of F, U, W may be NULL to skip it.  Every sum is formed in a fixed order
 * (the pairs within float32 rounding of rc, decided in float64, in 64-bit
 * fixed point), so a state gives the same F, U and W bit for bit from run to
 * run with the same kernel options (kernel 3 excepted, see NEMD_OPT_KERNEL). */
int nemd_compute_forces(nemd_ctx *ctx, float *F, double *U, double *W);

/* Time integration under the flow (Sec. 2.1: a particle (q, p) has images
 * (q + L_t n, p + A L_t n), so in peculiar momenta p - A q every image carries
 * the same momentum).  The paper fixes no integrator; this one integrates the
 * SLLOD equations for unit mass,
 *     dq/dt = p + A q,   dp/dt = F(q, t) - A p  (- alpha p, isokinetic),
 * with p the peculiar momentum, by a symmetric splitting per step of dt:
 *     p <- exp(-A dt/2) (p + F dt/2);  isokinetic rescale;
 *     q <- exp(A dt) q + Phi(dt) p,  Phi(dt) = int_0^dt exp(sA) ds  (exact for fixed p);
 *     t <- t + dt;  q wrapped into the unit cell of L(t);  F <- F(q, t);
 *     p <- F dt/2 + exp(-A dt/2) p;  isokinetic rescale.
 * The rescale (thermostat = 1) multiplies p by sqrt(K0 / sum |p|^2), K0 the
 * initial sum |p|^2 (Gaussian isokinetic in its velocity-rescaling form);
 * thermostat = 0 leaves it out.  Every force evaluation is the hot path of
 * this library (nemd_set_state, nemd_build_cells(variant, rc),
 * nemd_compute_forces) with the context's potential and options.
 *   q, p: N x 3 float64 DEVICE arrays (state at time t0), updated in place to
 *         t0 + nsteps dt: q wrapped into the unit cell, p peculiar momenta;
 *         they must stay valid until nemd_sync returns.
 *   dt > 0 finite; nsteps >= 0.  Asynchronous (enqueues every step); the
 *   context's time afterwards is t0 + nsteps dt.
 * Arithmetic: q and p are stored in float64; the kicks and the drift compute
 * in float-float (about 2^-47 relative per operation, the propagators applied
 * as x + (M - I) x) and round each stored component once, so a step adds an
 * error of a few 2^-47 |q| and |p|; components below 2^-100 in magnitude
 * count as 0 there (an error under 2^-100), and a particle with a component
 * of 2^100 or more, or not finite, is stepped in float64.
 * Errors: NEMD_ERR_ARG (host arrays, n < 0, bad dt or nsteps), NEMD_ERR_ORDER
 * (no flow), and the errors of the force evaluation. */
int nemd_integrate(nemd_ctx *ctx, double *q, double *p, int64_t n, double t0, double dt, int64_t nsteps,
                   int variant, double rc, int thermostat);

/* Verlet neighbour list with a skin for nemd_integrate.  The paper rebuilds
 * its cell list at every step (Sec. 4.1); it has no Verlet list, which is the
 * standard next stage.  With skin > 0 the integrator keeps the pairs within
 * rc + skin found by one cell-list search (nemd_build_cells(variant, rc + skin)
 * and the library's list kernel), evaluates only those at the following steps
 * (same pair decision, forces, energy and virial as the cell-list path), and
 * rebuilds the list when a pair outside it could have come within rc:
 *     exp(mu (t - t_b)) (rc + skin) - 2 delta < rc,
 * t_b the time of the build, mu <= 0 the smallest eigenvalue of (A + A^T)/2
 * (the flow shrinks no distance faster than exp(mu t)) and delta the largest
 * peculiar displacement |L(t) u_i| since the build (measured in the deformed
 * frame), and at every remap.
 * Positions are wrapped at every step; the images of the listed pairs follow
 * the wraps.  The rebuild decision is taken on the host (one synchronisation
 * per step), so these steps are launched rather than replayed as a graph.
 * skin = 0 (default) turns the list off; skin < 0 or not finite is
 * NEMD_ERR_ARG.  Setting it discards the current list. */
int nemd_set_verlet(nemd_ctx *ctx, double skin);

/* Since the last nemd_set_verlet: list builds, force evaluations from the list
 * (builds included), the entries per particle of the current list, and the
 * largest peculiar displacement since the build measured at the last check
 * that kept the list.  Any pointer may be NULL. */
int nemd_get_verlet_stats(nemd_ctx *ctx, int64_t *builds, int64_t *steps, int64_t *width, double *delta);

/* Wait for the stream and return any deferred device error. */
int nemd_sync(nemd_ctx *ctx);

/* Message of the last error of this context (never NULL). */
const char *nemd_last_error(const nemd_ctx *ctx);

/* Set an option (nemd_option).  Takes effect at the next nemd_build_cells. */
int nemd_set_option(nemd_ctx *ctx, int key, int64_t value);

/* Copy the current lattice to host memory (synchronises).  out[48]:
 * L(9) Linv(9) V h(3) Q(9) R(9) tau band(ignored) counts(3, as doubles) ncells variant
 * -- see nemd.py for the exact unpacking. */
int nemd_get_lattice(nemd_ctx *ctx, double *out);

/* Statistics of the last evaluation (synchronises). */
int nemd_get_stats(nemd_ctx *ctx, nemd_stats *out);

/* Verification mode (NEMD_OPT_RECORD_PAIRS > 0): copy the recorded unordered
 * pairs as int32 quintuples (i, j, n1, n2, n3) with i < j, or i == j and n
 * lexicographically positive, to host memory `out` (capacity `cap` pairs);
 * *count receives the number of pairs found (which may exceed cap or the
 * record capacity: then the record is incomplete and NEMD_ERR_CAPACITY is
 * returned).  Synchronises. */
int nemd_get_pairs(nemd_ctx *ctx, int32_t *out, int64_t cap, int64_t *count);

/* With NEMD_OPT_TIMING on: total device time (ms) of the force-kernel launches
 * recorded since the last call and their number; resets the record.  Events
 * are recorded on the context's stream, at most 4096 launches are kept.
 * Synchronises. */
int nemd_get_kernel_time(nemd_ctx *ctx, double *ms_total, int64_t *nlaunch);

/* ---- Autotuner ------------------------------------------------------------
 *
 * The paper has no counterpart (its cells are always at least the cut-off
 * wide, Sec. 4).  Every candidate configuration -- force kernel (plain, warp,
 * warp with half neighbourhoods, grouped, row), lanes per group (4, 8, 16),
 * cell-size factor k (1, 2) -- gives the same pair set and, up to rounding,
 * the same forces; only the time differs. */
typedef struct nemd_tune_config {
    int32_t kernel, group, cell_factor, pad;
} nemd_tune_config;

typedef struct nemd_tune_entry {
    nemd_tune_config cfg;
    double ms;  /* mean time of one nemd_build_cells + nemd_compute_forces */
} nemd_tune_entry;

/* Time every candidate on the current state (after nemd_set_state): one
 * untimed then `reps` timed repetitions of nemd_build_cells(variant, rc) +
 * nemd_compute_forces, with CUDA events on the context's stream.  The times
 * are added to the cache of the current shape class, (round(log2 N),
 * round(4 log2(rho rc^3))); the class's best mean over all calls so far is
 * applied to the context (kernel, group, cell factor) and written to *best
 * (optional).  times[0..cap) (optional) receives each candidate's mean time of
 * this call, *ntimes (optional) their number.  Leaves the cells built with the
 * chosen configuration.  Synchronises. */
int nemd_autotune(nemd_ctx *ctx, int variant, double rc, int reps, nemd_tune_config *best, nemd_tune_entry *times,
                  int cap, int *ntimes);

/* Save / load the autotuner cache: "NEMDTUNE", version, class count,
 * candidate count, the entries, and an FNV-1a 64-bit checksum of all of it.
 * Load rejects (NEMD_ERR_ARG) a file with another magic, version, candidate
 * count or checksum and then leaves the cache unchanged. */
int nemd_tune_save(nemd_ctx *ctx, const char *path);
int nemd_tune_load(nemd_ctx *ctx, const char *path);

/* ---- Learned cell-list selector -------------------------------------------
 *
 * The paper has no counterpart: its own rule for choosing between the two
 * cell lists is the neighbourhood-volume comparison of Sec. 5.1-5.2
 * (NEMD_AUTO_HEURISTIC), which remains the fallback.  A small multilayer
 * perceptron (12 -> 64 -> 64 -> 4, ReLU, float32) predicts, per step, the
 * normalised ln(time / N) of the four options o = (variant o & 1, cell factor
 * 1 + (o >> 1)) from the features of the step:
 *   x[0..8]  the entries of L(t) / V^(1/3) (row-major)
 *   x[9]     N / V        x[10]  rc        x[11]  ln N
 * With a model set, nemd_build_cells(NEMD_AUTO_LEARNED, rc) runs the forward
 * pass on the device and uses the option with the smallest prediction; the
 * pair set and forces do not depend on the choice.  All arrays below are host
 * memory; the training and inference run in the library's own kernels. */
#define NEMD_MLP_INPUTS 12
#define NEMD_MLP_OUTPUTS 4
#define NEMD_MLP_PARAMS 5252
#define NEMD_MLP_NORM 26   /* input means (12), input std (12), target mean, target std */

/* Features of the current state (after nemd_set_state).  Synchronises. */
int nemd_features(nemd_ctx *ctx, double rc, float out[12]);

/* Time the four options on the current state (one untimed, then `reps` timed
 * nemd_build_cells + nemd_compute_forces each, CUDA events): features[12] and
 * ms[4] (mean milliseconds) form one training row.  Synchronises. */
int nemd_time_options(nemd_ctx *ctx, double rc, int reps, float features[12], float ms[4]);

/* Train from scratch on `rows` rows (X: rows x 12 features, T_ms: rows x 4
 * times in ms, all > 0): inputs and ln(time / N) targets (time per particle,
 * N = exp(x[11])) normalised by their mean
 * and standard deviation, Glorot-uniform weights from `seed`, then `steps`
 * Adam steps (lr) on mini-batches of `batch` rows drawn with replacement.
 * loss_hist (optional) receives each step's mini-batch mean squared error.
 * The trained model becomes this context's selector. */
int nemd_model_train(nemd_ctx *ctx, const float *X, const float *T_ms, int64_t rows, int steps, int batch, double lr,
                     uint64_t seed, float *loss_hist);

/* Predicted normalised ln(time / N) (rows x 4) of raw feature rows X (rows x 12). */
int nemd_model_predict(nemd_ctx *ctx, const float *X, int64_t rows, float *Y);

/* Gradient (NEMD_MLP_PARAMS floats) and value of L = sum (y - t)^2 / (rows 4)
 * at the current parameters, for already normalised inputs Xn and targets Tn. */
int nemd_model_grad(nemd_ctx *ctx, const float *Xn, const float *Tn, int64_t rows, float *grad, double *loss);

/* Parameters: W1[64][12] b1[64] W2[64][64] b2[64] W3[4][64] b3[4] (row-major),
 * and the NEMD_MLP_NORM normalisation constants. */
int nemd_model_set_params(nemd_ctx *ctx, const float *params, const float *norm);
int nemd_model_get_params(nemd_ctx *ctx, float *params, float *norm);

/* Save / load the model: "NEMDMLP1", the three layer widths, parameters,
 * normalisation and an FNV-1a 64-bit checksum; load rejects any mismatch. */
int nemd_model_save(nemd_ctx *ctx, const char *path);
int nemd_model_load(nemd_ctx *ctx, const char *path);

/* Measure device peaks with the library's own kernels (synchronises):
 * out[0] FP32 FMA lane-ops/s, out[1] FP32 paired (f32x2) lane-ops/s,
 * out[2] FP64 FMA ops/s, out[3] copy bandwidth bytes/s, out[4] SM count,
 * out[5] SM clock kHz reported by the device. */
int nemd_measure_peaks(int device, double *out);

/* ---- Batches of independent systems -------------------------------------
 *
 * The paper treats one system at a time; a batch evaluates many independent
 * systems -- each with its own flow, lattice, potential, cut-off, N and cell
 * list variant -- in one step whose every stage (lattice, grid and stencil,
 * binning, chunk lists, force, reductions) is ONE kernel launch over all
 * systems, the force kernel being a single persistent launch over the chunks
 * of every system.  The step is captured once into a CUDA graph and replayed
 * (NEMD_BATCH_OPT_GRAPH).  Per system the results are those of a context with
 * the same flow, potential, variant and cell factor running the same force
 * kernel (NEMD_BATCH_OPT_KERNEL, as NEMD_OPT_KERNEL): same pair set, forces
 * per particle equal up to rounding; U and W are float64 sums of the same
 * pair terms in another order.  Several batches, each on its own stream, run
 * independently (a caller may keep two steps in flight on two streams).
 *
 * Call order: nemd_batch_create, nemd_batch_add (once per system, in order),
 * nemd_batch_finalize, then per step nemd_batch_set_state and
 * nemd_batch_compute; nemd_batch_sync returns the deferred device errors.
 * Particles of all systems are concatenated in system order: system s owns
 * rows offsets[s] .. offsets[s+1]-1 of q and F (nemd_batch_offsets). */
typedef struct nemd_batch nemd_batch;

typedef struct nemd_system {
    double A[9], L0[9];  /* flow and reference lattice, as nemd_set_flow            */
    int64_t M[9];        /* remap matrix in SL(3,Z), as nemd_set_flow              */
    double T;            /* period, as nemd_set_flow                               */
    double eps, sigma;   /* potential, as nemd_set_potential                       */
    double rc;           /* cut-off; WCA needs rc = 2^(1/6) sigma                   */
    int64_t n;           /* particles, 0 .. 2^21                                   */
    int32_t kind;        /* NEMD_LJ or NEMD_WCA                                    */
    int32_t shift;       /* energy shifted to 0 at rc (required for WCA)           */
    int32_t variant;     /* NEMD_DS, NEMD_DO or NEMD_AUTO_HEURISTIC (per step)     */
    int32_t remap;       /* as NEMD_OPT_REMAP: 0 tau in [0, T), 1 in [-T/2, T/2)   */
} nemd_system;

typedef struct nemd_batch_stats {
    int64_t pairs;       /* interacting unordered pairs of the last step           */
    int64_t candidates;  /* distance tests of the last step                        */
    int64_t band;        /* candidates decided with the float32 residuals added    */
    int32_t counts[3];   /* cell counts of the last step's grid                    */
    int32_t variant;     /* cell list used in the last step (NEMD_DS / NEMD_DO)    */
    int32_t cell_factor; /* cell-size factor of the last step                      */
    int32_t status;      /* nemd_status of the system's last step                  */
} nemd_batch_stats;

/* Batch options (nemd_batch_set_option). */
#define NEMD_BATCH_OPT_CELL_FACTOR 1  /* cells >= rc / k wide, k = 1 or 2 (default 1)   */
#define NEMD_BATCH_OPT_TILE 2         /* particles per chunk, 16 or 32 (default 32)     */
#define NEMD_BATCH_OPT_GRAPH 3        /* 1: capture and replay a CUDA graph (default);
                                         0: launch the kernels one by one             */
#define NEMD_BATCH_OPT_KERNEL 4       /* force kernel of the persistent launch: 4 the row
                                         kernel (default), 2 the warp kernel; same pair
                                         set and forces up to rounding                */

/* Create / destroy a batch on `device` working on `stream` (a cudaStream_t,
 * NULL = the legacy default stream).  Destroy synchronises and frees
 * everything the batch owns. */
int nemd_batch_create(nemd_batch **out, int device, void *stream);
int nemd_batch_destroy(nemd_batch *b);
const char *nemd_batch_last_error(const nemd_batch *b);

/* Append one system (host struct, copied); *index (optional) receives its
 * index.  The flow is validated as by nemd_set_flow (NEMD_ERR_NOT_SL3Z,
 * NEMD_ERR_TRACE, NEMD_ERR_NOT_KR), the potential and cut-off as by
 * nemd_set_potential / nemd_build_cells; NEMD_ERR_ORDER after finalize. */
int nemd_batch_add(nemd_batch *b, const nemd_system *sys, int64_t *index);

/* Size and allocate the device tables for the systems added: cell slots
 * k^3 V / rc^3 per system (k = 2, a bound that holds at every strain);
 * row-class slots from the largest class count over 257 states of the
 * period, times 1.25, plus 16 (a state that would need more sets
 * NEMD_ERR_CAPACITY for its system at that step).  Synchronises. */
int nemd_batch_finalize(nemd_batch *b);

/* Particle offsets: offsets[0..nsys] (host), offsets[nsys] = total N. */
int nemd_batch_offsets(const nemd_batch *b, int64_t *offsets, int64_t *nsys);

/* State of every system: q -- total N x 3 float64 (host or device; a device
 * pointer is read in place by the next nemd_batch_compute and must stay valid
 * until it has run); t -- nsys float64 times, HOST. */
int nemd_batch_set_state(nemd_batch *b, const double *q, const double *t);

/* One step for every system: F -- total N x 3 float32 (Cartesian, input
 * order), UW -- nsys x 10 float64 (U, then W row-major); each host or device
 * pointer, or NULL to skip.  Asynchronous for device outputs; with a host
 * output it synchronises before it returns.  A system whose step failed (see
 * nemd_batch_sync) gets U = W = 0 and unspecified forces.  Sums are formed in
 * a fixed order except for the pairs within float32 rounding of rc (decided in
 * float64 and added with float atomics): a particle with two or more of those
 * in one step can make its system's F, U, W differ in the last bit between
 * runs. */
int nemd_batch_compute(nemd_batch *b, float *F, double *UW);

/* Wait for the stream; return the first failing system's status (0 = all
 * OK).  status (optional, host, nsys ints) receives every system's status
 * since the previous sync. */
int nemd_batch_sync(nemd_batch *b, int32_t *status);

int nemd_batch_set_option(nemd_batch *b, int key, int64_t value);

/* Per-system statistics of the last step (host array of nsys entries).
 * *launches (optional) receives the kernel launches of one step.  Synchronises. */
int nemd_batch_get_stats(nemd_batch *b, nemd_batch_stats *out, int64_t *launches);

/* Autotuner of a batch: times `reps` steps (after one untimed step) of every
 * candidate -- cell factor 1, 2 x particles per chunk 16, 32 -- on the current
 * state and keeps the fastest.  times (optional, cap entries) receives each
 * candidate as {kernel = the batch's force kernel, group = tile, cell_factor,
 * ms}.  Synchronises. */
int nemd_batch_autotune(nemd_batch *b, int reps, nemd_tune_entry *times, int cap, int *ntimes);

/* ---- Force evaluation without any memory allocation --------------------
 *
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc -- for example a simulation loop that must never
 * allocate once it is running, or a plug-in that has no access to the CUDA
 * allocator of the process hosting it.  It performs one whole force
 * evaluation (the same kernels as nemd_set_state -> nemd_build_cells ->
 * nemd_compute_forces, dynamic size / dynamic offset / heuristic variant,
 * cell factor 1, float32 pair arithmetic) without allocating anything: no
 * cudaMalloc, no cudaFree, no allocating library routine.
 *
 * Scratch: one file-scope device array of NEMD_NOALLOC_SCRATCH_BYTES bytes
 * (about 10.6 MB), present on every GPU that loads the library until the
 * process exits.  It holds at most NEMD_NOALLOC_MAX_N particles and
 * NEMD_NOALLOC_MAX_CELLS cells; larger requests (N, or the cell bound
 * |det L0| / rc^3 + 1) return NEMD_ERR_CAPACITY before anything is launched.
 * Every call on a device shares that array and leaves its contents behind
 * (each call clears what must start at zero), so calls whose work overlaps on
 * the GPU -- on different streams, or from different threads -- race and give
 * wrong results: serialise them.
 *
 * Set-up: the first call on each device looks up the device address of the
 * array (cudaGetSymbolAddress, with that device current) and caches it; make
 * that first call before any stream capture begins.
 *
 * Arguments (the current CUDA device is used): A, L0 -- 9 float64 each, host
 * (the flow is not re-validated: pass one that nemd_set_flow accepts; T is the
 * KR period, t the time); q -- N x 3 float64, DEVICE; variant -- NEMD_DS,
 * NEMD_DO or NEMD_AUTO_HEURISTIC; rc, kind, eps, sigma, shift -- as in
 * nemd_build_cells / nemd_set_potential; F -- N x 3 float32, DEVICE; UW --
 * 10 float64, DEVICE, receives U then W (row-major); status -- optional int,
 * DEVICE, receives the deferred device error bits (0 = OK, 1 = box too small,
 * 2 = non-finite position, 4 = capacity); stream -- a cudaStream_t (NULL =
 * legacy default stream).  All work is asynchronous on `stream`.  q, F, UW and
 * status must be memory of the current device (or managed memory); a pointer
 * of another device or of the host is refused with NEMD_ERR_ARG. */
#define NEMD_NOALLOC_MAX_N 16384
#define NEMD_NOALLOC_MAX_CELLS 16384
#define NEMD_NOALLOC_SCRATCH_BYTES 11154432
int nemd_forces_noalloc(const double A[9], const double L0[9], double T, double t, const double *q, int64_t n,
                        int variant, double rc, int kind, double eps, double sigma, int shift, float *F, double *UW,
                        int *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NEMD_H */
