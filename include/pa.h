/*
 * pa.h -- C ABI of the GB300 (sm_103a) population-annealing library for the
 * two-dimensional q-state Potts model.
 *
 * The method is population annealing (PA) as defined in Barash, Weigel, Shchur
 * & Janke, "Exploring first-order phase transitions with population annealing"
 * (arXiv:1704.01888):
 *   Sec. 2, steps 1-5    the PA loop: start an equilibrium population at beta_0,
 *                        resample it to beta_i with the normalised Boltzmann
 *                        factors tau_i(E_j), update every replica by theta
 *                        Metropolis rounds at beta_i, measure population
 *                        averages, repeat;
 *   Sec. 2, Eq. 2        -beta_i F = ln Z_{beta_0} + sum_{m<=i} ln Q_m;
 *   Sec. 3, Eqs. 3-5     H = -sum_<ij> delta(s_i, s_j) on the periodic square
 *                        lattice, population averages, magnetisation;
 *   Sec. 5, Eq. 6        ground-state starts for heating runs (negative dbeta);
 *   Sec. 6, Eqs. 7-8     Z_{beta_0 = 0} = q^N and Z_{beta -> inf} = q e^{-beta E_0}.
 *
 * Conventions shared by every entry point
 *   - Spins take the values 0..q-1 (the paper's 1..q shifted by one).  Host
 *     copies use the canonical layout [replica][y][x], one byte per spin.
 *   - A context owns all of its device memory and runs all of its work on the
 *     CUDA stream given at creation (a cudaStream_t passed as void*, NULL for
 *     the legacy default stream).  Unless stated otherwise a call only enqueues
 *     work and returns; calls that hand results to host memory synchronise that
 *     stream first.
 *   - Host pointers passed in are read (inputs) or written (outputs) during the
 *     call only; the library keeps no reference to them.
 *   - Every call returns a pa_status.  Nothing aborts the process.  A call that
 *     fails leaves the context at its last complete temperature step.
 *   - Random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     the 64-bit seed and a counter made of (four same-colour sites, sweep and
 *     colour, step, slot) for sweeps, (site/4, init, slot) for initial states
 *     and (replica/4, resample, step) for copy numbers, with the stream number
 *     in the top byte of the last word, so results do not depend on launch
 *     shapes, stream timing or the number of replicas per block.
 */
#ifndef PA_H
#define PA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PA_OK = 0,
    PA_ERR_INVALID = 1,  /* an argument is out of range, see each call         */
    PA_ERR_CAPACITY = 2, /* a resampled population would exceed R_cap          */
    PA_ERR_CUDA = 3,     /* a CUDA runtime call failed; see pa_last_cuda_error */
    PA_ERR_TIMEOUT = 4,  /* reserved for bounded device waits; no call of this
                            version returns it (its kernels do not wait on one
                            another)                                          */
    PA_ERR_STATE = 5,    /* calls in the wrong order, or a failed context      */
    PA_ERR_NOMEM = 6,    /* device or host allocation failed                   */
    PA_ERR_TOO_LARGE = 7 /* a replica larger than one block's shared memory
                            holds (see pa_init), or a size beyond the fixed
                            working memory of pa_resample_noalloc            */
} pa_status;

/* Copy-number rule for the resampling step (Sec. 2, step 2).  The paper draws
 * r_j from a Poisson law with mean rho_j = (R/R_{i-1}) tau_i(E_j) (Eq. 1):
 * POISSON (inversion of the distribution, the mean split into pieces of at
 * most 64).  NEAREST_INT takes one of the two integers nearest to rho_j,
 * floor(rho_j) + 1 with probability frac(rho_j), so the mean is kept and the
 * spread is minimal; ROUND takes the nearest integer outright (halves up);
 * OFF keeps every replica once (the resampling-off comparison of Sec. 5,
 * Fig. 2 right; ln Q is still computed). */
enum { PA_RESAMPLE_NEAREST_INT = 0, PA_RESAMPLE_ROUND = 1, PA_RESAMPLE_POISSON = 2, PA_RESAMPLE_OFF = 3 };

/* Initial population (Sec. 2 step 1; Sec. 5 Eq. 6). */
enum { PA_INIT_RANDOM = 0, /* beta_0 = 0: independent uniform spins, ln Z_0 = N ln q        */
       PA_INIT_GROUND = 1  /* each replica a uniformly chosen ground state, ln Z_0 = ln q + 2 N beta_0 */ };

typedef struct {
    int32_t q;             /* Potts states, 2..128                                   */
    int32_t L;             /* linear size, even, 2..1024; N = L*L sites              */
    int32_t R;             /* target population size R (= R_0), >= 1                 */
    int32_t R_cap;         /* capacity; 0 selects R + R/4 + 1024                     */
    uint64_t seed;         /* Philox key                                             */
    int32_t resample_mode; /* PA_RESAMPLE_*                                          */
    int32_t init_mode;     /* PA_INIT_*                                              */
    double beta0;          /* inverse temperature of the initial population         */
    int32_t track_families;/* 1: keep ancestor ids and family statistics             */
    int32_t stream;        /* 0..255: runs with one seed and different streams are
                              independent (the stream is the top byte of the slot
                              counter word); 0 for a lone run                        */
} pa_config;

/* Population estimators of one temperature step (Sec. 2 step 4, Sec. 3 Eq. 4):
 *   meanE = sum_j E_j / R_i, meanE2 = sum_j E_j^2 / R_i (exact integer sums);
 *   C     = beta^2 (meanE2 - meanE^2) / N, the specific heat per site;
 *   meanM = (q sum_j Mt_j - N R_i) / ((q - 1) R_i) with Mt_j the occupation of
 *           replica j's most common state (Eq. 5);
 *   lnQ   = ln Q_i of the resampling into this step (0 at step 0);
 *   lnZ   = ln Z_{beta_0} + sum_{m<=i} ln Q_m = -beta_i F (Eq. 2);
 *   S_f   = -sum_f nu_f ln nu_f, nu_f the fraction of replicas descending from
 *           initial replica f (family entropy; the paper does not define it),
 *           n_families the number of such f with nu_f > 0.  Both 0 unless
 *           track_families;
 *   n_near_ties = copy numbers of the resampling into this step whose outcome
 *           a change of rho_j in its last places could have changed: for
 *           NEAREST_INT frac(rho_j) within 2^-48 max(1, rho_j) of u_j / 2^32,
 *           for ROUND within that distance of 1/2, for POISSON a uniform of
 *           the inversion within 2^-40 of the cumulative probability it is
 *           compared with (0 at step 0 and for OFF).  A diagnostic only: it
 *           changes no outcome. */
typedef struct {
    double beta, lnQ, lnZ, meanE, meanE2, C, meanM, S_f;
    int64_t R, n_families, sumE, sumE2, sumMt, n_near_ties;
} pa_obs;

typedef struct pa_ctx pa_ctx;

/* Creates a context, allocates its device buffers (two spin buffers of R_cap
 * replicas in the multi-spin-coded layout below, plus O(R_cap + N) words) and
 * enqueues the initial population at
 * cfg->beta0 (Sec. 2 step 1 or Sec. 5 Eq. 6) with its energies, largest-state
 * occupations, energy histogram and step-0 estimators.
 * Errors: PA_ERR_INVALID for q outside 2..128, odd or out-of-range L, R < 1,
 * R_cap < R or R_cap >= 2^24, beta0 < 0, an unknown mode, or a stream outside
 * 0..255; PA_ERR_TOO_LARGE when a replica's bit planes exceed 204800 bytes
 * (a sweep block keeps whole lattices in shared memory).  Device layout of a
 * replica: a state takes B = ceil(log2 q) bits, stored as P bit planes (B
 * rounded up to 1, 2 or 4 for B <= 4, else P = B); the sites of each colour ((x + y) mod 2) are
 * packed 32 to a 32-bit word per plane (row-major over the colour's sites
 * when L/2 divides 32; when L is a multiple of 16 but not of 64 and L > 32,
 * a word holds one 8-column segment of four rows L/4 apart; else each row is
 * padded to whole words), so a replica takes 2 W P 4 bytes, W = L^2/64 (the
 * first two cases) or L ceil(L/64) words per colour: L <= 640 for q <= 16,
 * 568 for q <= 32, 512 for q <= 64 and 456 for q <= 128.  PA_ERR_NOMEM or
 * PA_ERR_CUDA if allocation or a launch fails (nothing is leaked; *out = NULL). */
pa_status pa_init(const pa_config *cfg, void *cuda_stream, pa_ctx **out);

/* Resampling from beta_{i-1} to beta_i = beta_{i-1} + dbeta (Sec. 2 step 2):
 * computes ln Q_i from the current energy histogram, the copy numbers r_j
 * (per resample_mode), their exclusive scan and the parent map of the new
 * population.  The replica gather itself is fused into the next pa_sweep.
 * Arithmetic: with E_ref the lowest energy (highest for dbeta < 0), the
 * weights w = exp(-dbeta (E - E_ref)) come from a table the host computes
 * with the C library's exp (once per distinct dbeta, then kept on the device);
 * S = sum_j w_j is summed exactly and rounded once to the nearest double;
 * rho_j = (R w_j) / S; ln Q_i = -dbeta E_ref + ln(S / R_{i-1}).  So S, rho_j
 * and the copy numbers do not depend on the device's summation order.
 * `step` is the temperature-step index i >= 1 (part of the random key) and
 * must exceed the previous step's.  dbeta may be negative (heating, Sec. 5).
 * If lnQ_out or R_out is non-NULL the call synchronises and writes ln Q_i and
 * the new size R_i; otherwise it only enqueues.
 * Errors: PA_ERR_STATE if a resample is already pending or step does not
 * increase; PA_ERR_INVALID for a non-finite dbeta; PA_ERR_CAPACITY (reported
 * here when synchronising, else by the next synchronising call) if R_i would
 * exceed R_cap -- the population is then left at step i-1. */
pa_status pa_resample(pa_ctx *ctx, double dbeta, int32_t step, double *lnQ_out, int32_t *R_out);

/* theta checkerboard Metropolis sweeps at inverse temperature beta over every
 * replica of the current population (Sec. 2 step 3), fused with the pending
 * replica gather and followed by the per-replica energies, largest-state
 * occupations, the energy histogram and the step's estimators.  One sweep
 * updates the colour (x+y) even sites, then the odd ones; each attempt
 * proposes s' = s + d or s - d (mod q) with a random direction and
 * d = 1 + u, u uniform on B - 1 bits (B = ceil(log2 q); a symmetric proposal
 * over the q-1 other states, uniform when q-1 is a power of two), and accepts
 * it with probability min(1, exp(-beta dE)) quantised to 32 bits.
 * `step` must equal the step of the pending resample (or 0 for extra sweeps
 * at step 0 before any resample).  0 <= theta <= 2^21.
 * Errors: PA_ERR_INVALID for theta outside 0..2^21 or beta < 0;
 * PA_ERR_STATE for a step mismatch or a failed context. */
pa_status pa_sweep(pa_ctx *ctx, double beta, int32_t theta, int32_t step);

/* Per-replica energies E_j of the current population, int32, in slot order.
 * on_device = 1: E_out is a device pointer with room for R_cap values (the
 * copy is enqueued); 0: E_out is host memory with room for R_cap values (the
 * call synchronises).  Only the first R_i values are written. */
pa_status pa_energy(pa_ctx *ctx, int32_t *E_out, int32_t on_device);

/* Per-replica occupation of the most common state, Mt_j = max over states a
 * of the number of sites in state a (Sec. 3, Eq. 5: the magnetisation of
 * replica j is m_j = (q Mt_j / N - 1) / (q - 1)), of the current population,
 * [R_i] int32, into host memory (synchronises) or device memory (on_device
 * != 0, enqueued).  Errors as pa_energy. */
pa_status pa_occupations(pa_ctx *ctx, int32_t *Mt_out, int32_t on_device);

/* Synchronises and returns the estimators of the latest completed step.  If
 * hist_out is non-NULL, also the energy histogram of the current population:
 * hist_out[k] = number of replicas with E = k - 2N, k = 0..2N, so hist_len
 * must be >= 2N+1.  Errors: PA_ERR_CAPACITY / PA_ERR_TIMEOUT from enqueued
 * work, PA_ERR_INVALID for a short hist buffer. */
pa_status pa_observables(pa_ctx *ctx, pa_obs *out, int32_t *hist_out, int32_t hist_len);

/* Synchronises and copies the estimators of the last `count` completed steps
 * (oldest first) into out[0..count).  The context keeps at least the last
 * 1024 records (more after a longer pa_run).  PA_ERR_INVALID if count < 1 or
 * more records are asked for than are kept. */
pa_status pa_observables_history(pa_ctx *ctx, int32_t count, pa_obs *out);

/* Current population size R_i (synchronises). */
pa_status pa_population_size(pa_ctx *ctx, int32_t *R_out);

/* Copies replicas [slot_begin, slot_begin + count) of the current population
 * into host memory in the canonical layout [count][L][L] (synchronises).
 * Errors: PA_ERR_INVALID if the range exceeds R_i or host is NULL. */
pa_status pa_get_spins(pa_ctx *ctx, int64_t slot_begin, int64_t count, uint8_t *host);

/* Initial-replica (family) ids of the current population, host int32[R_i]
 * (synchronises).  PA_ERR_STATE unless track_families. */
pa_status pa_get_ancestors(pa_ctx *ctx, int32_t *host);

/* Parent map of the latest resampling step (Sec. 2 step 2): out[k] = the slot,
 * in the population before that step, of the replica that new slot k copies;
 * children of one parent are consecutive and parents ascend.  R_i int32
 * values (R_i the size after that step, pending or swept).  on_device = 0:
 * out is host memory (the call synchronises); 1: a device pointer (the copy is
 * enqueued).  PA_ERR_STATE before the first resample. */
pa_status pa_get_parents(pa_ctx *ctx, int32_t *out, int32_t on_device);

/* Runs the temperature schedule betas[1..K] from the context's current step:
 * for i = 1..K, resample by betas[i] - betas[i-1] then theta sweeps at
 * betas[i]; betas[0] must equal the current inverse temperature.  obs_out
 * (host, K entries, may be NULL) receives each step's estimators and hist_out
 * (host, may be NULL) the energy histograms after the steps listed in
 * hist_steps[0..n_hist) (each 2N+1 ints, in that order).  use_graph = 1
 * captures the K steps as one CUDA graph and launches it; 0 launches the
 * kernels directly.  Synchronises once at the end.
 * Errors: as pa_resample / pa_sweep; PA_ERR_INVALID for K < 1. */
pa_status pa_run(pa_ctx *ctx, const double *betas, int32_t K, int32_t theta, pa_obs *obs_out,
                 const int32_t *hist_steps, int32_t n_hist, int32_t *hist_out, int32_t use_graph);

/* ---- Differentiable reweighting (Sec. 2 step 2) --------------------------
 * For R energies E (device int32) and a step dbeta (device double, so no host
 * round trip is needed), with tau_j = exp(-dbeta E_j) / Q:
 *   out[0] = ln Q = ln( sum_j exp(-dbeta E_j) / R )
 *   out[1] = <E>_tau         (= -d ln Q / d dbeta)
 *   out[2] = var_tau(E)      (= -d <E>_tau / d dbeta)
 *   out[3] = <O>_tau = sum_j O_j tau_j / R   (0 if O is NULL)
 *   out[4] = cov_tau(O, E)   (= -d <O>_tau / d dbeta)
 *   out[5] = E_ref (lowest energy for dbeta >= 0, highest otherwise)
 *   out[6] = sum_j exp(-dbeta (E_j - E_ref))
 *   out[7] = k3_tau(E), the third central moment (= -d var_tau / d dbeta)
 * out is a device double[8]; O (device double[R]) may be NULL.  Enqueued on
 * `stream`; one block, fixed summation order, deterministic.
 * PA_ERR_INVALID for NULL pointers or R < 1. */
pa_status pa_reweight_forward(const int32_t *E, const double *O, int32_t R, const double *dbeta, double *out,
                              void *stream);

/* Backward of one forward output with respect to dbeta: dst[0] = sign * g[0] *
 * src[idx] (all device pointers), e.g. src = forward out, idx 1, sign -1 gives
 * d ln Q / d dbeta times the incoming gradient g. */
pa_status pa_reweight_scale(const double *src, int32_t idx, double sign, const double *g, double *dst, void *stream);

/* Backward of <O>_tau with respect to O: grad_O[j] = g[0] tau_j / R
 * (device double[R]), from the forward outputs `fwd` of the same E and dbeta. */
pa_status pa_reweight_grad_O(const int32_t *E, int32_t R, const double *dbeta, const double *fwd, const double *g,
                             double *grad_O, void *stream);

/* ---- Adaptive temperature step (the paper uses constant steps) ------------
 * Weight overlap of the populations at beta and beta + dbeta, with mean-one
 * weights t_j = R exp(-dbeta (E_j - E_ref)) / sum: out[0] = alpha =
 * (1/R) sum_j min(1, t_j), out[1] = d alpha / d dbeta = (1/R) sum_{t_j < 1}
 * t_j (<E>_tau - E_j).  Device pointers; out is double[2]. */
pa_status pa_overlap(const int32_t *E, int32_t R, const double *dbeta, double *out, void *stream);

/* The step dbeta in (0, dbeta_cap] at which the overlap of the context's
 * current population equals `target`: bisection-safeguarded Newton iterations
 * (at most `iters`, from the middle of the bracket [0, dbeta_cap], stopping once
 * |overlap - target| <= 1e-12) on the population's energy histogram, rounded
 * down to a multiple of 2^-24 (dbeta_cap itself if its overlap already reaches
 * the target).  Synchronises.  PA_ERR_INVALID for a
 * target outside (0, 1), a non-positive cap or iters outside 0..200;
 * PA_ERR_STATE with a resample pending. */
pa_status pa_next_dbeta(pa_ctx *ctx, double target, double dbeta_cap, int32_t iters, double *dbeta_out);

/* Runs PA from the current inverse temperature to beta_end with adaptive
 * steps: step i takes dbeta_i = pa_next_dbeta(target, min(dbeta_max, beta_end
 * - beta), iters), resamples and sweeps theta times at beta_i = beta_{i-1} +
 * dbeta_i (the last step lands on beta_end exactly), at most max_steps steps.
 * Writes the number of steps to *K_out, the betas to betas_out[0..K) and the
 * estimators to obs_out[0..K) (host; either may be NULL).  One host
 * synchronisation per step (the step size decides the acceptance thresholds). */
pa_status pa_run_adaptive(pa_ctx *ctx, double beta_end, double target, double dbeta_max, int32_t iters, int32_t theta,
                          int32_t max_steps, pa_obs *obs_out, double *betas_out, int32_t *K_out);

/* ---- Batches of independent runs ------------------------------------------
 * M independent PA runs, possibly with different q, L, R, theta and
 * schedules, advanced together: each temperature step is six launches that
 * cover every run (weights, copy numbers, parent map, one persistent sweep
 * kernel over all runs' replica groups, estimators, step counter), so a
 * captured CUDA graph of one step is replayed for the whole schedule.  All
 * runs of a batch share one seed and should differ in cfg.stream; run m then
 * gives exactly what a lone run (pa_init with cfg) gives on the same schedule. */
typedef struct {
    pa_config cfg;        /* as for pa_init; every run of a batch has the same seed  */
    const double *betas;  /* betas[0..K] (host, read during pa_batch_create);
                             betas[0] must equal cfg.beta0                          */
    int32_t K;            /* temperature steps, >= 1                                 */
    int32_t theta;        /* sweeps per step, >= 0                                   */
} pa_run_desc;

typedef struct pa_batch pa_batch;

/* Allocates every run's buffers, uploads all steps' parameters and enqueues
 * the initial populations with their step-0 estimators (synchronises).
 * Errors: PA_ERR_INVALID for M outside 1..1024, any invalid run (as pa_init),
 * differing seeds, K < 1, theta < 0 or a non-finite or negative beta;
 * PA_ERR_TOO_LARGE for a run whose replica is too large (as pa_init);
 * PA_ERR_NOMEM / PA_ERR_CUDA on allocation or launch failures. */
pa_status pa_batch_create(const pa_run_desc *runs, int32_t M, void *cuda_stream, pa_batch **out);

/* Picks the sweep kernel's shared-memory budget per block (which sets the
 * replicas per block of every run) and threads per block by timing the first
 * three temperature steps for each candidate from the same initial
 * populations, then restarts from them.  Results are cached per GPU (name and
 * SM count) and batch shape for the process and, when the environment
 * variable PA_AUTOTUNE_CACHE names a file, in that file (one line per shape,
 * appended), where later processes find them.  Only before pa_batch_run
 * (PA_ERR_STATE after). */
pa_status pa_batch_autotune(pa_batch *b, int32_t *smem_budget_out, int32_t *threads_out);

/* Sets the budget (bytes, >= the largest replica) and threads per block
 * (multiple of 32, 64..1024) by hand; PA_ERR_INVALID if they do not fit. */
pa_status pa_batch_set_launch(pa_batch *b, int32_t smem_budget, int32_t threads);

/* Current launch shape (any pointer may be NULL). */
pa_status pa_batch_get_launch(pa_batch *b, int32_t *smem_budget, int32_t *threads, int32_t *blocks);

/* Runs every run's schedule to its end (runs with fewer steps idle); use_graph
 * = 1 captures one step as a CUDA graph and launches it max(K) times.
 * Synchronises; returns PA_ERR_CAPACITY if a run outgrew its capacity.
 * A batch runs once (PA_ERR_STATE on a second call). */
pa_status pa_batch_run(pa_batch *b, int32_t use_graph);

/* Estimators of run m at steps 0..K_m (host, K_m + 1 records). */
pa_status pa_batch_observables(pa_batch *b, int32_t m, pa_obs *out);

/* Replicas [slot_begin, slot_begin + count) of run m's current population, in
 * the canonical [count][L][L] layout (host; synchronises). */
pa_status pa_batch_get_spins(pa_batch *b, int32_t m, int64_t slot_begin, int64_t count, uint8_t *host);

/* Current population size of run m (synchronises); returns that run's error
 * (e.g. PA_ERR_CAPACITY) if it stopped. */
pa_status pa_batch_population_size(pa_batch *b, int32_t m, int32_t *R_out);

/* Per-replica energies E_j (Eq. 3) and occupations of the most common state
 * Mt_j (Eq. 5) of run m's current population, [R_i] int32 each, into host
 * memory (synchronises); either pointer may be NULL. */
pa_status pa_batch_measurements(pa_batch *b, int32_t m, int32_t *E_out, int32_t *Mt_out);

/* Releases the batch (synchronises its stream). */
void pa_batch_destroy(pa_batch *b);

/* Checkpoint of the current population (Sec. 2: the PA state between
 * temperature steps): configuration, step, inverse temperature, ln Z, spins,
 * energies, occupations, energy histogram, family ids and the latest
 * estimators, with a checksum.  The random numbers are counter-based, so a
 * run resumed with pa_load continues bit for bit as the uninterrupted run.
 * Synchronises.  PA_ERR_STATE with a resample pending or a failed context;
 * PA_ERR_INVALID if the file cannot be written.  Spins are stored in the
 * canonical layout [replica][y][x], one byte per spin (format version 4), so
 * files do not depend on the device layout; integers and doubles are stored
 * in the machine's byte order. */
pa_status pa_save(pa_ctx *ctx, const char *path);

/* Creates a context from a checkpoint written by pa_save (synchronises).
 * PA_ERR_INVALID for a missing, truncated or corrupted file (bad header,
 * version, sizes, checksum or a state outside 0..q-1: checked before any
 * device work); otherwise as pa_init. */
pa_status pa_load(const char *path, void *cuda_stream, pa_ctx **out);

/* Releases the context and its device memory (synchronises its stream). */
void pa_destroy(pa_ctx *ctx);

/* Static description of a status code. */
const char *pa_status_str(pa_status s);

/* The last CUDA error string recorded by any call on this thread ("" if none). */
const char *pa_last_cuda_error(void);

/* Launch-shape control for the sweep kernel: replicas per block and threads
 * per block (0 = automatic).  Any choice gives bit-identical results; this
 * exists for autotuning and for tests that check exactly that.  Automatic:
 * 96 KB of lattices and up to 512 threads per block (two blocks per SM), or,
 * for L = 128 and 256 with states of at most five bits and at least 16
 * replicas per SM, one block of 1024 threads per SM holding as many whole
 * passes of lattices as fit 200 KB.  Errors: PA_ERR_INVALID for a shape that
 * does not fit (threads not a multiple of 32 or above 1024, lattices above
 * 200 KB); PA_ERR_TOO_LARGE if one lattice alone exceeds it. */
pa_status pa_set_launch(pa_ctx *ctx, int32_t replicas_per_block, int32_t threads_per_block);

/* The sweep kernel's current launch shape: replicas per block, threads per
 * block and blocks (persistent grid).  Any pointer may be NULL. */
pa_status pa_get_launch(pa_ctx *ctx, int32_t *replicas_per_block, int32_t *threads_per_block, int32_t *blocks);

/* Number of kernels this library has launched on any context since the
 * process started (a host-side counter; graph launches count their nodes). */
int64_t pa_kernel_launch_count(void);

/* Kernel timing with CUDA events recorded on the context's stream around each
 * sweep launch (the fused gather + theta sweeps + measurement kernel) and
 * around each resampling sequence.  enable = 1 clears the totals and starts
 * recording; 0 stops.  Not available inside pa_run(use_graph = 1). */
pa_status pa_profile(pa_ctx *ctx, int32_t enable);

/* Synchronises and returns the summed event times (milliseconds) and launch
 * counts recorded since profiling was enabled: [0] sweep kernel, [1]
 * resampling kernels.  Any pointer may be NULL. */
pa_status pa_profile_read(pa_ctx *ctx, double *ms_out2, int64_t *launches_out2);

/* ---- One population spread over several GPUs (Sec. 2: the replicas are
 * independent between resampling steps; a step couples them only through
 * the normaliser Q_i and the copy-number offsets) ------------------------
 * Rank g of `world` holds a contiguous range of global slots, about R/world
 * replicas.  Random numbers are keyed by global slot and global replica
 * index, and S is an exact sum of the histogram-weighted Boltzmann factors, so
 * any number of ranks gives the population, energies, estimators and ln Z of
 * one GPU (pa_init) bit for bit.  A rank's children are placed by
 * pa_shard_plan; it sends each other rank the runs of its children bound
 * there (a run: consecutive children of one parent), as the parent replica
 * with a child count, so it never sends more than its own replicas plus one
 * run per destination, and the receiving rank's next sweep gathers its new
 * replicas from the runs.  The caller moves data between the calls (the
 * library calls no collective):
 *   pa_shard_init                                  (each rank)
 *   sum hist, sums, fam over ranks; pa_shard_finalize(beta_0)
 *   for each step i:
 *     pa_shard_counts(dbeta_i, i, &T)              (needs the summed hist)
 *     gather T of every rank into totals[world]
 *     pa_shard_pack(totals, send_counts)           (runs for each rank)
 *     exchange the counts: recv_counts[g] = rank g's send_counts[this rank]
 *     exchange the runs: the send_counts[d] runs from entry sum_{d'<d}
 *       send_counts[d'] of send (replica_words 32-bit words each), send_cnt
 *       (one int32 each) and, with families, send_anc go to rank d; rank g's
 *       runs arrive in recv, recv_cnt, recv_anc, sources in rank order
 *     pa_shard_accept(recv_counts); pa_sweep(beta_i, theta, i)
 *     sum hist, sums, fam over ranks; pa_shard_finalize(beta_i)
 * Device buffers the caller reads or writes (owned by the context; recv and
 * recv_anc change with every step: query them after pa_shard_pack). */
typedef struct {
    int32_t *hist;          /* [n_bins] energy histogram (this rank's, to be summed in place) */
    int64_t *sums;          /* [4] sum E, sum E^2, sum Mt, near ties (this rank's, to be summed in place) */
    int32_t *fam;           /* [R] family counts (this rank's, to be summed); NULL without families */
    uint32_t *send;         /* [capacity + world runs x replica_words] run parents packed by pa_shard_pack */
    int32_t *send_anc;      /* their family ids; NULL without families */
    int32_t *send_cnt;      /* their child counts */
    uint32_t *recv;         /* [capacity runs x replica_words] where the runs for this rank arrive */
    int32_t *recv_anc;      /* NULL without families */
    int32_t *recv_cnt;      /* child counts of the received runs */
    int64_t replica_words;  /* 32-bit words per replica in the device layout */
    int64_t capacity;       /* replicas this rank can hold */
    int64_t n_bins;         /* 2N + 1 */
} pa_shard_buffers;

/* The exchange plan of one step (host only; no GPU needed): totals[g] = the
 * number of children rank g's replicas have after resampling.  The new
 * population has R_new = sum totals replicas; rank g's children are the new
 * global slots [O_g, O_g + totals[g]), O_g = sum_{h<g} totals[h], and rank d
 * holds the new slots [floor(d R_new / world), floor((d+1) R_new / world)).
 * Writes R_new, this rank's new range [lo, hi), send_counts[d] (replicas it
 * sends to rank d) and recv_counts[g] (replicas it receives from rank g); any
 * output pointer may be NULL.  PA_ERR_INVALID for a bad rank or world or a
 * negative total, PA_ERR_CAPACITY for R_new outside 1 .. 2^24 - 1. */
pa_status pa_shard_plan(const int64_t *totals, int32_t world, int32_t rank, int64_t *R_new, int64_t *lo, int64_t *hi,
                        int64_t *send_counts, int64_t *recv_counts);

/* Rank `rank` of `world` (2..1024) of the population cfg describes (cfg->R
 * and cfg->R_cap are the whole population's): initial replicas of the global
 * slots [floor(rank R / world), floor((rank+1) R / world)) with their
 * measurements (synchronises).  Errors as pa_init. */
pa_status pa_shard_init(const pa_config *cfg, int32_t rank, int32_t world, void *cuda_stream, pa_ctx **out);

/* The device buffers of the exchange (see above).  PA_ERR_STATE unless the
 * context came from pa_shard_init. */
pa_status pa_shard_get_buffers(pa_ctx *ctx, pa_shard_buffers *out);

/* Resampling of this rank's replicas from the summed histogram (Sec. 2 step 2,
 * Eq. 2; arithmetic as pa_resample): ln Q_i, copy numbers keyed by global
 * replica index, their scan and the local parent map.  Synchronises and writes
 * the number of this rank's children to *local_total.  PA_ERR_STATE out of
 * order, PA_ERR_CAPACITY if the children exceed this rank's capacity (the
 * population stays at step i-1). */
pa_status pa_shard_counts(pa_ctx *ctx, double dbeta, int32_t step, int64_t *local_total);

/* Plans the exchange (pa_shard_plan with every rank's total, host int64
 * [world]) and packs, destination by destination, the runs of this rank's
 * children into send / send_cnt / send_anc; synchronises and writes the
 * number of runs for each rank into send_counts (host int64[world]).
 * PA_ERR_CAPACITY if the new local range exceeds the capacity. */
pa_status pa_shard_pack(pa_ctx *ctx, const int64_t *totals, int64_t *send_counts);

/* After the exchange has filled recv, recv_cnt (and recv_anc) with
 * recv_counts[g] runs from each rank g (host int64[world]): the runs become
 * the parents of this rank's new replicas, global slots [lo, hi) of the plan,
 * which the next pa_sweep gathers.  PA_ERR_INVALID for counts that cannot
 * fill the range (a device check of the child counts flags the same, reported
 * by the next synchronising call). */
pa_status pa_shard_accept(pa_ctx *ctx, const int64_t *recv_counts);

/* Estimators of the step (Sec. 2 step 4) from the summed sums, family counts
 * and histogram; ln Z_i = ln Z_{i-1} + ln Q_i.  Read them with pa_observables. */
pa_status pa_shard_finalize(pa_ctx *ctx, double beta);

/* This rank's current global slot range [slot0, slot0 + count) and the size
 * of the whole population (synchronises). */
pa_status pa_shard_range(pa_ctx *ctx, int64_t *slot0, int64_t *count, int64_t *R_all);

/* Resampling without any device allocation.  This call has no counterpart in
 * the paper: it exists for callers that may not allocate device memory --
 * plug-ins whose host framework owns every device allocation (a cudaMalloc
 * behind its back would escape its accounting and limits), and runtimes that
 * must not call the allocator once set up (an allocation can synchronise the
 * device or fail under memory pressure in the middle of their work).
 *
 * It computes, for the R_prev energies E[0..R_prev) (device int32, each in
 * [-2N, 0], N = L*L) of a population, the same quantities as pa_resample
 * (same arithmetic, bit for bit): ln Q for the step dbeta, the copy numbers
 * under `mode` (random words keyed by seed, step and rng_stream, 0..255, the
 * pa_config stream of the run) and the parent map of the new population,
 * parent[0..R_i) (device int32, capacity parent_cap >= R_prev), with the new
 * size in *R_out and ln Q in *lnQ_out (both device pointers).  The work is
 * only enqueued on cuda_stream; read the outputs after synchronising.  If an
 * energy lies outside [-2N, 0] *R_out becomes -PA_ERR_INVALID, and if R_i would
 * exceed parent_cap, -PA_ERR_CAPACITY; parent is then unspecified.  The
 * Boltzmann factors are computed on the host and copied from host memory into
 * the working memory (skipped when the previous call on that device used the
 * same dbeta); that copy may wait for earlier work on cuda_stream.
 *
 * Working memory: one fixed array of about 3.6 MB inside the library's device
 * image, held by every GPU that loads the library until the process exits.
 * Limits: L <= 256 and R_prev <= 262144 (larger sizes return
 * PA_ERR_TOO_LARGE); parent_cap is the caller's and is not limited.  The first
 * call on each device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current); make that first call before
 * any stream capture.  All calls share the array and overwrite it: calls whose
 * work overlaps on the GPU race, calls ordered on one stream do not.  Returns
 * PA_ERR_INVALID for null pointers, odd L, R_prev < 1, R_target < 1,
 * parent_cap < R_prev, an unknown mode, rng_stream outside 0..255 or a
 * non-finite dbeta, and PA_ERR_CUDA if a launch fails or if a CUDA error is
 * already pending on the calling thread (left pending for its owner). */
pa_status pa_resample_noalloc(const int32_t *E, int32_t R_prev, int32_t L, double dbeta, int32_t R_target,
                              int32_t mode, int32_t step, uint64_t seed, int32_t rng_stream, int32_t *parent,
                              int32_t parent_cap, double *lnQ_out, int32_t *R_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PA_H */
