/*
 * sr.h -- C ABI of libsr: synchronous relaxation of the continuous-time
 * n-fold-way Ising simulation (Lubachevsky & Weiss, "Synchronous Relaxation
 * for Parallel Ising Spin Simulations"), GPU implementation for sm_103a.
 *
 * The lattice G (§2) is an L x L periodic square lattice of spins s = +-1,
 * partitioned into rectangular regions G_i of region_w x region_h sites
 * (§5: "The set G is partitioned into subsets G_i").  Each region plays the
 * part of one processing element of §4: it generates its own n-fold-way history
 * (§3) over a window [t_c, t_c + T_max), reading its neighbours' boundary
 * histories from the previous iteration; the iterations repeat until no
 * boundary history changes (§4, boxed procedure; §5).
 *
 * Conventions shared by every call:
 *   - Return value: SR_OK (0) on success, a negative SR_E* code otherwise.
 *     No call throws.  sr_strerror() names a code.
 *   - The library owns every device buffer it allocates; the caller owns every
 *     buffer it passes in (host memory unless the name ends in _device).
 *   - A context is not thread-safe.  All GPU work of a context runs on the
 *     stream given at creation (or a stream the library creates).
 *   - Spin arrays are int8, row-major, index y * L + x, values +1 / -1.
 *   - Region r covers x in [rx*region_w, (rx+1)*region_w) and y in
 *     [ry*region_h, (ry+1)*region_h) with r = ry * (L / region_w) + rx.
 */
#ifndef SR_H
#define SR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SR_OK 0
#define SR_EINVAL (-1)          /* bad argument (shape, L < 3, T <= 0, t0 != committed time ...) */
#define SR_ENOMEM (-2)          /* device or host allocation failed */
#define SR_ECUDA (-3)           /* a CUDA call failed */
#define SR_NOT_CONVERGED (-4)   /* iteration cap reached before a fixed point (§4, "UNTIL") */
#define SR_CAPACITY (-5)        /* boundary history larger than the largest allowed capacity */
#define SR_TIMEOUT (-6)         /* a bounded wait ran out: a grid-wide synchronize, or no task
                                   published for a whole limit (asynchronous schedule) */
#define SR_EUNSUPPORTED (-7)    /* valid but not supported by this build (e.g. region wider than 32) */
#define SR_ETOOLARGE (-8)       /* problem needs more than the fixed scratch of sr_run_noalloc */

/* ---- initial spins ---- */
#define SR_INIT_FAIR_COIN 0     /* bit 0 of Philox4x32-10(counter = (site, 0, 0, 1), key = seed) */
#define SR_INIT_ALL_UP 1
#define SR_INIT_ALL_DOWN 2

/* ---- flip probability p (§2) ---- */
#define SR_RATES_METROPOLIS 0   /* p = min(1, theta), Eq. 2.2 */
#define SR_RATES_GLAUBER 1      /* p = theta / (1 + theta), Eq. 2.3 */

typedef struct sr_ctx sr_ctx;   /* opaque, library-owned */

/* Creation parameters.  Zero-initialise and set what you need. */
typedef struct sr_params {
  int L;                        /* lattice side, >= 3 (§2, periodic in both directions) */
  double J;                     /* coupling of Eq. 2.1 (each nearest-neighbour bond counted once) */
  double h;                     /* field H of Eq. 2.1 */
  double T;                     /* temperature k_B T_abs of Eq. 2.2, > 0 */
  int region_w, region_h;       /* region extent in x and y; must divide L; each <= 32 */
  uint64_t seed;                /* key of every random stream */
  int init_mode;                /* SR_INIT_* */
  int rates;                    /* SR_RATES_* */
  int capacity;                 /* boundary events per region edge per iteration; 0 = automatic
                                   (grows by doubling when exceeded, see sr_run_windows) */
  int max_iters;                /* iteration cap per window; 0 = 1<<16 */
  int trace_capacity;           /* committed events recorded per region; 0 = no trace */
  int lanes_per_region;         /* 32 = one warp per region; 1 or 0 = one lane per region */
  int lanes_per_warp;           /* with one lane per region: region lanes in each warp (1..32);
                                   fewer lanes give more warps and less divergence; 0 = automatic */
  int time_arith;               /* waiting-time arithmetic with one lane per region: 1 = FP64
                                   instructions, 2 = integer-emulated doubles (identical bits),
                                   0 = automatic */
  int threads_per_block;        /* region slots per block (lanes, or warps with a warp per
                                   region); 0 = automatic */
  int blocks;                   /* 0 = automatic (all regions resident if they fit) */
  int barrier_timeout_ms;       /* bound on each wait of the relaxation kernel (a grid-wide
                                   synchronize; with the asynchronous schedule, a stretch with
                                   no task published); 0 = 2000 */
  int replay_records;           /* incremental replay (one lane per region): checkpoints kept per
                                   region of the break points consumed in a pass, so the next pass
                                   restarts after its last unchanged input; 0 = 64, -1 = off */
  int fresh_steps;              /* 0: each step continues every region's clock and random numbers
                                   (§5, "Subsequent steps"); 1: the alternate approach of §5:
                                   at every committed time each region's clock restarts with new
                                   random numbers (event j of window w: Philox counter
                                   (j, w, region, 2)); the trajectory then depends on the window
                                   ends.  One lane per region only (SR_EUNSUPPORTED otherwise) */
  int score;                    /* 1: also keep, per region, the committed events by class and
                                   the integrals of N_k dt (the statistics of the path's score
                                   function, see sr_score); one lane per region, no incremental
                                   replay (SR_EUNSUPPORTED with a warp per region) */
  int schedule;                 /* regions to slots in each iteration: 1 static (slot s owns
                                   regions s, s + slots, ...), 2 dynamic (warps claim the next
                                   regions from a counter; one more grid-wide synchronize per
                                   iteration), 3 asynchronous (one lane per region only: each
                                   lattice iterates and commits on its own through a task queue,
                                   with no grid-wide synchronize), 0 automatic (asynchronous
                                   for batches with one lane per region, dynamic for other
                                   batches or when regions outnumber slots, else static) */
  int test_barrier_skip_block;  /* test hook: this block never arrives at a barrier; -1 = off */
  void* stream;                 /* cudaStream_t; NULL = the library creates its own */
} sr_params;

/* One lattice of a batch (sr_create_batch): its own side, Hamiltonian,
 * temperature, seed, initial spins, rates and, optionally, region shape (the
 * partition of §5 into subsets G_i); every other setting comes from the
 * sr_params given with the batch. */
typedef struct sr_replica {
  int L;                        /* side, a multiple of the region extents, >= 3 */
  double J, h, T;               /* Eq. 2.1 and the temperature of Eq. 2.2 / 2.3 */
  uint64_t seed;                /* Philox key of this lattice's draws and fair-coin spins */
  int init_mode;                /* SR_INIT_* */
  int rates;                    /* SR_RATES_* */
  int region_w, region_h;       /* this lattice's region extents (each <= 32); 0 = the batch's
                                   common sr_params.region_w / region_h.  The rate grid follows
                                   the shape: F = 63 - bitlen(w h) */
} sr_replica;

/* Observables and counters (reduced over all regions at the committed time). */
typedef struct sr_obs {
  double t_c;                   /* committed time (§4) */
  int64_t mag;                  /* sum of spins */
  int64_t bonds;                /* sum over nearest-neighbour bonds of s s' */
  double m;                     /* mag / L^2 */
  double E;                     /* -J bonds - h mag (Eq. 2.1) */
  double int_mag;               /* integral of mag dt over [0, t_c] */
  double int_bonds;             /* integral of bonds dt over [0, t_c] */
  uint64_t committed;           /* committed events since creation */
  uint64_t generated;           /* events generated in every iteration (committed or discarded) */
  uint64_t breaks;              /* break points processed in every iteration (§5) */
  uint64_t windows;             /* committed windows */
  uint64_t iterations;          /* iterations over all windows */
  uint64_t sum_f;               /* sum over committed windows of f (§6): the most boundary
                                   events of a region in an iteration of the window */
  uint32_t last_iters;          /* iterations of the last window (g of §6) */
  uint32_t max_iters_seen;      /* largest g seen */
  uint32_t max_f;               /* largest number of boundary events of one region in one
                                   iteration (f of §6) */
  uint32_t capacity;            /* current history capacity per edge */
  uint64_t launches;            /* kernels this context has launched since creation */
  uint64_t region_passes;       /* region iterations replayed */
  uint64_t region_skips;        /* region iterations skipped (inputs unchanged) */
  uint64_t run_cycles;          /* SM cycles region slots spent on their regions, summed */
  uint64_t run_cycles_max;      /* the same for the busiest slot */
  uint64_t slots;               /* region slots (lanes or warps) that reported */
  double relax_ms;              /* device time of this context's relaxation launches since
                                   creation (CUDA events around each launch on its stream) */
  uint64_t relax_launches;      /* relaxation launches timed in relax_ms */
} sr_obs;

/* Create a context with Metropolis rates, fair-coin initial spins and
 * automatic settings.  Computes p_k for the ten classes k = 5*[s=+1] + n_up
 * (§3, Eqs. 3.1-3.2), allocates the device state, initialises the spins, the
 * class counts N_k and every region's first waiting time (Eq. 3.4 with
 * tau_0 = 0, §5 "First iteration, first step"); committed time t_c = 0.
 * *out receives the handle (NULL on failure).  Errors: SR_EINVAL, SR_ENOMEM,
 * SR_ECUDA, SR_EUNSUPPORTED. */
int sr_create(sr_ctx** out, int L, double J, double h, double T, int region_w, int region_h,
              uint64_t seed);

/* Same as sr_create with every setting of sr_params. */
int sr_create_ex(sr_ctx** out, const sr_params* params);

/* One step of the §4 procedure with T_max = Tw: make the canonical assumption
 * (no neighbour flips, §5), iterate "generate / synchronize / compare /
 * synchronize" until no region's boundary history changes, then increment the
 * committed time by Tw.  t0 must equal the committed time.  Blocks until the
 * window is done.  Errors: SR_EINVAL (t0 != t_c, Tw <= 0), SR_NOT_CONVERGED,
 * SR_CAPACITY, SR_TIMEOUT, SR_ECUDA.  On error the committed state is that of
 * the last window that converged. */
int sr_run_window(sr_ctx* ctx, double t0, double Tw);

/* n consecutive windows of length Tw from t0 (= t_c), in one persistent
 * launch; window k ends at the double t0 + Tw + ... + Tw (k+1 additions).
 * When a window overflows the history capacity and capacity was automatic,
 * the capacity is doubled and the remaining windows are re-run from the last
 * committed state (the result does not depend on the capacity).  Same errors as
 * sr_run_window. */
int sr_run_windows(sr_ctx* ctx, double t0, double Tw, int n);

/* Observables at the committed time; *out is caller-owned.  Errors: SR_EINVAL,
 * SR_ECUDA.  In a batch context: lattice 0 (the launch counters region_passes
 * .. slots cover the whole batch). */
int sr_observables(sr_ctx* ctx, sr_obs* out);

/* ---- batches of independent lattices ----
 * The paper simulates one lattice.  A batch holds n lattices that never
 * interact; each follows the §4 procedure on its own, with its own windows,
 * iterations and results, bit for bit the same as a context of its own with
 * the same region shape.  All lattices share one persistent launch: their
 * regions fill the GPU together, and each lattice commits as soon as its own
 * boundary histories stop changing.  Region r of lattice b is global region
 * off_b + r, off_b = sum of the region counts of lattices 0 .. b-1.
 *
 * The single-lattice calls act on a batch context as follows: sr_run_window(s)
 * runs every lattice (t0 must equal every lattice's t_c); sr_reset resets
 * every lattice; sr_observables, sr_get_spins(_device), sr_set_spins(_device),
 * sr_get_carry, sr_get_trace, sr_get_window_iters and sr_get_info refer to
 * lattice 0. */

/* reps: n >= 1 caller-owned descriptors (copied); common: region shape and
 * the settings of sr_params other than L, J, h, T, seed, init_mode, rates
 * (ignored).  Errors: SR_EINVAL, SR_ENOMEM, SR_ECUDA, SR_EUNSUPPORTED. */
int sr_create_batch(sr_ctx** out, const sr_replica* reps, int n, const sr_params* common);

/* For every lattice b, n_windows[b] >= 0 windows of length Tw[b] (> 0 where
 * n_windows[b] > 0) from its committed time, all in one persistent launch
 * (more after a capacity growth, as in sr_run_windows).  Host arrays of n
 * entries.  Errors as sr_run_windows; on error every lattice keeps the state of
 * its last converged window. */
int sr_run_batch(sr_ctx* ctx, const double* Tw, const int* n_windows);

/* ---- relaxation launches replayed from a CUDA graph ----
 * One launch is the whole procedure of §4 for the launch's windows (passes,
 * the fixed-point test, commits); the graph form has no counterpart in the
 * paper.  on != 0: every later relaxation launch of this context (those of
 * sr_run_window(s), sr_run_batch and sr_run_batch_adaptive) runs as one CUDA
 * graph -- the uploads of the launch plan, the resets of the launch state,
 * the persistent kernel as a cooperative kernel node and the read-back of
 * the status -- launched on the context's stream.  The graph is captured (on
 * a stream of its own) at the first launch and replayed while the kernel's
 * parameters and the number of first tasks stay the same; the plan's values
 * (committed times, window lengths and counts, first tasks) are staged in
 * pinned host memory that the graph's copies read each time it runs.  A new
 * ring length or history capacity recaptures it.  Trajectories, counts and
 * observables are those of launches without the graph, bit for bit;
 * sr_obs.relax_ms then times whole graphs (uploads and read-back included).
 * The call synchronises the context's stream; on == 0 frees the graph and
 * its staging.  Errors: SR_EINVAL (ctx NULL), SR_ENOMEM (pinned staging),
 * SR_ECUDA; a later launch returns SR_EUNSUPPORTED if the capture or the
 * instantiation is refused. */
int sr_set_graph_launch(sr_ctx* ctx, int on);

/* Graph captures and graph launches of this context so far (either pointer
 * may be NULL).  Errors: SR_EINVAL (ctx NULL). */
int sr_get_graph_stats(sr_ctx* ctx, unsigned long long* captures, unsigned long long* replays);

/* ---- window lengths matched to event rates ----
 * The paper leaves T_max free (§4, §6: the cost per step grows with the
 * boundary events f per region and the iterations g).  Window ends are not
 * break points, so the trajectory does not depend on the window lengths; only
 * the cost does.  The adaptive runner sizes each lattice's windows so that a
 * region sees about `kappa` committed events per window. */
typedef struct sr_adapt {
  double kappa;                 /* target committed events per region per window; 0 = 8 */
  double chunk;                 /* simulated time between window-length updates; 0 = 1 */
  double tw_first;              /* window length of a lattice's first chunk; 0 = 1/16 */
  double tw_min;                /* smallest window length; 0 = 2^-10 */
  double tw_max;                /* largest window length; 0 = chunk */
} sr_adapt;

/* Advance every lattice b from its committed time to t_end[b] (>= t_c; equal
 * means nothing to do) in chunks of `chunk` time units, all lattices of a
 * chunk in one persistent launch.  In each chunk lattice b runs windows of
 * length Tw_b = 2^round(log2(kappa / rho_b)) clamped to [tw_min, tw_max], with
 * rho_b its committed events per region per unit time in its previous chunk
 * (tw_first before it has one); a chunk ends early at t_end[b].  Window ends
 * are then sums of powers of two, exact in double for dyadic t_c and t_end.
 * opts may be NULL (all defaults).  last_tw (host, n entries, may be NULL)
 * receives each lattice's last window length.  Errors as sr_run_batch, plus
 * SR_EINVAL for t_end[b] < t_c or non-positive / non-finite options. */
int sr_run_batch_adaptive(sr_ctx* ctx, const double* t_end, const sr_adapt* opts, double* last_tw);

/* ---- autotuner ----
 * Chooses, for a batch of lattices, the region shape of every lattice, the
 * region lanes per warp (automatic, 8, 16, 32) and kappa (4, 8, 11.3, 16) by
 * timing trial runs of the real lattices.  A warm-up run (the first of the
 * shapes below that divides every L, to t = 8 t_trial) measures each
 * lattice's committed events per site per unit time rho_b over its second
 * half and keeps the spins it ends with; every trial starts from those
 * spins (the coarsened configurations of a long run, not the first quench
 * from the initial spins), runs the adaptive runner with one launch per
 * t_trial, untimed to t_trial (the window lengths settle), then timed to
 * 3 t_trial, and scores committed flips per second; a candidate replaces
 * the best so far only when it scores at least 2% higher.  One
 * coordinate at a time:
 *   1. one shape for every lattice, among 8x8, 16x8, 16x16, 32x16 and 32x32;
 *   2. a shape per lattice: the largest of those shapes (dividing L_b) with
 *      rho_b x sites <= R, else the smallest, for R in {32, 64, 128, 256}.
 *      A lattice's chain of iterations per unit time grows with the events
 *      per region (§6: the cost of a step grows with f and g), so small
 *      regions shorten the hot lattices' chains and large regions keep the
 *      cold ones' boundary traffic low;
 *   3. kappa, then 4. lanes per warp, with the best assignment.
 * The trajectory of a lattice depends on its region shape (its random streams
 * are per region) but not on the other choices.  common supplies every other
 * setting (as in sr_create_batch; shapes in reps and common are ignored).
 * t_trial > 0; 0 = 1.0.  region_wh (host, 2 n ints, may be NULL) receives
 * each lattice's chosen (w, h).  Blocks until done; allocates and frees
 * contexts.  Errors: those of sr_create_batch and sr_run_batch_adaptive;
 * SR_EUNSUPPORTED when no candidate shape divides every L. */
typedef struct sr_tune {
  int region_w, region_h;       /* chosen region shape of lattice 0 */
  int lanes_per_warp;           /* chosen region lanes per warp (0 = automatic) */
  double kappa;                 /* chosen target events per region per window */
  double flips_per_s;           /* trial throughput of the choice */
  int trials;                   /* configurations timed */
  double rate_threshold;        /* R of step 2 when a shape per lattice won, else 0 */
} sr_tune;
int sr_autotune(const sr_replica* reps, int n, const sr_params* common, double t_trial,
                sr_tune* out, int* region_wh);

/* ---- score function (differentiation) ----
 * A path of the chain of §3 on [0, t_c] has log-likelihood
 *   log L = sum over events of log p_k(event) - integral of sum_k N_k p_k dt
 * (k the class of the flipped site before the flip, N_k the class counts).
 * Its derivative, the score S = d log L / d theta for theta = (beta, h, J)
 * with beta = 1/T, gives unbiased gradients of expectations: d E[A] / d theta
 * = E[A S] for any A of the path (plus A's own explicit dependence).  Score
 * mode (sr_params.score) keeps per region, for the committed path, C_k (events
 * by class) and I_k (the integral of N_k dt; exact 128-bit fixed point within a
 * window, accumulated over windows in double).  The paper has no counterpart. */

/* S[b][0..2] = d log L / d(beta, h, J) of each lattice b's committed path:
 * sum_k C_k d log p_k - sum_k I_k d p_k, with d log p_k of Metropolis or
 * Glauber rates (Eqs. 2.2, 2.3) at the lattice's (J, h, T).  Metropolis:
 * -d(beta dE) where dE > 0, 0 where dE < 0, and -d(beta dE) / 2 on the kink
 * dE = 0 of min(1, exp(-beta dE)) (the mean of its left and right
 * derivatives; e.g. the n_up = 2 classes at h = 0).  out: host, 3 * n doubles.
 * Blocks.  Errors: SR_EINVAL, SR_EUNSUPPORTED (not score mode), SR_ECUDA. */
int sr_score(sr_ctx* ctx, double* out);

/* The statistics themselves for lattice `replica`, summed over its regions:
 * counts[k] = C_k, occupancy[k] = I_k (host arrays of 10; either may be NULL). */
int sr_score_stats(sr_ctx* ctx, int replica, uint64_t* counts, double* occupancy);

/* Backward of n replicas' time averages through their scores, on device
 * arrays (row-major, caller-owned): A [n][m] the averages, gA [n][m] the
 * gradient arriving at them, S [n][nq] the scores, E [n][m][nq] the averages'
 * explicit derivatives (may be NULL).  Writes G [n][nq]:
 * G[i][q] = sum_j gA[i][j] ((A[i][j] - base_ij) S[i][q] + E[i][j][q]),
 * base_ij = the mean of A[.][j] over the other replicas (a control variate;
 * it keeps the estimate unbiased since E[S] = 0).  Runs on `stream`, blocks.
 * Errors: SR_EINVAL, SR_ENOMEM, SR_ECUDA. */
int sr_score_grad(int n, int m, int nq, const double* A, const double* gA, const double* S,
                  const double* E, double* G, void* stream);

/* Observables of lattice `replica` (0 <= replica < n).  Errors: SR_EINVAL,
 * SR_ECUDA. */
int sr_observables_replica(sr_ctx* ctx, int replica, sr_obs* out);

/* Committed spins of lattice `replica` into a host buffer of n = L_b^2 int8. */
int sr_get_spins_replica(sr_ctx* ctx, int replica, int8_t* host_out, size_t n);

/* Restart lattice `replica` alone from a given configuration (host buffer of
 * n = L_b^2 int8, > 0 = up, caller-owned; pinned memory makes the copy a
 * plain DMA): its t_c = 0, every region's clock restarts as at creation
 * (§5 "First iteration, first step"), its counters are cleared; the other
 * lattices are untouched.  Blocks.  Errors: SR_EINVAL, SR_ECUDA. */
int sr_set_spins_replica(sr_ctx* ctx, int replica, const int8_t* host_in, size_t n);

/* Clock state of lattice `replica` as sr_get_carry, n = its region count. */
int sr_get_carry_replica(sr_ctx* ctx, int replica, uint64_t* index, double* x, double* b,
                         double* t_last, size_t n);

/* Checkpoint and resume (§5, "Subsequent steps": the state a window carries
 * to the next is the committed spins, the pending event's index and random
 * pair, the hazard b accrued since t_last, and t_last).  A checkpoint holds,
 * for every lattice of ctx, its committed time, committed windows and
 * counters (sr_obs), and per region the committed spin rows, that clock
 * carry, the running integrals of the spin sum and of the owned bonds and, in
 * score mode, the path statistics.  Ring contents and boundary histories are
 * not kept: the presimulated pairs are a function of the event index, and
 * every window starts from empty histories (§5, "Statement 2").  A context
 * loaded from a checkpoint continues bit for bit as the saved one would.
 * The format is this build's own (native byte order, checked by a tag).
 *   sr_checkpoint_size: *bytes = the size of ctx's checkpoint.
 *   sr_checkpoint_save: write it to `buf`, caller-owned host memory of `bytes`.
 *   sr_checkpoint_load: restore it into ctx, whose lattices must have the same
 *     L, J, h, T, seed and rates, and the same region shape, score mode and
 *     step rule, as the saved context's; the trace (sr_get_trace) is not
 *     restored.
 * Errors: SR_EINVAL (null pointers, a size other than the checkpoint's, or a
 * checkpoint that does not match ctx; ctx is then unchanged), SR_ENOMEM,
 * SR_ECUDA. */
int sr_checkpoint_size(sr_ctx* ctx, size_t* bytes);
int sr_checkpoint_save(sr_ctx* ctx, void* buf, size_t bytes);
int sr_checkpoint_load(sr_ctx* ctx, const void* buf, size_t bytes);

/* Free everything; NULL-safe. */
void sr_destroy(sr_ctx* ctx);

/* Copy the committed spins into a caller buffer of n = L*L int8.  Errors:
 * SR_EINVAL (n != L*L), SR_ECUDA. */
int sr_get_spins(sr_ctx* ctx, int8_t* host_out, size_t n);

/* Same into a device buffer (caller-owned, n = L*L bytes); ordered on the
 * context's stream, returns without waiting. */
int sr_get_spins_device(sr_ctx* ctx, int8_t* dev_out, size_t n);

/* Restart from a given configuration: spins > 0 are up, others down; t_c = 0
 * and every region's clock restarts as at creation (event index 0, tau_0 = 0).
 * Counters are cleared.  Errors: SR_EINVAL (n != L*L), SR_ECUDA. */
int sr_set_spins(sr_ctx* ctx, const int8_t* host_in, size_t n);

/* Same from a device buffer; ordered on the context's stream. */
int sr_set_spins_device(sr_ctx* ctx, const int8_t* dev_in, size_t n);

/* Back to the creation-time initial state (t_c = 0, counters cleared). */
int sr_reset(sr_ctx* ctx);

/* Per-region clock state at t_c (§5, "Subsequent steps"): index i of the
 * pending event, x = -log U_i, b = integral of Lambda since the last event up
 * to time t_last.  Arrays of n = number of regions; any may be NULL.  The
 * event index equals the number of committed events of the region. */
int sr_get_carry(sr_ctx* ctx, uint64_t* index, double* x, double* b, double* t_last, size_t n);

/* Committed events of every region in order (requires trace_capacity > 0):
 * lens[r] = number of committed events of region r (entries beyond
 * trace_capacity were not recorded); times[r * cap + j], sites[r * cap + j]
 * (site = y * L + x) for j < min(lens[r], cap), cap = trace_capacity.  Any
 * pointer may be NULL. */
int sr_get_trace(sr_ctx* ctx, uint64_t* lens, double* times, uint32_t* sites, size_t n_regions,
                 size_t cap);

/* Iteration count g of each of the last n windows run by the last
 * sr_run_window(s) call (at most 4096); returns how many were written or a
 * negative code. */
int sr_get_window_iters(sr_ctx* ctx, uint32_t* out, size_t n);

/* f of §6 for the same windows: the largest number of boundary events
 * (events at boundary sites, §5) of any region in any iteration of the
 * window.  Same conventions as sr_get_window_iters. */
int sr_get_window_f(sr_ctx* ctx, uint32_t* out, size_t n);

/* Geometry and the fixed-point rate table actually used: P[k] / 2^F is the
 * flip probability of class k (the grid keeps Lambda = sum N_k p_k exact);
 * threads_per_block receives the region lanes per block.  Any pointer may be
 * NULL. */
int sr_get_info(sr_ctx* ctx, int* n_regions, int* frac_bits, uint64_t* P, int* threads_per_block,
                int* blocks);

/* Evaluate on the GPU the random pairs of events i0 .. i0+n-1 of one region:
 * x[j] = -log U_i (the numerator of Eq. 3.4) and kV[j], the 52-bit integer of
 * V_i = (2 kV + 1) 2^-53 (Phase 1 of §3), for counter (i, region) under seed.
 * Host arrays of n entries; either may be NULL.  Blocks until done.  Errors:
 * SR_EINVAL, SR_ENOMEM, SR_ECUDA. */
int sr_eval_draws(uint64_t seed, uint32_t region, uint64_t i0, size_t n, double* x, uint64_t* kV);

/* Evaluate on the GPU the integer-emulated IEEE double operations used by the
 * time formula of the event loop (Eqs. 3.4, 5.2-5.6): op 0 a+b, 1 a-b,
 * 2 a*b, 3 a/b (operands >= 0, b > 0 for division), 4 a converted from an
 * unsigned integer (bits of a) times 2^-F with F = (int)b.  out[i] receives the
 * result for a[i], b[i].  Host arrays of n doubles.  Blocks until done.  Errors:
 * SR_EINVAL, SR_ENOMEM, SR_ECUDA. */
int sr_eval_softfloat(int op, const double* a, const double* b, double* out, size_t n);

/* Run a whole simulation without allocating any memory.  The paper has no
 * counterpart: this exists for callers that cannot allocate GPU memory at the
 * point where they simulate, e.g. code that runs inside a memory-pool budget
 * that must not grow, plug-ins whose host forbids cudaMalloc/cudaFree in their
 * callbacks, or long-running services that pre-plan every allocation.
 *
 * It simulates an L x L lattice from t = 0 through n_windows windows of length
 * Tw (same method, same results as sr_create + sr_run_windows with automatic
 * settings except a fixed history capacity) and writes the final spins.  All
 * working state lives in one fixed scratch array of SR_NOALLOC_SCRATCH_BYTES
 * that every GPU loading this library holds until the process exits.
 *   spins_in   device, L*L int8 (> 0 = up), or NULL for fair-coin spins from seed
 *   spins_out  device, L*L int8, caller-owned, written with the spins at the end
 *   counts_out device, (L/region_w)*(L/region_h) uint64 committed events per
 *              region, or NULL
 *   stream     cudaStream_t to run on, or NULL for the default stream
 * The call blocks until done.  On the first call on a device it looks up the
 * scratch address for that device, so make that first call before any stream
 * capture.  Every call uses the same scratch: calls that overlap on the GPU
 * (other threads, other streams) race and must not be made.  Errors: SR_EINVAL,
 * SR_ETOOLARGE (the state does not fit the scratch), SR_EUNSUPPORTED,
 * SR_CAPACITY (more than 64 boundary events on one region edge in one
 * iteration), SR_NOT_CONVERGED, SR_TIMEOUT, SR_ECUDA. */
#define SR_NOALLOC_SCRATCH_BYTES (8u << 20)
int sr_run_noalloc(int L, double J, double h, double T, int region_w, int region_h, uint64_t seed,
                   const int8_t* spins_in, double Tw, int n_windows, int8_t* spins_out,
                   uint64_t* counts_out, void* stream);

/* Name of a status code (static string). */
const char* sr_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SR_H */
