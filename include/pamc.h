/*
 * pamc.h -- C ABI of the GB300 (sm_103a) augmented Population Annealing Monte
 * Carlo library (libpamc.so).
 *
 * Method: Khan, Redding, Shukla, "Leveraging Population Dynamics to Steer
 * Efficient Search in Large-Scale Combinatorial Optimization".  The library
 * runs Algorithm 1 (augmented PAMC) on one GPU:
 *   - population resampling by Boltzmann weights, Eq. 1-2 (systematic
 *     resampling over an integer prefix scan of fixed-point weights);
 *   - S single-spin sweeps per temperature step in a random order shared by
 *     all replicas, Eq. 3-4 (heat-bath) or Metropolis, and the Max-3-Cut
 *     three-state Potts update of Eq. 6-7 with the cascaded sampler of
 *     Suppl. S3;
 *   - the best cut M* (cut = (W - E)/2), the stagnation-driven adaptive
 *     temperature control and restart of Algorithm 1 / Sec. III.C, and the
 *     energy-preserving non-local cluster moves (NCM) of Sec. III.C.
 * Every result is bit-identical to the plain CPU restatement of the same
 * steps for the same seed: random numbers come from counter-keyed
 * Philox4x32-10, thresholds and resampling weights from a deterministic
 * binary64 exp, and all energies, fields and cuts are exact integers.
 *
 * Conventions:
 *   - Max-Cut weights w (symmetric, zero diagonal); Ising couplings J = -w,
 *     energy H(s) = -sum_{i<j} J_ij s_i s_j, W = sum_{i<j} w_ij.
 *   - Spins are int8 +1/-1 (Ising) or labels 0,1,2 (Potts), replica-major:
 *     element [r*n + i].
 *
 * Errors: every call returns a pamc_status; nothing aborts, traps or prints.
 * A failed call leaves the handle usable unless it returns PAMC_ERR_CUDA.
 * pamc_last_error() gives a one-line message for the last failure on a
 * handle.  Device-side waits are bounded; a wait that runs out reports
 * PAMC_ERR_TIMEOUT.
 *
 * Threading: a handle is used by one host thread at a time.  All device work
 * of a handle is ordered on the stream given at creation.
 */
#ifndef PAMC_H
#define PAMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pamc_handle_s *pamc_handle;

typedef enum {
    PAMC_OK = 0,
    PAMC_ERR_ARG = 1,      /* null pointer, bad size or bad parameter */
    PAMC_ERR_ASYM = 2,     /* coupling matrix not symmetric */
    PAMC_ERR_DIAG = 3,     /* nonzero diagonal / self loop */
    PAMC_ERR_RANGE = 4,    /* a value outside what the kernels represent */
    PAMC_ERR_OOM = 5,      /* device allocation failed */
    PAMC_ERR_CUDA = 6,     /* CUDA runtime error (message in pamc_last_error) */
    PAMC_ERR_TIMEOUT = 7,  /* a bounded device wait gave up */
    PAMC_ERR_STATE = 8     /* call out of order (e.g. pamc_step before pamc_init) */
} pamc_status;

/* Parameters of one run (the inputs of Algorithm 1). */
typedef struct {
    int32_t kind;           /* 0 Max-Cut (Ising), 1 Max-K-Cut (K-state Potts) */
    int32_t rule;           /* Ising: 0 heat-bath (Eq. 4), 1 Metropolis;
                               Potts: 0 cascaded sampler (Suppl. S3, K = 3),
                               2 softmax noisy argmax (Sec. III.F, Eq. 8-9, 2 <= K <= 8) */
    int32_t R;              /* population size */
    int32_t sweeps;         /* S, sweeps per temperature step */
    int32_t steps;          /* iterations; dbeta = (beta1-beta0)/(steps-1) */
    double beta0, beta1;    /* linear schedule; beta <- beta + Delta each step */
    int32_t stagnation;     /* 0 conventional PAMC, 1 adaptive control + NCM */
    int32_t z_rst;          /* restart every z_rst iterations; <= 0 never */
    int32_t cooldown_tau;   /* NCM cooldown tau */
    int32_t n_top;          /* NCM applied to the n_top lowest-energy replicas */
    int32_t mis_trials;     /* randomised greedy MIS constructions per NCM */
    int32_t win_short, win_long;                       /* 25, 40 in the paper */
    int32_t max_distinct_short, max_distinct_long;     /* 3, 5 in the paper */
    double reheat_factor;   /* 0.8 in the paper */
    int64_t target_cut;     /* MC*: stop once M* >= target; < 0 none */
    uint64_t seed;          /* Philox key */
    int32_t restart_reinit; /* 1: a restart re-randomises the population */
    int32_t resample;       /* 1 PAMC; 0 independent chains (SA baseline) */
    int32_t K;              /* Potts labels; 0 means 3 */
    double gamma;           /* softmax noisy argmax: sigma <- argmax_c (P_c - gamma U_c),
                               U_c uniform on [0, 1); finite, >= 0 */
} pamc_params;

/* Optional device allocator (e.g. a framework's caching allocator).  Must be
 * set before any handle is created; NULL restores cudaMalloc/cudaFree. */
typedef void *(*pamc_alloc_fn)(size_t bytes, int device, void *stream, void *ctx);
typedef void (*pamc_free_fn)(void *ptr, int device, void *stream, void *ctx);
pamc_status pamc_set_allocator(pamc_alloc_fn alloc, pamc_free_fn free_fn, void *ctx);

/* Create a handle for a sparse Max-Cut instance given as symmetric CSR on the
 * HOST (row_ptr[n+1], col[nnz], w[nnz]; Algorithm 1's coupling-matrix input).
 * The arrays are validated and copied; the caller keeps ownership.
 * Limits: 1 <= n < 2^24, |w| <= 127, max_i sum_j |w_ij| <= 127 (the field
 * range held by the sweep kernels), else PAMC_ERR_RANGE.  Max-Cut runs keep
 * a replica group's spin words in shared memory while they fit (4n bytes)
 * and in device memory beyond; Max-3-Cut runs need 8n bytes of shared memory
 * per group (pamc_init returns PAMC_ERR_RANGE beyond).  Asymmetric input
 * gives PAMC_ERR_ASYM, a self loop PAMC_ERR_DIAG.  stream is a cudaStream_t
 * (NULL = legacy default stream) on device cuda_device. */
pamc_status pamc_create_csr(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const int32_t *w, int cuda_device, void *stream, pamc_handle *out);

/* Create a handle for a dense Max-Cut instance: w is n*n int8 row-major,
 * symmetric with zero diagonal, either in host memory (w_on_device = 0) or
 * in device memory of cuda_device (w_on_device = 1; only read during the
 * call).  Entries must lie in {-1, 0, +1}, else PAMC_ERR_RANGE. */
pamc_status pamc_create_dense(int32_t n, const int8_t *w, int w_on_device, int cuda_device,
                              void *stream, pamc_handle *out);

/* Set the run parameters, allocate the population and draw the random
 * initial population (Algorithm 1, Initialization).  1 <= R <= 1,048,576:
 * up to 16,384 replicas the population step runs in one CTA, above in
 * several kernels with the prefix sums in device memory (the same results),
 * where a Max-Cut run with cluster moves takes at most 16,384 targets
 * (n_top; PAMC_ERR_RANGE beyond).  Batches take members of up to 16,384.
 * Asynchronous. */
pamc_status pamc_init(pamc_handle h, const pamc_params *p);

/* Enqueue nsteps iterations of Algorithm 1 (asynchronous; iterations after
 * the target cut is reached do nothing). */
pamc_status pamc_step(pamc_handle h, int32_t nsteps);

/* Wait for the handle's stream and report device-side errors. */
pamc_status pamc_sync(pamc_handle h);

/* pamc_init + pamc_step(p->steps) + pamc_sync. */
pamc_status pamc_run(pamc_handle h, const pamc_params *p);

/* Best cut M* so far and its configuration (HOST buffer of n int8, may be
 * NULL).  Ising spins are returned with spin 0 = +1; Potts labels renamed in
 * order of first appearance.  Synchronises the stream. */
pamc_status pamc_best(pamc_handle h, int64_t *cut, int8_t *spins);

/* Current population and the last step's resampling, into HOST buffers
 * (any may be NULL): spins[R*n], E[R] (energies), parents[R] (old replica
 * index of each new slot), counts[R] (copies of each old replica).
 * Synchronises the stream. */
pamc_status pamc_state(pamc_handle h, int8_t *spins, int64_t *E, int32_t *parents,
                       int32_t *counts);

/* Controller state: iv[10] = t, z, cycle, cooldown, enable_cm, done,
 * NCM applied in the last iteration, history length, spins flipped by NCM so
 * far, largest |dE| across an NCM; dv[2] = beta, Delta.  Synchronises. */
pamc_status pamc_control_state(pamc_handle h, int64_t *iv, double *dv);

/* The rest of Algorithm 1's state, so that a run can be continued or
 * checked elsewhere from step t: hist (caller array of 64 int64, may be
 * NULL) receives the recent-progress history of M* that the stagnation
 * windows read, oldest first, and *hist_len its length; *mstar (may be
 * NULL) the best cut so far, INT64_MIN before the first iteration.
 * Synchronises. */
pamc_status pamc_control_history(pamc_handle h, int64_t *hist, int32_t *hist_len, int64_t *mstar);

/* Number of this library's kernels launched on the handle so far. */
int64_t pamc_launch_count(pamc_handle h);

/* Launch shape the sparse sweep of an initialised run uses: replica groups
 * per CTA (four replicas each; eight on 4-bit lanes, see pamc_sweep_mode),
 * warps per group, and lanes that share one position: Ising runs on ELL
 * schedules split a vertex's couplings over 1-32 lanes; Max-3-Cut runs take
 * lane pairs with the cascaded sampler on ELL schedules (each lane one
 * Philox call, half the couplings and two replicas' decisions) and quads
 * with the softmax sampler (one replica each); 1 otherwise.  Set by
 * pamc_init from the schedule's level widths, or by the environment variable
 * PAMC_SWEEP_CFG="gpc,wpg[,lpv]".  The shape changes speed only, never
 * results.  PAMC_ERR_STATE before pamc_init or for dense runs. */
pamc_status pamc_sweep_shape(pamc_handle h, int *groups_per_cta, int *warps_per_group, int *lanes_per_vertex);

/* How the sparse Ising sweeps of an initialised run keep the local fields
 * (Eq. 3): *mode = 0 pulled from the neighbours' spins at every visit over
 * the CSR rows, 1 the same over position-indexed (ELL) rows, plus 4 when the
 * replica groups' spin words are in device memory rather than shared memory
 * (groups too large for shared memory, or PAMC_SWEEP_GLOBAL=1), 2 kept in
 * shared memory and updated on every flip (push; chosen by the environment
 * variable PAMC_SWEEP_PUSH=1 for instances with max_i sum_j |w_ij| <= 63,
 * ELL rows, one lane per vertex, at least one sweep).  Plus 8 when the
 * fields take 16-bit lanes (max_i sum_j |w_ij| > 127), plus 16 when a word
 * holds eight replicas on 4-bit lanes (ELL rows, one lane per vertex, spin
 * words in shared memory, at least one sweep, and either sum_j |w_ij| <= 7
 * per vertex on rows of width 4 or 8, or at most 15 over each vertex's first
 * eight nonzero couplings in CSR order and over the rest, on rows up to 16
 * wide; off with PAMC_SWEEP_NIBBLE=0).  Speed only, never results.
 * PAMC_ERR_STATE before pamc_init or for dense or Potts runs. */
pamc_status pamc_sweep_mode(pamc_handle h, int *mode);

/* Sweep statistics.  pamc_set_sweep_timing(h, 1) makes every following
 * sweep launch of the handle (sparse or dense) record a CUDA event pair on
 * the handle's stream around it (the stream is waited for once every 1024
 * launches).  pamc_sweep_stats synchronises and returns, in any non-NULL
 * argument: *flips = replica spins the sparse Ising sweeps changed since
 * pamc_init (0 for dense and Potts runs); *launches and *ms = the sweep
 * launches timed since the last call and their summed device time, which
 * the call then resets. */
pamc_status pamc_set_sweep_timing(pamc_handle h, int on);
pamc_status pamc_sweep_stats(pamc_handle h, int64_t *flips, int64_t *launches, double *ms);

/* W = sum_{i<j} w_ij of the instance (cut = (W - E)/2). */
int64_t pamc_weight_sum(pamc_handle h);

/* Copy the last error message of h (or of the last failed create when h is
 * NULL) into buf. */
pamc_status pamc_last_error(pamc_handle h, char *buf, size_t len);

/* Replace the current population with caller values (host, R rows of n:
 * +-1 for Ising, labels 0..K-1 for Potts), e.g. a warm start.  The energies,
 * and for dense instances the fields H = J S (the full recompute), are
 * recomputed from the definition.  PAMC_ERR_RANGE for a value out of range,
 * PAMC_ERR_STATE once the run reached its target.  Synchronises. */
pamc_status pamc_set_population(pamc_handle h, const int8_t *spins);
/* Dense instances: coupling rows the sweeps' field updates gathered (one per
 * position that flipped in at least one replica; the rows a block's flips
 * need) and positions visited, both summed since pamc_init.  An update reads
 * the gathered rows over every field slice, so rows x n bytes is the sweep's
 * J traffic below the n^2 bytes of one full read per sweep.  PAMC_ERR_ARG for
 * sparse handles.  Synchronises. */
pamc_status pamc_dense_rows(pamc_handle h, int64_t *rows_gathered, int64_t *positions_visited);
/* Dense instances: the local fields H[r][k] = sum_j J_kj s_j of the current
 * population as the device holds them (R rows of n int32, caller-owned).
 * PAMC_ERR_ARG for sparse handles, which keep no field array. */
pamc_status pamc_fields(pamc_handle h, int32_t *H);
/* Diversity of the current population (Suppl., Hamming distance of
 * replicas): for every pair of replicas r < r', d = the number of spins in
 * which they differ, corrected for the global flip symmetry of Max-Cut as
 * dc = min(d, n - d).  hist (caller array of n/2 + 1 int64, floor division)
 * receives hist[k] = the number of pairs with dc = k, *sum the sum of dc over
 * all R(R-1)/2 pairs, so the mean normalised distance is
 * sum / (R(R-1)/2 * n).  Synchronises the handle's stream; allocates scratch
 * of R * ceil(n/32) words.  Ising (kind 0) runs, sparse or dense;
 * PAMC_ERR_ARG for Potts. */
pamc_status pamc_hamming(pamc_handle h, int64_t *hist, int64_t *sum);
/* Lineage of the current population (Sec. III.D, genealogy of the resampled
 * population): family[r] (caller array of R int32) = the slot of the initial
 * population, or of the last re-initialised one after a restart, that slot r
 * descends from through the resampling parent maps (NCM keeps the family).
 * *n_families (may be NULL) = the number of distinct families alive. */
pamc_status pamc_lineage(pamc_handle h, int32_t *family, int32_t *n_families);
void pamc_destroy(pamc_handle h);

/* ---- Batches: many independent instances advanced together ----
 * Not in the paper: a serving extension.  A batch advances every member by
 * one iteration of Algorithm 1 per step (resampling, tables, cluster
 * moves, sweeps, controller, a restart's re-draw) with one launch per kernel
 * type, the sweep launched once per
 * size class of n with its own shape, so uneven instances share the GPU.
 * Each launch reads the member's step index from the member's device-side
 * controller, so one step's launches are captured into a CUDA graph once per
 * change of membership and replayed.  A member computes exactly what
 * pamc_step computes for it alone (same random streams, orders, tables and
 * controller): its spins, energies, parents, counts and best cut are
 * identical in and out of the batch.
 * Members: initialised sparse handles of Max-Cut (kind 0, either rule,
 * with or without the stagnation controller and its cluster moves) or
 * Max-3-Cut with the cascaded sampler (kind 1, rule 0), restarts with or
 * without re-draws, field ranges up to 127 and populations up to 16,384;
 * others are refused with PAMC_ERR_ARG.  A member must stay alive and must
 * not be stepped or re-initialised on its own while it is in the batch.  The batch runs on its
 * own stream (the one given, or one it creates when stream is NULL); read a
 * member's results (pamc_best, pamc_state) after pamc_batch_retire returned
 * it or after pamc_batch_sync. */
typedef struct pamc_batch_s *pamc_batch;

/* Device bytes of a sparse handle running with p: the instance (CSR) plus
 * what pamc_init allocates (two spin buffers, energies, resampling weights,
 * parents, counts, the schedule ring of 16 steps, the threshold table, NCM
 * buffers, the controller).  For admission by HBM footprint; 0 for a null argument or a
 * dense handle. */
size_t pamc_footprint(pamc_handle h, const pamc_params *p);
/* stream: a cudaStream_t, or NULL for a new non-blocking stream. */
pamc_status pamc_batch_create(int cuda_device, void *stream, pamc_batch *out);
/* Add an initialised handle (tops up its schedule ring and waits for its
 * stream).  Takes effect at the next pamc_batch_step. */
pamc_status pamc_batch_add(pamc_batch b, pamc_handle h);
/* Enqueue nsteps batch steps (asynchronous).  Members that completed
 * p->steps iterations do nothing. */
pamc_status pamc_batch_step(pamc_batch b, int32_t nsteps);
/* Remove up to max_out members that completed their iterations and write
 * them to out, after waiting for the batch stream; returns how many, or -1
 * on error (null batch, out NULL with max_out > 0, CUDA error). */
int32_t pamc_batch_retire(pamc_batch b, pamc_handle *out, int32_t max_out);
/* Size class of an n-spin member: 0 for n <= 2048, 1 for n <= 8192, 2 above. */
int pamc_size_class(int32_t n);
/* Launch shape of the batched sweep for one size class: replica groups (of
 * four replicas) per CTA and warps per group, groups * warps <= 32.  Where the
 * class's largest member needs it, fewer groups per CTA are used so that the
 * spins fit shared memory.  The shape changes speed only, never results.
 * Takes effect at the next pamc_batch_step.  PAMC_ERR_ARG when out of range. */
pamc_status pamc_batch_set_shape(pamc_batch b, int size_class, int groups_per_cta, int warps_per_group);
pamc_status pamc_batch_get_shape(pamc_batch b, int size_class, int *groups_per_cta, int *warps_per_group);
/* Lanes that share one vertex's couplings in the batched Ising sweep of a size
 * class (1, 2 or 4; default 1), for members on ELL schedules.  Speed only,
 * never results.  PAMC_ERR_ARG for another value or class. */
pamc_status pamc_batch_set_lanes(pamc_batch b, int size_class, int lanes_per_vertex);
pamc_status pamc_batch_get_lanes(pamc_batch b, int size_class, int *lanes_per_vertex);
/* Where the batched Ising sweep of a size class keeps each replica group's
 * spin words: 0 shared memory (default), 1 device memory (a buffer of the
 * member's, allocated at the next pamc_batch_step; then one lane per vertex
 * and no shared-memory limit on n or on groups per SM).  Members whose groups
 * do not fit shared memory use device memory in any class.  Speed only,
 * never results.  PAMC_ERR_ARG for a bad class. */
pamc_status pamc_batch_set_placement(pamc_batch b, int size_class, int global_spins);
pamc_status pamc_batch_get_placement(pamc_batch b, int size_class, int *global_spins);
int32_t pamc_batch_size(pamc_batch b);      /* members, finished or not */
int32_t pamc_batch_active(pamc_batch b);    /* members with steps left */
int64_t pamc_batch_launch_count(pamc_batch b);  /* kernel launches enqueued */
int64_t pamc_batch_graph_builds(pamc_batch b);  /* CUDA graphs captured */
pamc_status pamc_batch_sync(pamc_batch b);
pamc_status pamc_batch_last_error(pamc_batch b, char *buf, size_t len);
void pamc_batch_destroy(pamc_batch b);

/* ---- Checkpoints ----
 * pamc_save writes the whole state of a run at the start of its next
 * iteration -- the parameters, the controller of Algorithm 1 (beta, Delta,
 * z, cycle, cooldown, flags, the M* history, M*, counters), the population
 * and its energies, the last iteration's parents and copy counts, the
 * lineage and the best configuration -- into a HOST buffer of *size bytes
 * (buf = NULL: only *size is set; capacity too small: PAMC_ERR_RANGE).
 * pamc_load re-initialises a handle of the SAME instance (checked against
 * n, the couplings and W; PAMC_ERR_ARG otherwise) from such a buffer; the
 * run then continues exactly as the uninterrupted one, since every random
 * draw is keyed by the step index.  Both synchronise; the caller owns the
 * buffer.  Split populations (pamc_shard_*) are refused (PAMC_ERR_STATE). */
pamc_status pamc_save(pamc_handle h, void *buf, size_t capacity, size_t *size);
pamc_status pamc_load(pamc_handle h, const void *buf, size_t size);

/* ---- One population split over several processes (one GPU each) ----
 * The population step of Algorithm 1 (Eq. 1-2) is global over the R
 * replicas, so a population split over nranks processes exchanges once per
 * iteration: every process gathers all R energies, computes the same
 * parent map and controller decisions from them, and receives the parent
 * replicas of its slots that live elsewhere.  Process `rank` owns slots
 * [rank R/nranks, (rank + 1) R/nranks); R must be a multiple of 4 nranks.
 * The random draws are keyed by each replica's index in the whole
 * population, so the split run equals pamc_step on one handle with the same
 * parameters, bit for bit (spins, energies, parents, counts, controller, M*).
 * The library makes no collective call: the caller moves the data
 * (all-gather of energies, all-to-all of replica rows), in the order below,
 * on the handle's stream or synchronised with it.  One iteration:
 *   pamc_shard_energies -> all-gather E_own into E_all (slot order)
 *   pamc_shard_resample(E_all) -> parent map -> pamc_shard_plan
 *   pamc_shard_pack -> all-to-all of rows (send_counts / recv_counts)
 *   pamc_shard_sweep -> all-gather E_own into E_all
 *   pamc_shard_control(E_all)
 * (the first all-gather may reuse the last one when no restart redraws the
 * population: p->z_rst == 0 or p->restart_reinit == 0).  Sparse and dense
 * instances (dense: at most 64 replicas per process).  pamc_step,
 * pamc_set_population, pamc_hamming and batches
 * refuse a split handle; pamc_state returns its own slots; the NCM counters
 * of pamc_control_state count its own slots. */

/* Own slots of process `rank`: *base = rank * R / nranks, *count = R /
 * nranks.  PAMC_ERR_ARG unless 0 <= rank < nranks and R % (4 nranks) == 0.
 * Host only. */
pamc_status pamc_shard_range(int32_t R, int32_t nranks, int32_t rank, int32_t *base, int32_t *count);

/* pamc_init for this process's share (same parameters on every process,
 * p->R the whole population).  Draws the own slots of the initial
 * population. */
pamc_status pamc_shard_init(pamc_handle h, const pamc_params *p, int32_t rank, int32_t nranks);

/* Copy the own slots' current energies (count int64) to E_own (DEVICE). */
pamc_status pamc_shard_energies(pamc_handle h, int64_t *E_own);

/* The population step (reweighting by Delta beta, systematic resampling,
 * NCM target choice; Eq. 1-2 and Algorithm 1) on E_all (DEVICE, R int64:
 * every process's energies in slot order).  parent (HOST, R int32)
 * receives the parent map: slot m copies old replica parent[m].
 * Synchronises the stream. */
pamc_status pamc_shard_resample(pamc_handle h, const int64_t *E_all, int32_t *parent);

/* Host only: the exchange that parent implies for process `rank`.
 * send_counts[nranks]: own replicas to send to each process (0 to itself);
 * send_rows (capacity R - R/nranks): their own-row indices (0 .. count-1),
 * process by process in rank order, ascending within a process.
 * recv_counts[nranks]: replicas received from each process, arriving in rank
 * order, ascending within a process.  local_parent[count]: the source row
 * of each own slot's parent: an own row (< count), or count + its position
 * among the received rows.  PAMC_ERR_RANGE on a parent outside [0, R). */
pamc_status pamc_shard_plan(int32_t R, int32_t nranks, int32_t rank, const int32_t *parent,
                            int32_t *send_counts, int32_t *send_rows, int32_t *recv_counts,
                            int32_t *local_parent);

/* Gather the nrows own replicas rows[] (HOST, own-row indices) into sendbuf
 * (DEVICE, nrows * n int8, caller-owned) for the all-to-all.  Asynchronous. */
pamc_status pamc_shard_pack(pamc_handle h, const int32_t *rows, int32_t nrows, int8_t *sendbuf);

/* Copy the own slots' parents (local_parent: HOST, from pamc_shard_plan;
 * imports: DEVICE, nimports received rows of n int8), apply the cluster
 * moves of the own NCM targets, and run the S sweeps of the own slots
 * (Algorithm 1).  E_all must still hold the energies given to
 * pamc_shard_resample.  E_own (DEVICE, count int64, may be NULL) receives
 * the own energies after the sweeps.  Asynchronous. */
pamc_status pamc_shard_sweep(pamc_handle h, const int64_t *E_all, const int32_t *local_parent,
                             const int8_t *imports, int32_t nimports, int64_t *E_own);

/* M* and the controller (Algorithm 1) on E_all (DEVICE, R int64: the
 * energies after the sweeps, all processes); a restart that re-initialises
 * redraws the own slots, and E_own (DEVICE, may be NULL) receives their
 * energies (unchanged without a restart).  Asynchronous. */
pamc_status pamc_shard_control(pamc_handle h, const int64_t *E_all, int64_t *E_own);

/* M* (the same on every process) and, when this process holds it (*owned =
 * 1), its configuration (HOST n int8, as pamc_best).  Synchronises. */
pamc_status pamc_shard_best(pamc_handle h, int64_t *cut, int8_t *spins, int32_t *owned);

/* Size limits of pamc_sweeps_noalloc and the bytes of device memory its
 * file-scope scratch array takes on every GPU that loads the library. */
#define PAMC_NOALLOC_MAX_N 32768
#define PAMC_NOALLOC_MAX_NNZ 262144
#define PAMC_NOALLOC_MAX_SWEEPS 8
#define PAMC_NOALLOC_MAX_R 16384
#define PAMC_NOALLOC_SCRATCH_BYTES 5377280

/* S sweeps (heat-bath rule = 0 or Metropolis rule = 1) of an Ising
 * population at a fixed beta, with no device or host allocation -- for
 * callers that cannot call cudaMalloc (code that may only use the buffers it
 * is handed: a plug-in inside a framework that owns all device memory, or a
 * loop where allocation is forbidden).  The paper has no counterpart; the
 * result is bit-identical to S sweeps of pamc_step on the same population at
 * step index t without resampling (same Philox keys, same sweep orders).
 * Inputs and outputs are DEVICE pointers owned by the caller: the CSR of the
 * Max-Cut weights (row_ptr[n+1], col[nnz], w[nnz]; symmetric, no diagonal,
 * |w| <= 127), H >= max_i sum_j |w_ij| (<= 127), spins_in and spins_out
 * (R*n int8, +1/-1, replica-major; may be the same buffer) and E_out (R
 * energies H(s) = -sum_{i<j} J_ij s_i s_j of the result).  In-place use
 * (spins_in == spins_out) is supported because the sweep reads each replica
 * group's rows completely into shared memory, in the CTA that later writes
 * them, before any write.  err (optional) receives a one-line message.
 * Limits: n <= PAMC_NOALLOC_MAX_N, nnz <= PAMC_NOALLOC_MAX_NNZ,
 * sweeps <= PAMC_NOALLOC_MAX_SWEEPS, R <= PAMC_NOALLOC_MAX_R; larger sizes
 * return PAMC_ERR_RANGE before any device work.  An invalid instance returns
 * PAMC_ERR_ARG / ASYM / DIAG / RANGE after a validation kernel, before any
 * kernel indexes through it; symmetry is checked as a multiset (a neighbour
 * listed twice in one row must be listed twice in the other).
 * Scratch: one static device array of PAMC_NOALLOC_SCRATCH_BYTES per GPU,
 * held from library load until process exit, shared by every call on that
 * GPU and keeping the last call's contents (the call resets what must start
 * fresh).  Calls whose device work overlaps on one GPU (different streams or
 * threads) race on it: serialise them.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the process.  A cudaDeviceReset while the
 * library is loaded is not supported (the kept address would be stale).
 * Each call waits for its
 * stream twice: after validating the instance and before returning. */
pamc_status pamc_sweeps_noalloc(int32_t n, int32_t nnz, const int32_t *row_ptr, const int32_t *col,
                                const int32_t *w, int32_t H, int32_t rule, int32_t R,
                                int32_t sweeps, double beta, uint64_t seed, int32_t t,
                                const int8_t *spins_in, int8_t *spins_out, int64_t *E_out,
                                void *stream, char *err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif
