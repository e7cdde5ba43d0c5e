/*
 * pamc_oracle.h -- plain, slow, single-threaded CPU restatement of augmented
 * Population Annealing Monte Carlo (Khan, Redding, Shukla, "Leveraging
 * Population Dynamics to Steer Efficient Search in Large-Scale Combinatorial
 * Optimization").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the checker for the CUDA path:
 * only tests, the smoke entry point and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header or table with the CUDA library.
 *
 * Every function follows the paper's text step by step (section / equation /
 * algorithm cited beside it) with plain loops; where the paper is silent or
 * ambiguous the reading taken is stated beside the function.
 *
 * Every function is pinned by a test against something fixed outside the
 * oracle (known answers, libm, closed forms, exhaustive enumeration, exact
 * Boltzmann distributions, invariants, hand-built populations), including
 * the initial population and its restart re-draw (uniform, independent,
 * re-keyed) and the choice of cluster-move targets (lowest energy, ties to
 * the lower slot).  What no pin can fix are the readings where the paper is
 * silent, stated beside each function: the NCM defaults (MIS trials, n top
 * replicas, cooldown), that a restart re-draws the population, and the beta
 * factor of Eq. 8.
 */
#ifndef PAMC_ORACLE_H
#define PAMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Random-stream tags (upper 8 bits of counter word 3). */
enum { ORC_TAG_INIT = 1, ORC_TAG_PERM = 2, ORC_TAG_FLIP = 3, ORC_TAG_RESAMPLE = 4, ORC_TAG_NCM = 5 };

/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11: 10 rounds of the Philox S-box over a 4x32-bit
 * counter with a 2x32-bit key bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Deterministic exp in binary64: Cody-Waite range reduction x = k ln2 + r,
 * |r| <= ln2/2, then the degree-13 Taylor polynomial of e^r by Horner's rule
 * with explicit fused multiply-adds, then scaling by 2^k.  Returns 0 for
 * x < -707 and +inf for x > 709.  Every operation is correctly rounded, so
 * any IEEE-754 implementation of the same steps gives the same bits. */
double orc_det_exp(double x);

/* round(x) for x >= 0 with halves rounded up, computed as floor + fraction
 * test so that it is exact for every binary64 input. */
uint64_t orc_round_nonneg(double x);

/* Heat-bath threshold (Eq. 4): T(h) = round(2^32 / (1 + det_exp(-2 beta h))),
 * s <- +1 iff u < T(h), u a 32-bit uniform draw.  Value in [0, 2^32]. */
uint64_t orc_thr_heatbath(double beta, int64_t h);
/* Metropolis threshold for an energy change dE of the proposed single flip:
 * 2^32 if dE <= 0 else round(2^32 det_exp(-beta dE)). */
uint64_t orc_thr_metropolis(double beta, int64_t dE);
/* Cascaded three-state sampler thresholds (Suppl. S3, Eq. S10-S15) on the
 * Eq. 8 target P(k) ~ exp(beta syn_k):
 *   b1: P(label 0) = 1 / (1 + e^{beta a} + e^{beta b}),  a = syn1-syn0, b = syn2-syn0
 *   b2: P(label 1 | not 0) = 1 / (1 + e^{beta c}),        c = syn2-syn1 */
uint64_t orc_thr_potts_b1(double beta, int64_t a, int64_t b);
uint64_t orc_thr_potts_b2(double beta, int64_t c);

/* Random permutation of 0..n-1 shared by all replicas for (t, sweep):
 * vertices sorted by the 32-bit key Philox((k, sweep, t, PERM<<24))[0],
 * equal keys by vertex index (Sec. III.A: spins updated once per sweep in a
 * randomised order). */
void orc_permutation(int32_t n, uint64_t seed, int32_t t, int32_t sweep, int32_t *perm);

/* Systematic resampling (Eq. 1-2) of R replicas with integer energies E,
 * signed increment delta, energy scale escale (1 for Ising, 1/2 for Potts)
 * and step index t.  Writes parent[m] for each new slot m (non-decreasing)
 * and the copy count of each old replica.  Returns 0 on success. */
int orc_resample(int32_t R, const int64_t *E, double delta, double escale, uint64_t seed,
                 int32_t t, int32_t *parent, int32_t *count);

/* ---- Whole Algorithm 1 on a CSR instance ---- */

typedef struct {
    int32_t kind;            /* 0 Max-Cut / Ising, 1 Max-K-Cut / K-state Potts */
    int32_t rule;            /* Ising: 0 heat-bath (Eq. 4), 1 Metropolis;
                                Potts: 0 cascaded sampler (K = 3), 2 softmax noisy argmax */
    int32_t R, sweeps, steps;
    double beta0, beta1;     /* linear increment dbeta = (beta1-beta0)/(steps-1) */
    int32_t stagnation;      /* 0 conventional PAMC, 1 Algorithm 1 controller */
    int32_t z_rst;           /* restart after this many iterations; <= 0 never */
    int32_t cooldown_tau, n_top, mis_trials, win_short, win_long, max_distinct_short, max_distinct_long;
    double reheat_factor;
    int64_t target_cut;      /* stop once M* >= target; < 0 none */
    uint64_t seed;
    int32_t restart_reinit;
    int32_t resample;        /* 1 PAMC; 0 independent chains (the SA baseline) */
    int32_t K;               /* Potts labels (3 for the cascaded sampler; 2..8 softmax) */
    double gamma;            /* softmax noisy argmax: noise amplitude */
} orc_params;

/* Softmax noisy-argmax label choice (Sec. III.F, Eq. 8-9, first Potts update):
 * P_k = exp(beta syn_k) / sum_m exp(beta syn_m), new label =
 * argmax_k (P_k - gamma U_k), U_k = u[k] / 2^32.  Decided in binary32 with
 * round-to-nearest operations in this order: d_k = max_m syn_m - syn_k,
 * e_k = (float) det_exp(-(beta * d_k)), S = e_0 + ... + e_{K-1} (left to
 * right), P_k = e_k / S, U_k = (float) u[k] * 2^-32,
 * v_k = P_k - (float) gamma * U_k; the first maximal k wins. */
int32_t orc_softmax_pick(int32_t K, const int32_t *syn, double beta, double gamma, const uint32_t *u);

typedef struct orc_state orc_state;

/* Controller state of Algorithm 1 (z, cycle, beta, Delta, cooldown,
 * enable-cluster-move and the recent M* history). */
#define ORC_HIST_MAX 64
typedef struct {
    int32_t z, cycle, cooldown, enable_cm, hist_len;
    double beta, delta;
    int64_t hist[ORC_HIST_MAX];
} orc_ctl;

/* Everything Algorithm 1 does after the sweeps and the M* update: record M*,
 * apply the adaptive temperature rule (Sec. III.C) when cooldown = 0 and the
 * history is full, then restart (returns 1) or advance z and beta (returns 0). */
int orc_control(orc_ctl *c, const orc_params *p, double dbeta, int64_t mstar);

/* The couplings are J_ij = -w_ij for Max-Cut weights w (symmetric CSR, no
 * diagonal).  Returns NULL on invalid input. */
orc_state *orc_create(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                      const orc_params *p);
void orc_destroy(orc_state *st);
/* Runs up to nsteps iterations of Algorithm 1; returns the number run
 * (fewer once the target cut is reached). */
int32_t orc_step(orc_state *st, int32_t nsteps);

/* Accessors (copies into caller buffers). */
void orc_get_spins(const orc_state *st, int8_t *out);          /* R*n */
void orc_get_fields(const orc_state *st, int32_t *out);        /* Ising R*n ; Potts R*n*3 */
void orc_get_energy(const orc_state *st, int64_t *out);        /* R */
void orc_get_parents(const orc_state *st, int32_t *parent, int32_t *count); /* last step */
void orc_get_best(const orc_state *st, int64_t *mstar, int8_t *spins);  /* canonical form */
/* iv[10] = t, z, cycle, cooldown, enable_cm, done, ncm applied in the last
 * iteration, history length, spins flipped by NCM so far, largest |dE| seen
 * across an NCM flip;  dv[2] = beta, delta */
void orc_get_ctl(const orc_state *st, int64_t *iv, double *dv);
int64_t orc_weight_sum(const orc_state *st);
/* Overwrite the population (spins) and recompute fields and energies from
 * the definition; used by tests that start from a hand-built state. */
void orc_set_spins(orc_state *st, const int8_t *spins);

/* ---- Step replay from a state reached elsewhere (parity at full size) ----
 * orc_set_state loads a whole state of Algorithm 1 -- step index t, the
 * controller (z, cycle, cooldown, enable_cm, beta, Delta and the M* history
 * in ctl), the best cut so far mstar (INT64_MIN for none) and its
 * configuration best (n values, may be NULL), and the population spins
 * (R*n) -- and recomputes fields and energies from the definition.  The
 * NCM counters restart at zero.  The next iterations run from it as from a
 * state the oracle reached itself. */
void orc_set_state(orc_state *st, int32_t t, const orc_ctl *ctl, int64_t mstar, const int8_t *best,
                   const int8_t *spins);
/* Sampled sweeps: in the following iterations only the replicas with
 * mask[r] != 0 are swept; every other replica takes its configuration after
 * the sweeps from spins_after (R*n, results computed elsewhere), with its
 * fields and energy recomputed from the definition.  Resampling, cluster
 * moves, M*, the best configuration and the controller then run on the
 * whole population exactly as in Algorithm 1, so an iteration of a large
 * population can be checked with the sweeps of a sample only.  mask NULL
 * switches the mode off. */
void orc_set_sweep_replay(orc_state *st, const uint8_t *mask, const int8_t *spins_after);
/* Ising: replica spins the sweeps changed since orc_create (a visit whose
 * new spin differs from the old one counts once). */
int64_t orc_sweep_flips(const orc_state *st);
/* The M* history of the stagnation windows, oldest first (hist_len values
 * of orc_get_ctl). */
void orc_get_history(const orc_state *st, int64_t *hist);
/* The slots that took the cluster move in the last iteration, in the order
 * chosen (lowest (energy, slot) first); *count = 0 when none did. */
void orc_get_ncm_targets(const orc_state *st, int32_t *targets, int32_t *count);

/* ---- One population split over several processes ----
 * orc_step runs orc_iter_population (resampling at the new beta, then the
 * cluster moves), orc_iter_sweeps (the S sweeps) and orc_iter_control (M*,
 * the controller, a restart's re-draw) in turn.  A process that holds slots
 * [lo, hi) of the population calls orc_set_own(lo, hi): the cluster moves
 * and sweeps then touch those slots only (the NCM target list still covers
 * the whole population), and the best configuration is copied only when
 * the replica holding the new M* is an own slot (orc_best_owned).  Between
 * the parts it loads the energies of every process (orc_set_energies, R
 * values: resampling, the choice of NCM targets and M* read them) and the
 * replicas it received (orc_set_rows: spins, with fields and energies
 * recomputed from the definition). */
void orc_iter_population(orc_state *st);
void orc_iter_sweeps(orc_state *st);
void orc_iter_control(orc_state *st);
void orc_set_own(orc_state *st, int32_t lo, int32_t hi);
void orc_set_energies(orc_state *st, const int64_t *E);
void orc_set_rows(orc_state *st, int32_t r0, int32_t count, const int8_t *rows);
int32_t orc_best_owned(const orc_state *st);

/* Energy from the definition (i<j pairs), used by the pins. */
int64_t orc_energy_ising(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *J,
                         const int8_t *s);
int64_t orc_energy_potts(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *J,
                         const int8_t *sigma);

/* Non-local cluster move (Sec. III.C, first bullet) on one replica: spins s,
 * fields h (Ising).  Applies mis_trials randomised greedy MIS constructions
 * over the iso-sites and flips the largest.  Returns the number flipped. */
int32_t orc_ncm_replica(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *J,
                        int8_t *s, int32_t *h, int32_t mis_trials, uint64_t seed, int32_t t,
                        int32_t r);

#ifdef __cplusplus
}
#endif
#endif
